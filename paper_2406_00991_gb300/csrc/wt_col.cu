// Column (sigma-direction) kernels: one thread owns one vertical column and
// keeps it in registers; the Chebyshev matrices sit in shared memory padded
// to MAXM x MAXM with zeros, so every loop has compile-time bounds.
//
//  k_op_cols      the sigma part of A_{a,b} (Eq. 1_chain, poissonp, bcpdneu):
//                 P_s = D p, G = (P_x + sx_b P_s, P_y + sy_b P_s, Z_b P_s),
//                 part = sx_a D G_x + sy_a D G_y + Z_a Z_b D P_s (interior),
//                 p (surface row), h_x G_x + h_y G_y + Z_b P_s (bottom row).
//  k_smooth_cols  damped block-Jacobi update x += omega sum_class B_class^{-1} r_class
//                 (Sec. 4.3, Nyquist-split column blocks).
//  k_col_matrix   out = M in along sigma (Chebyshev transfers of Sec. 4.2, filter).
//  k_block_inverse  builds and inverts the (Nz+1)^2 diagonal block of every
//                 column by Gauss-Jordan with partial pivoting, one warp per column.
#include "wt_internal.h"

#include <algorithm>

namespace wt {

template <typename T, int MAXM>
__device__ __forceinline__ void load_padded(T* sM, const T* __restrict__ M, int M1) {
  for (int i = threadIdx.x; i < MAXM * MAXM; i += blockDim.x) {
    const int r = i / MAXM, c = i - r * MAXM;
    sM[i] = (r < M1 && c < M1) ? M[r * M1 + c] : T(0);
  }
}

// Every thread keeps the input column of a contraction in registers (static
// indices, inner loop unrolled) and walks the output rows with a rolled loop;
// intermediate columns go through shared memory laid out [row][thread].
template <typename T, int MAXM, int DIM>
__global__ void __launch_bounds__(128) k_op_cols(LevelView<T> L, const T* __restrict__ p,
                                                 const T* __restrict__ Px, const T* __restrict__ Py,
                                                 T* __restrict__ Gx, T* __restrict__ Gy,
                                                 T* __restrict__ part) {
  __shared__ T sD[MAXM * MAXM];
  __shared__ T ssig[MAXM];
  __shared__ T sPs[MAXM * 128];
  const int M1 = L.M1;
  load_padded<T, MAXM>(sD, L.D, M1);
  for (int i = threadIdx.x; i < MAXM; i += blockDim.x) ssig[i] = i < M1 ? L.sigma[i] : T(0);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.ncols) return;
  const int t = threadIdx.x;
  const long nc = L.ncols;
  const T* meta = L.meta;
  T p0;
  {
    T v[MAXM];
#pragma unroll
    for (int k = 0; k < MAXM; ++k) v[k] = (k < M1) ? p[k * nc + c] : T(0);
    p0 = v[0];
#pragma unroll 1
    for (int m = 0; m < M1; ++m) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < MAXM; ++k) acc += sD[m * MAXM + k] * v[k];
      sPs[m * 128 + t] = acc;                        // P_s = D p
    }
  }
  const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
  const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
  const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
  const T HX = meta[M_HX * nc + c];
  T ps[MAXM], gx[MAXM];
#pragma unroll
  for (int k = 0; k < MAXM; ++k) {
    if (k < M1) {
      ps[k] = sPs[k * 128 + t];
      gx[k] = Px[k * nc + c] + (AXb - ssig[k] * BXb) * ps[k];   // G_x
      Gx[k * nc + c] = gx[k];
    } else {
      ps[k] = T(0);
      gx[k] = T(0);
    }
  }
  T gy[DIM == 3 ? MAXM : 1];
  T AYa = 0, BYa = 0, HY = 0;
  if constexpr (DIM == 3) {
    const T AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
    AYa = meta[M_AYa * nc + c];
    BYa = meta[M_BYa * nc + c];
    HY = meta[M_HY * nc + c];
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      if (k < M1) {
        gy[k] = Py[k * nc + c] + (AYb - ssig[k] * BYb) * ps[k];  // G_y
        Gy[k * nc + c] = gy[k];
      } else {
        gy[k] = T(0);
      }
    }
  }
  const T ZZ = Za * Zb;
  part[c] = p0;                                                  // surface row
  {
    // bottom row n . Grad_b p; indexed through shared / global memory so that
    // the register arrays keep static indices only
    const int mb = M1 - 1;
    const T psb = sPs[mb * 128 + t];
    const T sb = ssig[mb];
    T bot = HX * (Px[mb * nc + c] + (AXb - sb * BXb) * psb) + Zb * psb;
    if constexpr (DIM == 3)
      bot += HY * (Py[mb * nc + c] + (meta[M_AYb * nc + c] - sb * meta[M_BYb * nc + c]) * psb);
    part[mb * nc + c] = bot;                                     // bottom row
  }
#pragma unroll 1
  for (int m = 1; m < M1 - 1; ++m) {
    T q = 0, s = 0, qy = 0;
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      const T d = sD[m * MAXM + k];
      q += d * gx[k];
      s += d * ps[k];
      if constexpr (DIM == 3) qy += d * gy[k];
    }
    T out = (AXa - ssig[m] * BXa) * q + ZZ * s;
    if constexpr (DIM == 3) out += (AYa - ssig[m] * BYa) * qy;
    part[m * nc + c] = out;
  }
}

template <typename T, int MAXM, int DIM>
__global__ void __launch_bounds__(128) k_smooth_cols(LevelView<T> L, const T* __restrict__ r,
                                                     const T* __restrict__ rhoX,
                                                     const T* __restrict__ rhoY,
                                                     const T* __restrict__ rhoXY,
                                                     const T* __restrict__ Binv, int nclass,
                                                     T* __restrict__ x, T omega, int first) {
  __shared__ T sE[MAXM * 128];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.ncols) return;
  const int t = threadIdx.x;
  const int M1 = L.M1;
  const long nc = L.ncols;
  const int jx = c % L.Nx, jy = c / L.Nx;
  const T sx = (jx & 1) ? T(-1) : T(1);
  const T sy = (jy & 1) ? T(-1) : T(1);
  const long blk = (long)M1 * M1;
  // residual split by Nyquist class: 0 regular, 1 x-Nyquist, 2 y-Nyquist, 3 both
  constexpr int NC = DIM == 2 ? 2 : 4;
#pragma unroll 1
  for (int cls = 0; cls < NC; ++cls) {
    T v[MAXM];
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      T val = 0;
      if (k < M1) {
        T rNx = 0, rNy = 0, rNN = 0;
        if constexpr (DIM == 2) {
          if (rhoX) rNx = rhoX[k] * sx;
        } else {
          const T cxy = rhoXY ? rhoXY[k] : T(0);
          rNN = cxy * sx * sy;
          if (rhoX) rNx = (rhoX[k * L.Ny + jy] - cxy * sy) * sx;
          if (rhoY) rNy = (rhoY[k * L.Nx + jx] - cxy * sx) * sy;
        }
        if (cls == 0) val = r[k * nc + c] - rNx - rNy - rNN;
        else if (cls == 1) val = rNx;
        else if (cls == 2) val = rNy;
        else val = rNN;
      }
      v[k] = val;
    }
    const T* B = Binv + cls * blk * nc + c;
#pragma unroll 1
    for (int m = 0; m < M1; ++m) {
      T e = 0;
      const T* Bm = B + (long)m * M1 * nc;
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k < M1) e += Bm[(long)k * nc] * v[k];
      sE[m * 128 + t] = (cls == 0 ? T(0) : sE[m * 128 + t]) + e;
    }
  }
#pragma unroll 1
  for (int m = 0; m < M1; ++m) {
    const T xo = first ? T(0) : x[m * nc + c];
    x[m * nc + c] = xo + omega * sE[m * 128 + t];
  }
  (void)nclass;
}

template <typename T, int MAXM>
__global__ void __launch_bounds__(128) k_col_matrix(const T* __restrict__ M, int Mo, int Mi,
                                                    const T* __restrict__ in, T* __restrict__ out,
                                                    int ncols, int accumulate) {
  __shared__ T sM[MAXM * MAXM];
  for (int i = threadIdx.x; i < MAXM * MAXM; i += blockDim.x) {
    const int r = i / MAXM, k = i - r * MAXM;
    sM[i] = (r < Mo && k < Mi) ? M[r * Mi + k] : T(0);
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long nc = ncols;
  T v[MAXM];
#pragma unroll
  for (int k = 0; k < MAXM; ++k) v[k] = (k < Mi) ? in[k * nc + c] : T(0);
#pragma unroll 1
  for (int m = 0; m < Mo; ++m) {
    T acc = 0;
#pragma unroll
    for (int k = 0; k < MAXM; ++k) acc += sM[m * MAXM + k] * v[k];
    if (accumulate) acc += out[m * nc + c];
    out[m * nc + c] = acc;
  }
}

// Diagonal column block of A_{a,b} (the same expression the oracle pins
// against its dense assembly): interior rows
//   cdiag I + (sx_a AX_b + sy_a AY_b + Z_a Z_b) D^2 - (sx_a BX_b + sy_a BY_b) D diag(sigma) D,
// surface row e_0, bottom row (h_x sx_b + h_y sy_b + Z_b) D[Nz, :].
template <typename T>
__global__ void __launch_bounds__(128) k_block_inverse(LevelView<T> L, T* __restrict__ Binv,
                                                       int nclass, T cxx, T cyy, int* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M1 = L.M1;
  const int W = 2 * M1 + 1;                 // padded row of the augmented matrix
  T* A = reinterpret_cast<T*>(smraw) + (threadIdx.x >> 5) * (M1 * W);
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  const long nc = L.ncols;
  const long blk = (long)M1 * M1;
  for (long task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < nc * nclass;
       task += warps_total) {
    const int c = (int)(task % nc), cls = (int)(task / nc);
    const int ix = cls & 1, iy = (cls >> 1) & 1;
    const T cdiag = (ix ? T(0) : cxx) + (iy ? T(0) : cyy);
    const T* meta = L.meta;
    const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
    const T AYa = meta[M_AYa * nc + c], BYa = meta[M_BYa * nc + c];
    const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
    const T AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
    const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
    const T HX = meta[M_HX * nc + c], HY = meta[M_HY * nc + c];
    const T sbot = L.sigma[M1 - 1];
    const T cbot = HX * (AXb - sbot * BXb) + HY * (AYb - sbot * BYb) + Zb;
    for (int i = lane; i < M1 * M1; i += 32) {
      const int m = i / M1, k = i - m * M1;
      T v;
      if (m == 0) {
        v = (k == 0) ? T(1) : T(0);
      } else if (m == M1 - 1) {
        v = cbot * L.D[m * M1 + k];
      } else {
        const T s = L.sigma[m];
        const T sxa = AXa - s * BXa, sya = AYa - s * BYa;
        v = (sxa * AXb + sya * AYb + Za * Zb) * L.D2[m * M1 + k] -
            (sxa * BXb + sya * BYb) * L.DSD[m * M1 + k];
        if (m == k) v += cdiag;
      }
      A[m * W + k] = v;
      A[m * W + M1 + k] = (m == k) ? T(1) : T(0);
    }
    __syncwarp();
    bool bad = false;
    for (int piv = 0; piv < M1; ++piv) {
      // pivot search over rows piv..M1-1
      T best = T(-1);
      int bi = piv;
      for (int i = piv + lane; i < M1; i += 32) {
        const T a = fabs(A[i * W + piv]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (!(best > T(0)) || !isfinite(best)) { bad = true; break; }
      if (bi != piv) {
        for (int j = lane; j < 2 * M1; j += 32) {
          const T t0 = A[piv * W + j];
          A[piv * W + j] = A[bi * W + j];
          A[bi * W + j] = t0;
        }
      }
      __syncwarp();
      const T inv = T(1) / A[piv * W + piv];
      __syncwarp();
      for (int j = lane; j < 2 * M1; j += 32) A[piv * W + j] *= inv;
      __syncwarp();
      for (int i = lane; i < M1; i += 32) {
        if (i == piv) continue;
        const T f = A[i * W + piv];
        if (f != T(0)) {
          for (int j = 0; j < 2 * M1; ++j) A[i * W + j] -= f * A[piv * W + j];
        }
      }
      __syncwarp();
    }
    if (bad) {
      if (lane == 0) atomicOr(flag, 1);
    }
    for (int i = lane; i < M1 * M1; i += 32) {
      const int m = i / M1, k = i - m * M1;
      Binv[(cls * blk + i) * nc + c] = bad ? T(0) : A[m * W + M1 + k];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ launchers
static inline int grid_for(long n, int bs) { return (int)std::max<long>(1, (n + bs - 1) / bs); }

#define WT_MAXM_DISPATCH(M1, CALL)              \
  do {                                          \
    if ((M1) <= 9) { constexpr int MM = 9; CALL; } \
    else if ((M1) <= 17) { constexpr int MM = 17; CALL; } \
    else if ((M1) <= 25) { constexpr int MM = 25; CALL; } \
    else { constexpr int MM = 33; CALL; }       \
  } while (0)

template <typename T>
cudaError_t launch_op_cols(const LevelView<T>& L, const T* p, const T* Px, const T* Py, T* Gx,
                           T* Gy, T* part, cudaStream_t s) {
  const int g = grid_for(L.ncols, 128);
  if (L.Ny == 1) {
    WT_MAXM_DISPATCH(L.M1, (k_op_cols<T, MM, 2><<<g, 128, 0, s>>>(L, p, Px, Py, Gx, Gy, part)));
  } else {
    WT_MAXM_DISPATCH(L.M1, (k_op_cols<T, MM, 3><<<g, 128, 0, s>>>(L, p, Px, Py, Gx, Gy, part)));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_cols(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                               const T* rhoXY, const T* Binv, int nclass, T* x, T omega, int first,
                               cudaStream_t s) {
  const int g = grid_for(L.ncols, 128);
  if (L.Ny == 1) {
    WT_MAXM_DISPATCH(L.M1, (k_smooth_cols<T, MM, 2><<<g, 128, 0, s>>>(L, r, rhoX, rhoY, rhoXY,
                                                                        Binv, nclass, x, omega, first)));
  } else {
    WT_MAXM_DISPATCH(L.M1, (k_smooth_cols<T, MM, 3><<<g, 128, 0, s>>>(L, r, rhoX, rhoY, rhoXY,
                                                                        Binv, nclass, x, omega, first)));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col_matrix(const T* M, int Mo, int Mi, const T* in, T* out, int ncols,
                              int accumulate, cudaStream_t s) {
  const int g = grid_for(ncols, 128);
  const int mm = std::max(Mo, Mi);
  WT_MAXM_DISPATCH(mm, (k_col_matrix<T, MM><<<g, 128, 0, s>>>(M, Mo, Mi, in, out, ncols, accumulate)));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_inverse(const LevelView<T>& L, T* Binv, int nclass, T cxx, T cyy,
                                 int* flag, cudaStream_t s) {
  const int W = 2 * L.M1 + 1;
  const size_t smem = 4 * (size_t)L.M1 * W * sizeof(T);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_block_inverse<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const long tasks = (long)L.ncols * nclass;
  const int g = (int)std::min<long>(std::max<long>(1, (tasks + 3) / 4), 152 * 8);
  k_block_inverse<T><<<g, 128, smem, s>>>(L, Binv, nclass, cxx, cyy, flag);
  return cudaGetLastError();
}

#define WT_INST(T)                                                                              \
  template cudaError_t launch_op_cols<T>(const LevelView<T>&, const T*, const T*, const T*, T*,  \
                                         T*, T*, cudaStream_t);                                 \
  template cudaError_t launch_smooth_cols<T>(const LevelView<T>&, const T*, const T*, const T*,  \
                                             const T*, const T*, int, T*, T, int, cudaStream_t); \
  template cudaError_t launch_col_matrix<T>(const T*, int, int, const T*, T*, int, int,         \
                                            cudaStream_t);                                      \
  template cudaError_t launch_block_inverse<T>(const LevelView<T>&, T*, int, T, T, int*,        \
                                               cudaStream_t);
WT_INST(float)
WT_INST(double)

}  // namespace wt
