// Column (sigma-direction) kernels on shared-memory tiles of 16 columns x all
// sigma rows (see TC / RG below).
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

// Column kernels work on tiles of TC consecutive columns x all M1 sigma rows
// held in shared memory ([row][column-in-tile]); thread (rg, tc) of a
// 128-thread CTA owns column tc of the tile and the rows rg, rg+8, rg+16, ...
// so every sigma contraction has M1 x TC independent outputs per CTA and the
// global loads of a warp cover 16 consecutive columns.
constexpr int TC = 16;
constexpr int RG = 8;                 // row groups: 128 threads = RG x TC

template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_op_cols(LevelView<T> L, const T* __restrict__ p,
                                                 const T* __restrict__ Px, const T* __restrict__ Py,
                                                 T* __restrict__ Gx, T* __restrict__ Gy,
                                                 T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M1 = L.M1;
  T* sD = reinterpret_cast<T*>(smraw);            // M1*M1
  T* sP = sD + M1 * M1;                          // p tile
  T* sPs = sP + M1 * TC;                         // D p
  T* sGx = sPs + M1 * TC;                        // G_x (Px on entry)
  T* sGy = sGx + M1 * TC;                        // G_y (Py on entry), 3D only
  const int tc = threadIdx.x % TC, rg = threadIdx.x / TC;
  const long nc = L.ncols;
  const long c0 = (long)blockIdx.x * TC;
  const long c = c0 + tc;
  const bool live = c < nc;
  for (int i = threadIdx.x; i < M1 * M1; i += blockDim.x) sD[i] = L.D[i];
  for (int i = threadIdx.x; i < M1 * TC; i += blockDim.x) {
    const int m = i / TC, cc = i % TC;
    const long col = c0 + cc;
    const bool ok = col < nc;
    sP[i] = ok ? p[m * nc + col] : T(0);
    sGx[i] = ok ? Px[m * nc + col] : T(0);
    if constexpr (DIM == 3) sGy[i] = ok ? Py[m * nc + col] : T(0);
  }
  __syncthreads();
  // P_s = D p
  for (int m = rg; m < M1; m += RG) {
    T acc = 0;
    for (int k = 0; k < M1; ++k) acc += sD[m * M1 + k] * sP[k * TC + tc];
    sPs[m * TC + tc] = acc;
  }
  __syncthreads();
  const T* meta = L.meta;
  const long cm = live ? c : 0;
  const T AXb = meta[M_AXb * nc + cm], BXb = meta[M_BXb * nc + cm];
  const T AXa = meta[M_AXa * nc + cm], BXa = meta[M_BXa * nc + cm];
  const T Za = meta[M_Za * nc + cm], Zb = meta[M_Zb * nc + cm];
  const T HX = meta[M_HX * nc + cm];
  T AYa = 0, BYa = 0, AYb = 0, BYb = 0, HY = 0;
  if constexpr (DIM == 3) {
    AYa = meta[M_AYa * nc + cm]; BYa = meta[M_BYa * nc + cm];
    AYb = meta[M_AYb * nc + cm]; BYb = meta[M_BYb * nc + cm];
    HY = meta[M_HY * nc + cm];
  }
  // G = (P_x + sx_b P_s, P_y + sy_b P_s, .)
  for (int m = rg; m < M1; m += RG) {
    const T s = L.sigma[m];
    const T ps = sPs[m * TC + tc];
    const T gx = sGx[m * TC + tc] + (AXb - s * BXb) * ps;
    sGx[m * TC + tc] = gx;
    if (live) Gx[m * nc + c] = gx;
    if constexpr (DIM == 3) {
      const T gy = sGy[m * TC + tc] + (AYb - s * BYb) * ps;
      sGy[m * TC + tc] = gy;
      if (live) Gy[m * nc + c] = gy;
    }
  }
  __syncthreads();
  const T ZZ = Za * Zb;
  for (int m = rg; m < M1; m += RG) {
    T out;
    if (m == 0) {
      out = sP[tc];                                         // surface row: p
    } else if (m == M1 - 1) {                               // bottom row: n . Grad_b p
      out = HX * sGx[m * TC + tc] + Zb * sPs[m * TC + tc];
      if constexpr (DIM == 3) out += HY * sGy[m * TC + tc];
    } else {
      T q = 0, sum = 0, qy = 0;
      for (int k = 0; k < M1; ++k) {
        const T d = sD[m * M1 + k];
        q += d * sGx[k * TC + tc];
        sum += d * sPs[k * TC + tc];
        if constexpr (DIM == 3) qy += d * sGy[k * TC + tc];
      }
      const T s = L.sigma[m];
      out = (AXa - s * BXa) * q + ZZ * sum;
      if constexpr (DIM == 3) out += (AYa - s * BYa) * qy;
    }
    if (live) part[m * nc + c] = out;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_smooth_cols(LevelView<T> L, const T* __restrict__ r,
                                                     const T* __restrict__ rhoX,
                                                     const T* __restrict__ rhoY,
                                                     const T* __restrict__ rhoXY,
                                                     const T* __restrict__ Binv,
                                                     T* __restrict__ x, T omega, int first) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NC = DIM == 2 ? 2 : 4;
  const int M1 = L.M1;
  T* sR = reinterpret_cast<T*>(smraw);            // [NC][M1][TC] residual parts
  const int tc = threadIdx.x % TC, rg = threadIdx.x / TC;
  const long nc = L.ncols;
  const long c0 = (long)blockIdx.x * TC;
  for (int i = threadIdx.x; i < M1 * TC; i += blockDim.x) {
    const int m = i / TC, cc = i % TC;
    const long col = c0 + cc;
    T rr = 0, rNx = 0, rNy = 0, rNN = 0;
    if (col < nc) {
      rr = r[m * nc + col];
      const int jx = (int)(col % L.Nx), jy = (int)(col / L.Nx);
      const T sx = (jx & 1) ? T(-1) : T(1), sy = (jy & 1) ? T(-1) : T(1);
      if constexpr (DIM == 2) {
        if (rhoX) rNx = rhoX[m] * sx;
      } else {
        const T cxy = rhoXY ? rhoXY[m] : T(0);
        rNN = cxy * sx * sy;
        if (rhoX) rNx = (rhoX[m * L.Ny + jy] - cxy * sy) * sx;
        if (rhoY) rNy = (rhoY[m * L.Nx + jx] - cxy * sx) * sy;
      }
    }
    sR[(0 * M1 + m) * TC + cc] = rr - rNx - rNy - rNN;
    sR[(1 * M1 + m) * TC + cc] = rNx;
    if constexpr (DIM == 3) {
      sR[(2 * M1 + m) * TC + cc] = rNy;
      sR[(3 * M1 + m) * TC + cc] = rNN;
    }
  }
  __syncthreads();
  const long c = c0 + tc;
  if (c >= nc) return;
  const long blk = (long)M1 * M1;
  for (int m = rg; m < M1; m += RG) {
    T e = 0;
#pragma unroll
    for (int cls = 0; cls < NC; ++cls) {
      const T* B = Binv + (cls * blk + (long)m * M1) * nc + c;
      const T* R = sR + cls * M1 * TC + tc;
#pragma unroll 5
      for (int k = 0; k < M1; ++k) e += B[(long)k * nc] * R[k * TC];
    }
    const T xo = first ? T(0) : x[m * nc + c];
    x[m * nc + c] = xo + omega * e;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_col_matrix(const T* __restrict__ M, int Mo, int Mi,
                                                    const T* __restrict__ in, T* __restrict__ out,
                                                    int ncols, int accumulate) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sM = reinterpret_cast<T*>(smraw);            // Mo*Mi
  T* sIn = sM + Mo * Mi;                          // [Mi][TC]
  const int tc = threadIdx.x % TC, rg = threadIdx.x / TC;
  const long nc = ncols;
  const long c0 = (long)blockIdx.x * TC;
  for (int i = threadIdx.x; i < Mo * Mi; i += blockDim.x) sM[i] = M[i];
  for (int i = threadIdx.x; i < Mi * TC; i += blockDim.x) {
    const int k = i / TC, cc = i % TC;
    const long col = c0 + cc;
    sIn[i] = col < nc ? in[k * nc + col] : T(0);
  }
  __syncthreads();
  const long c = c0 + tc;
  if (c >= nc) return;
  for (int m = rg; m < Mo; m += RG) {
    T acc = 0;
    for (int k = 0; k < Mi; ++k) acc += sM[m * Mi + k] * sIn[k * TC + tc];
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

template <typename T>
static cudaError_t set_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t launch_op_cols(const LevelView<T>& L, const T* p, const T* Px, const T* Py, T* Gx,
                           T* Gy, T* part, cudaStream_t s) {
  const int g = grid_for(L.ncols, TC);
  const size_t smem = sizeof(T) * ((size_t)L.M1 * L.M1 + 4 * (size_t)L.M1 * TC);
  if (L.Ny == 1) {
    cudaError_t e = set_smem<T>((const void*)k_op_cols<T, 2>, smem);
    if (e != cudaSuccess) return e;
    k_op_cols<T, 2><<<g, 128, smem, s>>>(L, p, Px, Py, Gx, Gy, part);
  } else {
    cudaError_t e = set_smem<T>((const void*)k_op_cols<T, 3>, smem);
    if (e != cudaSuccess) return e;
    k_op_cols<T, 3><<<g, 128, smem, s>>>(L, p, Px, Py, Gx, Gy, part);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_cols(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                               const T* rhoXY, const T* Binv, int nclass, T* x, T omega, int first,
                               cudaStream_t s) {
  const int g = grid_for(L.ncols, TC);
  const size_t smem = sizeof(T) * (size_t)nclass * L.M1 * TC;
  if (L.Ny == 1)
    k_smooth_cols<T, 2><<<g, 128, smem, s>>>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
  else
    k_smooth_cols<T, 3><<<g, 128, smem, s>>>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col_matrix(const T* M, int Mo, int Mi, const T* in, T* out, int ncols,
                              int accumulate, cudaStream_t s) {
  const int g = grid_for(ncols, TC);
  const size_t smem = sizeof(T) * ((size_t)Mo * Mi + (size_t)Mi * TC);
  k_col_matrix<T><<<g, 128, smem, s>>>(M, Mo, Mi, in, out, ncols, accumulate);
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
