// Coarsest p-multigrid level: direct solve u = A^{-1} f (Algorithm 1, p = 1),
// in FP64 for both solver modes.  The dense A_{a,b} of the level is assembled
// on the device entry by entry from the composite operator and inverted in
// shared memory by one CTA (Gauss-Jordan with partial pivoting, once per
// geometry); every V-cycle then applies the inverse with one thread per row.
//
// Entry of A_{a,b} for row i = (m, y, x) and column j = (m', y', x'), with
// dense per-level D_x, D_y (zero diagonal) and D (d/dsigma):
//  interior m:
//   d_yy' [ d_mm' (D_x D_x)_xx' + (D_x)_xx' sxb(m,y,x') D_mm' ]
//   + sxa(m,y,x) d_yy' [ D_mm' (D_x)_xx' + d_xx' (AXb D^2 - BXb D S D)_mm' ]
//   + d_xx' [ d_mm' (D_y D_y)_yy' + (D_y)_yy' syb(m,y',x) D_mm' ]
//   + sya(m,y,x) d_xx' [ D_mm' (D_y)_yy' + d_yy' (AYb D^2 - BYb D S D)_mm' ]
//   + d_yy' d_xx' Za Zb (D^2)_mm'
//  surface m = 0: identity row;  bottom m = Nz:
//   HX [ d_Nz m' d_yy' (D_x)_xx' + d_yy' d_xx' sxb D_Nz m' ]
//   + HY [ d_Nz m' d_xx' (D_y)_yy' + d_yy' d_xx' syb D_Nz m' ] + d_yy' d_xx' Zb D_Nz m'
// (S = diag(sigma); sxb(m, .) = AXb - sigma_m BXb etc.)
#include "wt_internal.h"

namespace wt {

__global__ void __launch_bounds__(256) k_coarse_factor(LevelView<double> L, const double* __restrict__ Dx,
                                                      const double* __restrict__ Dy,
                                                      double* __restrict__ LUout, int* __restrict__ piv,
                                                      int* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Nx = L.Nx, Ny = L.Ny, M1 = L.M1;
  const int n = M1 * Ny * Nx;
  const int ld = n + 1;
  double* A = reinterpret_cast<double*>(smraw);
  __shared__ int spiv;
  const double* Dxx = Dx + Nx * Nx;
  const double* Dyy = Dy + Ny * Ny;
  const long nc = L.ncols;
  const double* meta = L.meta;
  const double* D = L.D;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    const int m = i / (Ny * Nx), y = (i / Nx) % Ny, x = i % Nx;
    const int mp = j / (Ny * Nx), yp = (j / Nx) % Ny, xp = j % Nx;
    const int c = y * Nx + x;
    const bool sy_ = (y == yp), sx_ = (x == xp), sm_ = (m == mp);
    double v = 0.0;
    if (m == 0) {
      v = (i == j) ? 1.0 : 0.0;
    } else if (m == M1 - 1) {
      const double s = L.sigma[m];
      const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double HX = meta[M_HX * nc + c], HY = meta[M_HY * nc + c];
      const double Zb = meta[M_Zb * nc + c];
      const double Dm = D[m * M1 + mp];
      if (sy_) v += HX * ((mp == m ? Dx[x * Nx + xp] : 0.0) + (sx_ ? sxb * Dm : 0.0));
      if (sx_) v += HY * ((mp == m ? Dy[y * Ny + yp] : 0.0) + (sy_ ? syb * Dm : 0.0));
      if (sx_ && sy_) v += Zb * Dm;
    } else {
      const double s = L.sigma[m];
      const double Dm = D[m * M1 + mp];
      const double AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
      const double AYa = meta[M_AYa * nc + c], BYa = meta[M_BYa * nc + c];
      const double sxa = AXa - s * BXa, sya = AYa - s * BYa;
      const double D2m = L.D2[m * M1 + mp], DSDm = L.DSD[m * M1 + mp];
      if (sy_) {
        const int cp = y * Nx + xp;   // column (y, x')
        const double sxb_p = meta[M_AXb * nc + cp] - s * meta[M_BXb * nc + cp];
        v += (sm_ ? Dxx[x * Nx + xp] : 0.0) + Dx[x * Nx + xp] * sxb_p * Dm;
        v += sxa * Dm * Dx[x * Nx + xp];
      }
      if (sx_) {
        const int cp = yp * Nx + x;   // column (y', x)
        const double syb_p = meta[M_AYb * nc + cp] - s * meta[M_BYb * nc + cp];
        v += (sm_ ? Dyy[y * Ny + yp] : 0.0) + Dy[y * Ny + yp] * syb_p * Dm;
        v += sya * Dm * Dy[y * Ny + yp];
      }
      if (sx_ && sy_) {
        const double AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
        const double AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
        v += sxa * (AXb * D2m - BXb * DSDm) + sya * (AYb * D2m - BYb * DSDm);
        v += meta[M_Za * nc + c] * meta[M_Zb * nc + c] * D2m;
      }
    }
    A[i * ld + j] = v;
  }
  __syncthreads();
  // in-place Gauss-Jordan inversion with row pivoting (the pivot column is
  // overwritten by the inverse's column; row swaps become column swaps at the end)
  __shared__ int perm[128];
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        const double a = fabs(A[i * ld + k]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        spiv = bi;
        perm[k] = bi;
        if (!(best > 0.0) || !isfinite(best)) atomicOr(flag, 2);
      }
    }
    __syncthreads();
    const int p = spiv;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t0 = A[k * ld + j];
        A[k * ld + j] = A[p * ld + j];
        A[p * ld + j] = t0;
      }
      __syncthreads();
    }
    const double inv = 1.0 / A[k * ld + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[k * ld + j] = (j == k ? 1.0 : A[k * ld + j]) * inv;
    __syncthreads();
    // eliminate column k from every other row; column k of those rows becomes -f * inv
    for (int idx = threadIdx.x; idx < (n - 1) * n; idx += blockDim.x) {
      int i = idx / n;
      const int j = idx - i * n;
      if (i >= k) ++i;
      const double f = A[i * ld + k];
      if (j != k) A[i * ld + j] -= f * A[k * ld + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) A[i * ld + k] = -A[i * ld + k] * A[k * ld + k];
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t0 = A[i * ld + k];
        A[i * ld + k] = A[i * ld + p];
        A[i * ld + p] = t0;
      }
    }
    __syncthreads();
  }
  // store the inverse transposed: LUout[j * n + i] = Ainv[i][j] (coalesced solve)
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    LUout[j * n + i] = A[i * ld + j];
  }
}

// x = A^{-1} f with the stored (transposed) inverse: one thread per row.
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_solve(int n, const double* __restrict__ AinvT,
                                                     const int* __restrict__ piv,
                                                     const T* __restrict__ f, T* __restrict__ x) {
  __shared__ double b[128];
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (double)f[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int j = 0; j < n; ++j) acc += AinvT[j * n + i] * b[j];
    x[i] = (T)acc;
  }
  (void)piv;
}

cudaError_t launch_coarse_factor(const LevelView<double>& L, const double* Dx, const double* Dy,
                                 double* LU, int* piv, int* flag, cudaStream_t s) {
  const int n = L.M1 * L.Ny * L.Nx;
  if (n > 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n * (n + 1) * sizeof(double);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_coarse_factor<<<1, 256, smem, s>>>(L, Dx, Dy, LU, piv, flag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(int n, const double* LU, const int* piv, const T* f, T* x,
                                cudaStream_t s) {
  k_coarse_solve<T><<<1, 128, 0, s>>>(n, LU, piv, f, x);
  return cudaGetLastError();
}

template cudaError_t launch_coarse_solve<float>(int, const double*, const int*, const float*, float*,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(int, const double*, const int*, const double*,
                                                 double*, cudaStream_t);

}  // namespace wt
