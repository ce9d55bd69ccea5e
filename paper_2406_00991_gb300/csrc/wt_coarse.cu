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
#include "wt_dev.cuh"

namespace wt {

__global__ void __launch_bounds__(256) k_coarse_factor(LevelView<double> L, const double* __restrict__ Dx,
                                                      const double* __restrict__ Dy,
                                                      double* __restrict__ LUout, int* __restrict__ piv,
                                                      int* flag) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  coarse_factor_body(L, Dx, Dy, LUout, flag, smraw);
  (void)piv;
}

// x = A^{-1} f (tr = 0) or x = A^{-T} f (tr = 1) with the stored (transposed)
// inverse: one thread per row.
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_solve(int n, const double* __restrict__ AinvT,
                                                     const int* __restrict__ piv, int tr,
                                                     const T* __restrict__ f, T* __restrict__ x) {
  pdl_enter();
  __shared__ double b[128];
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (double)f[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int j = 0; j < n; ++j) acc += AinvT[tr ? i * n + j : j * n + i] * b[j];
    x[i] = (T)acc;
  }
  (void)piv;
}

cudaError_t launch_coarse_factor(const LevelView<double>& L, const double* Dx, const double* Dy,
                                 double* LU, int* piv, int* flag, cudaStream_t s) {
  const int n = L.M1 * L.Ny * L.Nx;
  if (n > 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n * (n + 1) * sizeof(double) + sizeof(int) * (n + 1);
  if (smem > 32 * 1024) {
    cudaError_t e = ensure_dyn_smem((const void*)k_coarse_factor, smem);
    if (e != cudaSuccess) return e;
  }
  return launch_k(k_coarse_factor, dim3(1), dim3(256), smem, s, L, Dx, Dy, LU, piv, flag);
}

template <typename T>
cudaError_t launch_coarse_solve(int n, const double* LU, const int* piv, int tr, const T* f, T* x,
                                cudaStream_t s) {
  return launch_k(k_coarse_solve<T>, dim3(1), dim3(128), 0, s, n, LU, piv, tr, f, x);
}

template cudaError_t launch_coarse_solve<float>(int, const double*, const int*, int, const float*,
                                                float*, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(int, const double*, const int*, int, const double*,
                                                 double*, cudaStream_t);

}  // namespace wt
