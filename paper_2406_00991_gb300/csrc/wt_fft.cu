// Spectral passes along x-rows and y-lines (paper Sec. 3.5 and 4.2):
//   derivative   D f = F^{-1}( i kappa F f ), Nyquist coefficient multiplied by 0
//   resampling   Fourier truncation (restriction) / zero padding (prolongation)
//   filter       exponential cut-off on |n| (Sec. 3.6)
// followed by a fused epilogue (store / add / residual / accumulate) and an
// optional per-row Nyquist coefficient (used by the Nyquist-split smoother).
//
// Design: one CTA transforms `nb` pairs of real rows in shared memory; the
// two real rows of a pair are packed as real and imaginary part of one
// complex sequence.  Every operation above is a real linear map (its
// multiplier is Hermitian), so the real and imaginary parts of the result are
// the results for the two rows.  The transform is a radix-4 (plus one
// radix-2 stage for odd log2 N) Stockham self-sorting FFT with host-computed
// FP64 twiddles staged in shared memory.
#include "wt_dev.cuh"

#include <algorithm>

namespace wt {

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass(RowPass<T> a, int ppc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  rowpass_body<T>(a, ppc, blockIdx.x, gridDim.x, smraw);
}

template <typename T>
cudaError_t launch_rowpass(const RowPass<T>& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  const int Nmax = std::max(a.Nin, a.Nout);
  const int npairs = (a.nrows + 1) / 2;
  int ppc = std::max(1, 1024 / Nmax);
  const int want = (npairs + 303) / 304;     // spread small passes over the SMs
  ppc = std::max(1, std::min(ppc, want));
  const size_t smem = rowpass_smem(a, ppc);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_rowpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int grid = (npairs + ppc - 1) / ppc;
  grid = std::min(grid, 152 * 16);
  return launch_k(k_rowpass<T>, dim3(grid), dim3(256), smem, s, a, ppc);
}

template cudaError_t launch_rowpass<float>(const RowPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass<double>(const RowPass<double>&, cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass_multi(const __grid_constant__ MultiPass<T> m) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int i = 0;
  while (i + 1 < m.n && (int)blockIdx.x >= m.start[i + 1]) ++i;
  const int u = blockIdx.x - m.start[i];
  rowpass_body<T>(m.d[i], 1, u, m.start[i + 1] - m.start[i], smraw);
}

template <typename T>
cudaError_t launch_rowpass_multi(const MultiPass<T>& m0, cudaStream_t s) {
  if (m0.n <= 0) return cudaSuccess;
  if (m0.n > kMaxPasses) return cudaErrorInvalidValue;
  MultiPass<T> m = m0;
  size_t smem = 0;
  m.start[0] = 0;
  for (int i = 0; i < m.n; ++i) {
    const int npairs = (m.d[i].nrows + 1) / 2;
    m.start[i + 1] = m.start[i] + npairs;
    smem = std::max(smem, rowpass_smem(m.d[i], 1));
  }
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_rowpass_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  if (m.start[m.n] <= 0) return cudaSuccess;
  k_rowpass_multi<T><<<m.start[m.n], 256, smem, s>>>(m);
  return cudaGetLastError();
}

template cudaError_t launch_rowpass_multi<float>(const MultiPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass_multi<double>(const MultiPass<double>&, cudaStream_t);

}  // namespace wt
