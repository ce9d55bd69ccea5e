// The lower part of the p-multigrid V-cycle (Algorithm 1) in a single CTA.
//
// On small levels every phase of the V-cycle (smoothing sweep, residual,
// restriction, coarsest solve, prolongation) is a few microseconds of
// latency when launched as its own kernel, but only a few thousand unknowns
// of work.  This kernel runs all levels from l0 down to the coarsest and
// back up inside one CTA: the phases are the same device bodies the
// multi-CTA kernels use (wt_dev.cuh), separated by __syncthreads, with the
// level buffers in global memory (L2-resident at these sizes).  The kernel
// has no inter-CTA dependencies and no waits besides __syncthreads.
#define WT_DEV_RESTRICT
#include "wt_cta.cuh"

#include <algorithm>

namespace wt {

template <typename T, int DIM>
__global__ void __launch_bounds__(512) k_vcycle_tail(TailArgs<T> A) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char sm[];
  vcycle_cta<T, DIM>(A, sm);
}

template <typename T>
cudaError_t launch_vcycle_tail(const TailArgs<T>& a, int dim, cudaStream_t s) {
  cudaError_t e = dim == 3 ? ensure_dyn_smem((const void*)k_vcycle_tail<T, 3>, (size_t)a.smem)
                           : ensure_dyn_smem((const void*)k_vcycle_tail<T, 2>, (size_t)a.smem);
  if (e != cudaSuccess) return e;
  if (dim == 3) return launch_k(k_vcycle_tail<T, 3>, dim3(1), dim3(512), a.smem, s, a);
  return launch_k(k_vcycle_tail<T, 2>, dim3(1), dim3(512), a.smem, s, a);
}

template cudaError_t launch_vcycle_tail<float>(const TailArgs<float>&, int, cudaStream_t);
template cudaError_t launch_vcycle_tail<double>(const TailArgs<double>&, int, cudaStream_t);

}  // namespace wt
