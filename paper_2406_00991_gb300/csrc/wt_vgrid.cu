// The whole p-multigrid V-cycle (Algorithm 1) in one cooperative launch.
//
// Launched as separate kernels, a V-cycle of the 1024 x 24 tank is ~170
// launches of a few microseconds each, most of it launch and drain latency
// rather than work.  Here every CTA of a cooperative (co-resident) grid takes
// its share of each phase - row passes by row pair, column kernels by column
// - and a grid barrier separates the phases (wt_cta.cuh: grid_sync, bounded
// by the SM clock).  The phases are the same device bodies as the
// multi-kernel path.
#define WT_DEV_RESTRICT
#include "wt_cta.cuh"

#include <algorithm>

namespace wt {

template <typename T, int DIM>
__global__ void __launch_bounds__(512, 1) k_vcycle_grid(TailArgs<T> A, GridBar* bar, int* flag) {
  extern __shared__ __align__(16) unsigned char sm[];
  vcycle_grid<T, DIM, GridSync>(A, bar, flag, sm);
}

// The levels from A.l0 down and back up in one thread-block cluster: the
// grid is the cluster, and the phases are separated by the cluster's
// hardware barrier (every CTA runs every phase, so all of them arrive).
template <typename T, int DIM>
__global__ void __launch_bounds__(512, 1) k_vcycle_cluster(TailArgs<T> A) {
  extern __shared__ __align__(16) unsigned char sm[];
  vcycle_grid<T, DIM, ClusterSync>(A, nullptr, nullptr, sm);
}

template <typename T, int DIM>
static cudaError_t launch_cluster_dim(const TailArgs<T>& a, int csize, cudaStream_t s) {
  const void* fn = (const void*)k_vcycle_cluster<T, DIM>;
  cudaError_t e = ensure_dyn_smem(fn, (size_t)a.smem);
  if (e != cudaSuccess) return e;
  if (csize > 8 && (e = ensure_nonportable_cluster(fn)) != cudaSuccess) return e;   // above the portable 8
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = a.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if ((e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_cluster<T, DIM>, &cfg)) != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorInvalidConfiguration;   // this cluster size cannot be resident
  return cudaLaunchKernelEx(&cfg, k_vcycle_cluster<T, DIM>, a);
}

template <typename T>
cudaError_t launch_vcycle_cluster(const TailArgs<T>& a, int dim, int csize, cudaStream_t s) {
  if (csize < 1 || csize > 16) return cudaErrorInvalidValue;
  return dim == 3 ? launch_cluster_dim<T, 3>(a, csize, s) : launch_cluster_dim<T, 2>(a, csize, s);
}

template cudaError_t launch_vcycle_cluster<float>(const TailArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_vcycle_cluster<double>(const TailArgs<double>&, int, int, cudaStream_t);

template <typename T, int DIM>
static cudaError_t launch_dim(const TailArgs<T>& a, GridBar* bar, int* flag, cudaStream_t s) {
  cudaError_t e = ensure_dyn_smem((const void*)k_vcycle_grid<T, DIM>, (size_t)a.smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vcycle_grid<T, DIM>, 512, a.smem)) !=
      cudaSuccess)
    return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;  // one CTA per SM must fit for co-residency
  const int nblocks = nsm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = a.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_vcycle_grid<T, DIM>, a, bar, flag);
}

template <typename T>
cudaError_t launch_vcycle_grid(const TailArgs<T>& a, int dim, GridBar* bar, int* flag, cudaStream_t s) {
  return dim == 3 ? launch_dim<T, 3>(a, bar, flag, s) : launch_dim<T, 2>(a, bar, flag, s);
}

template cudaError_t launch_vcycle_grid<float>(const TailArgs<float>&, int, GridBar*, int*, cudaStream_t);
template cudaError_t launch_vcycle_grid<double>(const TailArgs<double>&, int, GridBar*, int*, cudaStream_t);

}  // namespace wt
