// CTA-level building blocks: one CTA runs whole phases of the method (an
// operator apply, a smoothing sweep, a V-cycle) with __syncthreads between
// the phases, on level buffers in global memory.  Used by the single-CTA
// V-cycle kernel (wt_tail.cu) and the batched persistent tank kernel
// (wt_batch.cu).  Include after defining WT_DEV_RESTRICT as empty: these
// phases read buffers written earlier in the same launch.
#pragma once

#include "wt_dev.cuh"

namespace wt {

template <typename T>
__device__ RowPass<T> tpass(const LevelView<T>& V, const T* in, T* out, int nrows, int Nin, int logNin,
                            int Nout, int logNout, int op) {
  RowPass<T> a;
  a.in = in;
  a.out = out;
  a.nrows = nrows;
  a.Nin = Nin;
  a.Nout = Nout;
  a.logNin = logNin;
  a.logNout = logNout;
  a.op = op;
  a.kscale = T(6.283185307179586476925286766559) / V.L;
  a.tw = V.tw;
  a.logNtw = V.logNtw;
  return a;
}

template <typename T>
__device__ void t_rowpass(const RowPass<T>& a0, int smem, unsigned char* sm) {
  RowPass<T> a = a0;
  const int npairs = (a.nrows + 1) >> 1;
  int ppc = npairs;
  while (ppc > 1 && rowpass_smem(a, ppc) > (size_t)smem) ppc = (ppc + 1) / 2;
  if (rowpass_smem(a, ppc) > (size_t)smem) a.prefetch = 0;   // large rows: epilogue from global
  rowpass_body<T>(a, ppc, 0, 1, sm);
  __syncthreads();
}

// out = A x (f == nullptr) or f - A x, with Nyquist coefficients of out.
template <typename T, int DIM>
__device__ void t_apply_op(const TailLevel<T>& L, const T* x, T* out, const T* f, bool nyq, int smem,
                           unsigned char* sm) {
  const LevelView<T>& V = L.V;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  if (DIM == 2) {
    t_rowpass(tpass(V, x, L.t1, V.M1, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV), smem, sm);
    opcols_body<T, 2>(V, x, L.t1, nullptr, L.t2, nullptr, L.t3, 0, 1, sm);
    RowPass<T> a = tpass(V, L.t2, out, V.M1, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV);
    a.skip_bc = 1;
    a.Ny = 1;
    a.M1 = V.M1;
    a.add = L.t3;
    a.rhs = f;
    a.epi = f ? EPI_RESID : EPI_ADD;
    a.nyq = nyq ? L.rhoX : nullptr;
    t_rowpass(a, smem, sm);
  } else {
    t_rowpass(tpass(V, x, L.t1, V.M1 * V.Ny, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV), smem, sm);
    RowPass<T> y1 = tpass(V, x, L.t4, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_DERIV);
    y1.ylines = 1;
    y1.Nxl = V.Nx;
    t_rowpass(y1, smem, sm);
    opcols_body<T, 3>(V, x, L.t1, L.t4, L.t2, L.t5, L.t3, 0, 1, sm);
    RowPass<T> a = tpass(V, L.t2, L.t6, V.M1 * V.Ny, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV);
    a.skip_bc = 1;
    a.Ny = V.Ny;
    a.M1 = V.M1;
    a.add = L.t3;
    a.epi = EPI_ADD;
    t_rowpass(a, smem, sm);
    RowPass<T> b = tpass(V, L.t5, out, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_DERIV);
    b.ylines = 1;
    b.Nxl = V.Nx;
    b.skip_bc = 1;
    b.M1 = V.M1;
    b.add = L.t6;
    b.rhs = f;
    b.epi = f ? EPI_RESID : EPI_ADD;
    b.nyq = nyq ? L.rhoY : nullptr;
    t_rowpass(b, smem, sm);
    if (nyq) {
      nyquist_body<T>(out, V.M1 * V.Ny, V.Nx, L.rhoX, w, nw);
      __syncthreads();
      nyquist_body<T>(L.rhoX, V.M1, V.Ny, L.rhoXY, w, nw);
      __syncthreads();
    }
  }
}

// Nyquist coefficients of a right-hand side (first sweep of a level).
template <typename T, int DIM>
__device__ void t_nyquist_of(const TailLevel<T>& L, const T* f, int smem, unsigned char* sm) {
  const LevelView<T>& V = L.V;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  if (DIM == 2) {
    nyquist_body<T>(f, V.M1, V.Nx, L.rhoX, w, nw);
    __syncthreads();
  } else {
    RowPass<T> b = tpass(V, f, L.t6, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_NONE);
    b.ylines = 1;
    b.Nxl = V.Nx;
    b.nyq = L.rhoY;
    t_rowpass(b, smem, sm);
    nyquist_body<T>(f, V.M1 * V.Ny, V.Nx, L.rhoX, w, nw);
    __syncthreads();
    nyquist_body<T>(L.rhoX, V.M1, V.Ny, L.rhoXY, w, nw);
    __syncthreads();
  }
}

template <typename T, int DIM>
__device__ void t_sweep(const TailArgs<T>& A, const TailLevel<T>& L, T* x, const T* f, int smem,
                        unsigned char* sm) {
  t_apply_op<T, DIM>(L, x, L.r, f, true, smem, sm);
  smooth_any<T, DIM>(L.V, L.r, L.rhoX, DIM == 3 ? L.rhoY : nullptr, DIM == 3 ? L.rhoXY : nullptr,
                      L.Binv, x, A.omega, 0, 0, 1, sm);
}

// The V-cycle from level A.l0 down to the coarsest and back, in this CTA.
template <typename T, int DIM>
__device__ void vcycle_cta(const TailArgs<T>& A, unsigned char* sm) {
  const int smem = A.smem;
  const int nl = A.nl, l0 = A.l0;
  // ---- down: pre-smoothing, residual, restriction
  for (int l = l0; l < nl - 1; ++l) {
    const TailLevel<T>& L = A.lv[l];
    const TailLevel<T>& C = A.lv[l + 1];
    const LevelView<T>& V = L.V;
    const T* f = (l == l0) ? A.f0 : L.f;
    T* x = (l == l0) ? A.x0 : L.x;
    const bool fnyq = (l == l0) ? (A.f0_nyq != 0) : (A.lv[l - 1].V.Nx == V.Nx);
    const T* resid = f;
    if (A.nu1 > 0) {
      if (fnyq) t_nyquist_of<T, DIM>(L, f, smem, sm);
      smooth_any<T, DIM>(V, f, fnyq ? L.rhoX : nullptr, (fnyq && DIM == 3) ? L.rhoY : nullptr,
                          (fnyq && DIM == 3) ? L.rhoXY : nullptr, L.Binv, x, A.omega, 1, 0, 1, sm);
      for (int i = 1; i < A.nu1; ++i) t_sweep<T, DIM>(A, L, x, f, smem, sm);
      t_apply_op<T, DIM>(L, x, L.r, f, false, smem, sm);     // r = f - A u
      resid = L.r;
    } else {
      for (long i = threadIdx.x; i < V.n; i += blockDim.x) x[i] = T(0);
      __syncthreads();
    }
    const T* cur = resid;
    if (C.V.Nx != V.Nx) {
      t_rowpass(tpass(V, cur, L.t4, V.M1 * V.Ny, V.Nx, V.logNx, C.V.Nx, C.V.logNx, XOP_RESAMPLE), smem, sm);
      cur = L.t4;
      if (DIM == 3) {
        RowPass<T> a = tpass(V, cur, L.t5, V.M1 * C.V.Nx, V.Ny, V.logNy, C.V.Ny, C.V.logNy, XOP_RESAMPLE);
        a.ylines = 1;
        a.Nxl = C.V.Nx;
        t_rowpass(a, smem, sm);
        cur = L.t5;
      }
    }
    colmat_body<T>(L.Rsig, C.V.M1, V.M1, cur, C.f, C.V.ncols, 0, 0, 1, sm);
  }
  // ---- coarsest level: x = A^{-1} f (FP64 inverse)
  {
    const TailLevel<T>& Cc = A.lv[nl - 1];
    const T* f = (nl - 1 == l0) ? A.f0 : Cc.f;
    T* x = (nl - 1 == l0) ? A.x0 : Cc.x;
    const int n = (int)Cc.V.n;
    double* b = reinterpret_cast<double*>(sm);
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (double)f[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += A.AinvT[j * n + i] * b[j];
      x[i] = (T)acc;
    }
    __syncthreads();
  }
  // ---- up: prolongation + correction, post-smoothing
  for (int l = nl - 2; l >= l0; --l) {
    const TailLevel<T>& L = A.lv[l];
    const TailLevel<T>& C = A.lv[l + 1];
    const LevelView<T>& V = L.V;
    const T* f = (l == l0) ? A.f0 : L.f;
    T* x = (l == l0) ? A.x0 : L.x;
    if (C.V.Nx == V.Nx) {
      colmat_body<T>(L.Psig, V.M1, C.V.M1, C.x, x, V.ncols, 1, 0, 1, sm);
    } else {
      colmat_body<T>(L.Psig, V.M1, C.V.M1, C.x, L.t4, C.V.ncols, 0, 0, 1, sm);
      const T* cur = L.t4;
      if (DIM == 3) {
        RowPass<T> a = tpass(V, cur, L.t5, V.M1 * C.V.Nx, C.V.Ny, C.V.logNy, V.Ny, V.logNy, XOP_RESAMPLE);
        a.ylines = 1;
        a.Nxl = C.V.Nx;
        t_rowpass(a, smem, sm);
        cur = L.t5;
      }
      RowPass<T> a = tpass(V, cur, x, V.M1 * V.Ny, C.V.Nx, C.V.logNx, V.Nx, V.logNx, XOP_RESAMPLE);
      a.epi = EPI_ACC;
      t_rowpass(a, smem, sm);
    }
    for (int i = 0; i < A.nu2; ++i) t_sweep<T, DIM>(A, L, x, f, smem, sm);
  }
}

}  // namespace wt

// ---------------------------------------------------------------------------
// Grid-wide versions: every CTA of a cooperative launch (or of a launch that
// is one thread-block cluster) takes its share of a phase (unit blockIdx.x of
// gridDim.x), and the phases are separated by a grid (or cluster) barrier.  The barrier is release/acquire at GPU scope: arrivals
// publish the CTA's writes, the spin reads the generation with ld.acquire so
// that later loads see the other CTAs' writes.  Every wait is bounded by the
// SM clock; a barrier that gives up sets the shared abort flag, and any CTA
// that sees it returns false so the kernel ends within one more phase.
namespace wt {

constexpr long long kBarrierCycles = 2000000000LL;   // about one second at 2 GHz

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrive with one acquire-release add on the monotonic counter; the barrier of this
// arrival completes when the counter reaches the next multiple of the grid
// size, which the CTA waits for with acquire loads.
__device__ inline bool grid_sync(GridBar* b, int* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long nb = gridDim.x;
    const unsigned long long old = atom_add_acq_rel_u64(&b->count, 1ull);
    const unsigned long long target = (old / nb + 1ull) * nb;
    if (old + 1ull != target) {
      const long long lim = b->limit > 0 ? b->limit : kBarrierCycles;
      const long long t0 = clock64();
      unsigned polls = 0;
      while (ld_acquire_u64(&b->count) < target) {
        if (clock64() - t0 > lim) {
          atomicExch(&b->abort, 1);
          atomicOr(flag, 32);
          ok = 0;
          break;
        }
        if ((++polls & 63u) == 0u && ld_relaxed_s32(&b->abort)) {
          ok = 0;
          break;
        }
      }
    } else if (ld_relaxed_s32(&b->abort)) {
      ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Phase separators: the bounded grid barrier of a cooperative launch, or
// the hardware barrier of a thread-block cluster when the grid is a single
// cluster (release / acquire at cluster scope; no spin in this code).
struct GridSync {
  __device__ static bool sync(GridBar* b, int* flag) { return grid_sync(b, flag); }
};
struct ClusterSync {
  __device__ static bool sync(GridBar*, int*) {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    return true;
  }
};

template <typename T, typename S>
__device__ inline bool g_rowpass(const RowPass<T>& a0, int smem, unsigned char* sm, GridBar* b, int* flag) {
  RowPass<T> a = a0;
  if (rowpass_smem(a, 1) > (size_t)smem) a.prefetch = 0;
  rowpass_body<T>(a, 1, blockIdx.x, gridDim.x, sm);
  return S::sync(b, flag);
}

template <typename T, int DIM, typename S>
__device__ bool g_apply_op(const TailLevel<T>& L, const T* x, T* out, const T* f, bool nyq, int smem,
                           unsigned char* sm, GridBar* b, int* flag) {
  const LevelView<T>& V = L.V;
  const int nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + (threadIdx.x >> 5), gws = gridDim.x * nw;
  if (DIM == 2) {
    if (!g_rowpass<T, S>(tpass(V, x, L.t1, V.M1, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV), smem, sm, b, flag))
      return false;
    opcols_body<T, 2>(V, x, L.t1, nullptr, L.t2, nullptr, L.t3, blockIdx.x, gridDim.x, sm);
    if (!S::sync(b, flag)) return false;
    RowPass<T> a = tpass(V, L.t2, out, V.M1, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV);
    a.skip_bc = 1;
    a.Ny = 1;
    a.M1 = V.M1;
    a.add = L.t3;
    a.rhs = f;
    a.epi = f ? EPI_RESID : EPI_ADD;
    a.nyq = nyq ? L.rhoX : nullptr;
    return g_rowpass<T, S>(a, smem, sm, b, flag);
  }
  if (!g_rowpass<T, S>(tpass(V, x, L.t1, V.M1 * V.Ny, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV), smem, sm, b, flag))
    return false;
  RowPass<T> y1 = tpass(V, x, L.t4, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_DERIV);
  y1.ylines = 1;
  y1.Nxl = V.Nx;
  if (!g_rowpass<T, S>(y1, smem, sm, b, flag)) return false;
  opcols_body<T, 3>(V, x, L.t1, L.t4, L.t2, L.t5, L.t3, blockIdx.x, gridDim.x, sm);
  if (!S::sync(b, flag)) return false;
  RowPass<T> a = tpass(V, L.t2, L.t6, V.M1 * V.Ny, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV);
  a.skip_bc = 1;
  a.Ny = V.Ny;
  a.M1 = V.M1;
  a.add = L.t3;
  a.epi = EPI_ADD;
  if (!g_rowpass<T, S>(a, smem, sm, b, flag)) return false;
  RowPass<T> c = tpass(V, L.t5, out, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_DERIV);
  c.ylines = 1;
  c.Nxl = V.Nx;
  c.skip_bc = 1;
  c.M1 = V.M1;
  c.add = L.t6;
  c.rhs = f;
  c.epi = f ? EPI_RESID : EPI_ADD;
  c.nyq = nyq ? L.rhoY : nullptr;
  if (!g_rowpass<T, S>(c, smem, sm, b, flag)) return false;
  if (nyq) {
    nyquist_body<T>(out, V.M1 * V.Ny, V.Nx, L.rhoX, gw, gws);
    if (!S::sync(b, flag)) return false;
    nyquist_body<T>(L.rhoX, V.M1, V.Ny, L.rhoXY, gw, gws);
    if (!S::sync(b, flag)) return false;
  }
  return true;
}

template <typename T, int DIM, typename S>
__device__ bool g_nyquist_of(const TailLevel<T>& L, const T* f, int smem, unsigned char* sm, GridBar* b,
                             int* flag) {
  const LevelView<T>& V = L.V;
  const int nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + (threadIdx.x >> 5), gws = gridDim.x * nw;
  if (DIM == 2) {
    nyquist_body<T>(f, V.M1, V.Nx, L.rhoX, gw, gws);
    return S::sync(b, flag);
  }
  RowPass<T> c = tpass(V, f, L.t6, V.M1 * V.Nx, V.Ny, V.logNy, V.Ny, V.logNy, XOP_NONE);
  c.ylines = 1;
  c.Nxl = V.Nx;
  c.nyq = L.rhoY;
  if (!g_rowpass<T, S>(c, smem, sm, b, flag)) return false;
  nyquist_body<T>(f, V.M1 * V.Ny, V.Nx, L.rhoX, gw, gws);
  if (!S::sync(b, flag)) return false;
  nyquist_body<T>(L.rhoX, V.M1, V.Ny, L.rhoXY, gw, gws);
  return S::sync(b, flag);
}

template <typename T, int DIM, typename S>
__device__ bool g_sweep(const TailArgs<T>& A, const TailLevel<T>& L, T* x, const T* f, int smem,
                        unsigned char* sm, GridBar* b, int* flag) {
  if (!g_apply_op<T, DIM, S>(L, x, L.r, f, true, smem, sm, b, flag)) return false;
  smooth_any<T, DIM>(L.V, L.r, L.rhoX, DIM == 3 ? L.rhoY : nullptr, DIM == 3 ? L.rhoXY : nullptr, L.Binv, x,
                      A.omega, 0, blockIdx.x, gridDim.x, sm);
  return S::sync(b, flag);
}

// The V-cycle of vcycle_cta with every phase spread over the grid.
template <typename T, int DIM, typename S>
__device__ void vcycle_grid(const TailArgs<T>& A, GridBar* b, int* flag, unsigned char* sm) {
  const int smem = A.smem;
  const int nl = A.nl, l0 = A.l0;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x, gts = (long)gridDim.x * blockDim.x;
  for (int l = l0; l < nl - 1; ++l) {
    const TailLevel<T>& L = A.lv[l];
    const TailLevel<T>& C = A.lv[l + 1];
    const LevelView<T>& V = L.V;
    const T* f = (l == l0) ? A.f0 : L.f;
    T* x = (l == l0) ? A.x0 : L.x;
    const bool fnyq = (l == l0) ? (A.f0_nyq != 0) : (A.lv[l - 1].V.Nx == V.Nx);
    const T* resid = f;
    if (A.nu1 > 0) {
      if (fnyq && !g_nyquist_of<T, DIM, S>(L, f, smem, sm, b, flag)) return;
      smooth_any<T, DIM>(V, f, fnyq ? L.rhoX : nullptr, (fnyq && DIM == 3) ? L.rhoY : nullptr,
                          (fnyq && DIM == 3) ? L.rhoXY : nullptr, L.Binv, x, A.omega, 1, blockIdx.x, gridDim.x, sm);
      if (!S::sync(b, flag)) return;
      for (int i = 1; i < A.nu1; ++i)
        if (!g_sweep<T, DIM, S>(A, L, x, f, smem, sm, b, flag)) return;
      if (!g_apply_op<T, DIM, S>(L, x, L.r, f, false, smem, sm, b, flag)) return;
      resid = L.r;
    } else {
      for (long i = gt; i < V.n; i += gts) x[i] = T(0);
      if (!S::sync(b, flag)) return;
    }
    const T* cur = resid;
    if (C.V.Nx != V.Nx) {
      if (!g_rowpass<T, S>(tpass(V, cur, L.t4, V.M1 * V.Ny, V.Nx, V.logNx, C.V.Nx, C.V.logNx, XOP_RESAMPLE), smem, sm, b,
                     flag))
        return;
      cur = L.t4;
      if (DIM == 3) {
        RowPass<T> a = tpass(V, cur, L.t5, V.M1 * C.V.Nx, V.Ny, V.logNy, C.V.Ny, C.V.logNy, XOP_RESAMPLE);
        a.ylines = 1;
        a.Nxl = C.V.Nx;
        if (!g_rowpass<T, S>(a, smem, sm, b, flag)) return;
        cur = L.t5;
      }
    }
    colmat_body<T>(L.Rsig, C.V.M1, V.M1, cur, C.f, C.V.ncols, 0, blockIdx.x, gridDim.x, sm);
    if (!S::sync(b, flag)) return;
  }
  {
    // coarsest level: x = A^{-1} f with the FP64 inverse, one CTA
    const TailLevel<T>& Cc = A.lv[nl - 1];
    const T* f = (nl - 1 == l0) ? A.f0 : Cc.f;
    T* x = (nl - 1 == l0) ? A.x0 : Cc.x;
    const int n = (int)Cc.V.n;
    if (blockIdx.x == 0) {
      double* bb = reinterpret_cast<double*>(sm);
      for (int i = threadIdx.x; i < n; i += blockDim.x) bb[i] = (double)f[i];
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += A.AinvT[j * n + i] * bb[j];
        x[i] = (T)acc;
      }
    }
    if (!S::sync(b, flag)) return;
  }
  for (int l = nl - 2; l >= l0; --l) {
    const TailLevel<T>& L = A.lv[l];
    const TailLevel<T>& C = A.lv[l + 1];
    const LevelView<T>& V = L.V;
    const T* f = (l == l0) ? A.f0 : L.f;
    T* x = (l == l0) ? A.x0 : L.x;
    if (C.V.Nx == V.Nx) {
      colmat_body<T>(L.Psig, V.M1, C.V.M1, C.x, x, V.ncols, 1, blockIdx.x, gridDim.x, sm);
      if (!S::sync(b, flag)) return;
    } else {
      colmat_body<T>(L.Psig, V.M1, C.V.M1, C.x, L.t4, C.V.ncols, 0, blockIdx.x, gridDim.x, sm);
      if (!S::sync(b, flag)) return;
      const T* cur = L.t4;
      if (DIM == 3) {
        RowPass<T> a = tpass(V, cur, L.t5, V.M1 * C.V.Nx, C.V.Ny, C.V.logNy, V.Ny, V.logNy, XOP_RESAMPLE);
        a.ylines = 1;
        a.Nxl = C.V.Nx;
        if (!g_rowpass<T, S>(a, smem, sm, b, flag)) return;
        cur = L.t5;
      }
      RowPass<T> a = tpass(V, cur, x, V.M1 * V.Ny, C.V.Nx, C.V.logNx, V.Nx, V.logNx, XOP_RESAMPLE);
      a.epi = EPI_ACC;
      if (!g_rowpass<T, S>(a, smem, sm, b, flag)) return;
    }
    for (int i = 0; i < A.nu2; ++i)
      if (!g_sweep<T, DIM, S>(A, L, x, f, smem, sm, b, flag)) return;
  }
}

}  // namespace wt
