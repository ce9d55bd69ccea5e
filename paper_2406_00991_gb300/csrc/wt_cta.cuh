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
