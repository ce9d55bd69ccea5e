// Batched uneven 2D tanks in one persistent launch.
//
// One CTA owns one tank for the whole launch and runs every Runge-Kutta step
// of it: the exponential filter, the kinematic free-surface update
// (Eq. kinematicFS), the sigma metric of every multigrid level (Eq. 1_Scoef),
// the smoother's block inverses and the coarsest inverse, the forcing and
// right-hand side (Eq. forc1, poissonp, bcpdneu), the mixed-stage Poisson
// solve - FP64 flexible GMRES (Sec. 4.4) preconditioned by the p-multigrid
// V-cycle (Algorithm 1) in FP32 (mixed form) or in FP64 (plain form: every
// level, smoother block and transfer in FP64), or FP64 iterative refinement
// around an FP32 flexible GMRES with the FP32 V-cycle (refinement form) - and
// the projection (Eq. rkforc1).
// Tanks are launched in decreasing order of size (longest-processing-time
// first) so the large ones start first.  The phases are the device bodies of
// wt_dev.cuh / wt_cta.cuh; no CTA waits on another.
#define WT_DEV_RESTRICT
#include "wt_cta.cuh"
#include "../../include/wt.h"

namespace wt {

__constant__ double c_alpha[5] = {0.0, -567301805773.0 / 1357537059087.0,
                                  -2404267990393.0 / 2016746695238.0,
                                  -3550918686646.0 / 2091501179385.0,
                                  -1275806237668.0 / 842570457699.0};
__constant__ double c_beta[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};

constexpr int kMaxRestart = 31;

struct KrylovSmem {
  double H[(kMaxRestart + 1) * kMaxRestart];
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double red[16][33];
  double h[33];
  double scal[4];
};

// out[i] = sum_e w[e] V_i[e] for i < nvec (and out[nvec] = ||w||^2 if norm),
// accumulated in FP64 whatever the vectors' precision.
template <typename K>
__device__ void cta_dots(const K* w, const K* V, long ld, int nvec, long n, bool norm, KrylovSmem& KS) {
  double acc[33];
#pragma unroll
  for (int i = 0; i < 33; ++i) acc[i] = 0.0;
  for (long e = threadIdx.x; e < n; e += blockDim.x) {
    const double wv = (double)w[e];
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < nvec) acc[i] += wv * (double)V[i * ld + e];
    acc[32] += wv * wv;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 33; ++i) {
    if (!(i < nvec || (i == 32 && norm))) continue;
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) KS.red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 33) {
    const int i = threadIdx.x;
    if (i < nvec || (i == 32 && norm)) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += KS.red[k][i];
      KS.h[i] = s;
    }
  }
  __syncthreads();
}

// w -= sum_i c_i V_i (c from KS.h), optionally scaled into out.
template <typename K>
__device__ void cta_update(K* w, const K* V, long ld, int nvec, long n, const double* c, double scale, K* out) {
  for (long e = threadIdx.x; e < n; e += blockDim.x) {
    double wv = (double)w[e];
    for (int i = 0; i < nvec; ++i) wv -= c[i] * (double)V[i * ld + e];
    out[e] = (K)(wv * scale);
  }
  __syncthreads();
}

// Preconditioners of the CTA's flexible GMRES.
enum BatchPre {
  PRE_F32_OF_F64 = 0,   // FP64 Krylov vectors, the FP32 V-cycle on their rounding
  PRE_F64 = 1,          // FP64 Krylov vectors, the FP64 V-cycle
  PRE_F32 = 2           // FP32 Krylov vectors, the FP32 V-cycle
};

// Flexible GMRES(m) on the finest level of precision K, in this CTA: x is the
// initial guess and the result, bn the norm the residual is measured against;
// returns the last true relative residual ||b - A x|| / bn (precision K).
template <typename K, int PRE>
__device__ double fgmres_cta(const BatchTankDesc& B, const TailLevel<K>& F, const K* b, K* x, K* V, K* Z,
                             double bn, double tol, int maxit, int* its_out, int smem, unsigned char* sm,
                             KrylovSmem& KS) {
  const long n = B.n;
  const int m = B.restart;
  int its = 0;
  double rel = 1.0;
  for (;;) {
    t_apply_op<K, 2>(F, x, V, b, false, smem, sm);            // r = b - A x
    cta_dots<K>(V, nullptr, 0, 0, n, true, KS);
    const double beta = sqrt(KS.h[32]);
    rel = beta / bn;
    if (rel <= tol || its >= maxit || !isfinite(rel)) break;
    for (long e = threadIdx.x; e < n; e += blockDim.x) V[e] = (K)((double)V[e] / beta);
    if (threadIdx.x == 0) {
      for (int i = 0; i <= m; ++i) KS.g[i] = 0.0;
      KS.g[0] = beta;
    }
    __syncthreads();
    int k = 0;
    for (int j = 0; j < m; ++j) {
      K* vj = V + (long)j * n;
      K* zj = Z + (long)j * n;
      K* w = V + (long)(j + 1) * n;
      if constexpr (PRE == PRE_F64) {
        TailArgs<double> A;
        A.lv = B.lv64; A.l0 = 0; A.nl = B.nl;
        A.f0 = reinterpret_cast<const double*>(vj);
        A.x0 = reinterpret_cast<double*>(zj);
        A.f0_nyq = 1; A.omega = B.omega; A.nu1 = B.nu1; A.nu2 = B.nu2; A.AinvT = B.AinvT; A.smem = smem;
        vcycle_cta<double, 2>(A, sm);                            // z_j = M^{-1} v_j (FP64)
        __syncthreads();
      } else {
        TailArgs<float> A;
        A.lv = B.lv32; A.l0 = 0; A.nl = B.nl;
        A.f0_nyq = 1; A.omega = (float)B.omega; A.nu1 = B.nu1; A.nu2 = B.nu2; A.AinvT = B.AinvT; A.smem = smem;
        if constexpr (PRE == PRE_F32) {                          // z_j = M^{-1} v_j (FP32)
          A.f0 = reinterpret_cast<const float*>(vj);
          A.x0 = reinterpret_cast<float*>(zj);
          vcycle_cta<float, 2>(A, sm);
          __syncthreads();
        } else {                                                 // the FP32 V-cycle on (float) v_j
          A.f0 = B.b32;
          A.x0 = B.e32;
          for (long e = threadIdx.x; e < n; e += blockDim.x) B.b32[e] = (float)vj[e];
          __syncthreads();
          vcycle_cta<float, 2>(A, sm);
          for (long e = threadIdx.x; e < n; e += blockDim.x) zj[e] = (K)B.e32[e];
          __syncthreads();
        }
      }
      t_apply_op<K, 2>(F, zj, w, nullptr, false, smem, sm);     // w = A z_j
      cta_dots<K>(w, V, n, j + 1, n, false, KS);                 // classical Gram-Schmidt, twice
      if (threadIdx.x <= j) KS.H[j * (m + 1) + threadIdx.x] = KS.h[threadIdx.x];
      __syncthreads();
      cta_update<K>(w, V, n, j + 1, n, KS.h, 1.0, w);
      cta_dots<K>(w, V, n, j + 1, n, true, KS);
      if (threadIdx.x == 0) {
        double* H = KS.H + j * (m + 1);
        double hh = KS.h[32];
        for (int i = 0; i <= j; ++i) {
          H[i] += KS.h[i];
          hh -= KS.h[i] * KS.h[i];
        }
        const double hn = hh > 0 ? sqrt(hh) : 0.0;
        for (int i = 0; i < j; ++i) {
          const double t = KS.cs[i] * H[i] + KS.sn[i] * H[i + 1];
          H[i + 1] = -KS.sn[i] * H[i] + KS.cs[i] * H[i + 1];
          H[i] = t;
        }
        const double den = hypot(H[j], hn);
        const double c = den > 0 ? H[j] / den : 1.0, sg = den > 0 ? hn / den : 0.0;
        KS.cs[j] = c;
        KS.sn[j] = sg;
        H[j] = den;
        const double gj = KS.g[j];
        KS.g[j + 1] = -sg * gj;
        KS.g[j] = c * gj;
        const bool breakdown = !(hn > 1e-14 * den);
        KS.scal[0] = breakdown ? 0.0 : 1.0 / hn;
        KS.scal[1] = (fabs(KS.g[j + 1]) <= tol * bn || breakdown) ? 1.0 : 0.0;
      }
      __syncthreads();
      cta_update<K>(w, V, n, j + 1, n, KS.h, KS.scal[0], w);      // v_{j+1}
      ++its;
      k = j + 1;
      if (KS.scal[1] != 0.0 || its >= maxit) break;
    }
    if (threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double sacc = KS.g[i];
        for (int l = i + 1; l < k; ++l) sacc -= KS.H[l * (m + 1) + i] * KS.y[l];
        KS.y[i] = sacc / KS.H[i * (m + 1) + i];
      }
    }
    __syncthreads();
    for (long e = threadIdx.x; e < n; e += blockDim.x) {
      double acc = (double)x[e];
      for (int i = 0; i < k; ++i) acc += KS.y[i] * (double)Z[(long)i * n + e];
      x[e] = (K)acc;
    }
    __syncthreads();
  }
  *its_out = its;
  return rel;
}

// The stage's pressure solve in this CTA, in the batch's form: FP64 GMRES with
// the FP32 V-cycle (MODE 0) or the FP64 V-cycle (MODE 1); or FP64 iterative
// refinement (MODE 2): r = b - A x in FP64, an FP32 flexible GMRES with the
// FP32 V-cycle solves A e = r / |r| to inner_tol, x += |r| e.
template <int MODE>
__device__ void solve_cta(const BatchTankDesc& B, const double* b, double* x, int smem, unsigned char* sm,
                          KrylovSmem& KS) {
  const long n = B.n;
  cta_dots<double>(b, nullptr, 0, 0, n, true, KS);
  const double bn = sqrt(KS.h[32]);
  int its = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    for (long e = threadIdx.x; e < n; e += blockDim.x) x[e] = 0.0;
    __syncthreads();
  } else if constexpr (MODE == 2) {
    int refinements = 0;
    for (;;) {
      t_apply_op<double, 2>(B.lv64[0], x, B.r64, b, false, smem, sm);   // r = b - A x (FP64)
      cta_dots<double>(B.r64, nullptr, 0, 0, n, true, KS);
      const double rn = sqrt(KS.h[32]);
      rel = rn / bn;
      if (rel <= B.tol || refinements >= B.max_ir || its >= B.max_it || !isfinite(rel)) break;
      for (long e = threadIdx.x; e < n; e += blockDim.x) {
        B.b32[e] = (float)(B.r64[e] / rn);
        B.e32[e] = 0.0f;
      }
      __syncthreads();
      int it = 0;
      const int cap = min(B.restart, B.max_it - its);
      fgmres_cta<float, PRE_F32>(B, B.lv32[0], B.b32, B.e32, B.V32, B.Z32, 1.0, B.inner_tol, cap, &it, smem, sm, KS);
      its += it;
      for (long e = threadIdx.x; e < n; e += blockDim.x) x[e] += rn * (double)B.e32[e];
      __syncthreads();
      ++refinements;
    }
  } else {
    rel = fgmres_cta<double, MODE == 1 ? PRE_F64 : PRE_F32_OF_F64>(B, B.lv64[0], b, x, B.V64, B.Z64, bn, B.tol,
                                                                   B.max_it, &its, smem, sm, KS);
  }
  if (threadIdx.x == 0) {
    B.stats[0] += 1.0;
    B.stats[1] += its;
    B.stats[2] = rel;
    if (!(rel <= B.tol)) atomicOr(B.flag, 16);
  }
  __syncthreads();
}

__device__ RowPass<double> pass64(const BatchTankDesc& B, const double* in, double* out, int nrows, int Nin,
                                  int logNin, int Nout, int logNout, int op) {
  return tpass<double>(B.lv64[0].V, in, out, nrows, Nin, logNin, Nout, logNout, op);
}

// One Runge-Kutta stage k of one tank (the same sequence as the host-driven
// stage in wt_capi.cu, linear = free-surface and advection terms dropped).
template <int MODE>
__device__ void stage_cta(const BatchTankDesc& B, int k, double dt, int smem, unsigned char* sm,
                          KrylovSmem& K) {
  constexpr bool P64 = MODE == 1;                 // FP64 V-cycle: FP64 blocks, no FP32 metric
  const double a = c_alpha[k - 1], b = c_beta[k - 1];
  const int M1 = B.M1, Nx = B.Nx, lx = B.logNx;
  const long n = B.n;
  const int nc = B.ncols;
  const int t0 = threadIdx.x, ts = blockDim.x;
  double* const* W = B.work;
  if (B.filter) {
    RowPass<double> f1 = pass64(B, B.eta, B.eta, 1, Nx, lx, Nx, lx, XOP_FILTER);
    f1.filt = B.filt_x;
    t_rowpass(f1, smem, sm);
    for (int qi = 0; qi < 2; ++qi) {
      double* q = qi ? B.w : B.u;
      RowPass<double> f2 = pass64(B, q, q, M1, Nx, lx, Nx, lx, XOP_FILTER);
      f2.filt = B.filt_x;
      t_rowpass(f2, smem, sm);
      colmat_body<double>(B.Fcheb, M1, M1, q, q, nc, 0, 0, 1, sm);
    }
  }
  // free-surface update
  t_rowpass(pass64(B, B.eta, B.eta_x, 1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  stage_eta_body(t0, ts, nc, B.linear, a, b, dt, B.u, nullptr, B.w, B.eta_x, B.zero_s, B.Keta, B.eta,
                 B.eta_new, B.f_eta, B.flag);
  __syncthreads();
  // metric of every level: a = eta^(k), b = eta^(k-1) (still water in the linear model)
  const double* ea = B.linear ? B.zero_s : B.eta_new;
  const double* eb = B.linear ? B.zero_s : B.eta;
  for (int l = 0; l < B.nl; ++l) {
    const SurfDesc& S = B.S[l];
    const LevelView<double>& V = B.lv64[l].V;
    for (int g2 = 0; g2 < 2; ++g2) {
      const double* fine = g2 ? eb : ea;
      double* out = g2 ? S.eb : S.ea;
      double* outx = g2 ? S.ebx : S.eax;
      if (l == 0) {
        for (int c = t0; c < nc; c += ts) out[c] = fine[c];
        __syncthreads();
      } else {
        t_rowpass(pass64(B, fine, out, 1, Nx, lx, V.Nx, V.logNx, XOP_RESAMPLE), smem, sm);
      }
      t_rowpass(tpass<double>(V, out, outx, 1, V.Nx, V.logNx, V.Nx, V.logNx, XOP_DERIV), smem, sm);
    }
    metric_body(t0, ts, V.ncols, S.h, S.hx, nullptr, S.ea, S.eax, nullptr, S.eb, S.ebx, nullptr,
                const_cast<double*>(V.meta), B.flag);
    __syncthreads();
    if (!P64) {
      float* m32 = const_cast<float*>(B.lv32[l].V.meta);
      for (long i = t0; i < (long)kMeta * V.ncols; i += ts) m32[i] = (float)V.meta[i];
      __syncthreads();
    }
  }
  for (int l = 0; l + 1 < B.nl; ++l) {
    if (P64) {
      const TailLevel<double>& L = B.lv64[l];
      const int per_warp = L.V.M1 * (2 * L.V.M1 + 1) * (int)sizeof(double);
      blockinv_body<double>(L.V, const_cast<double*>(L.Binv), L.nclass, L.cxx, L.cyy, B.flag, 0, 1,
                            smem / per_warp, sm);
    } else {
      const TailLevel<float>& L = B.lv32[l];
      const int per_warp = L.V.M1 * (2 * L.V.M1 + 1) * (int)sizeof(float);
      blockinv_body<float>(L.V, const_cast<float*>(L.Binv), L.nclass, L.cxx, L.cyy, B.flag, 0, 1,
                           smem / per_warp, sm);
    }
    __syncthreads();
  }
  coarse_factor_body(B.lv64[B.nl - 1].V, B.cDx, B.cDy, B.AinvT, B.flag, sm);
  __syncthreads();
  // forcing without p_D and u* = u + beta (alpha K + dt F)
  StageArgs sa;
  sa.Nx = Nx; sa.Ny = 1; sa.M1 = M1; sa.ncols = nc;
  sa.g = B.g; sa.alpha = a; sa.beta = b; sa.dt = dt; sa.linear = B.linear;
  sa.sigma = B.lv64[0].V.sigma; sa.D = B.lv64[0].V.D; sa.meta = B.lv64[0].V.meta;
  double *ux = W[0], *wx = W[4], *us = W[6], *ws = W[8], *usx = W[9], *Dus = W[11], *Dws = W[13],
         *rhs = W[14], *px = W[15], *Dp = W[17];
  const double* Dm = B.lv64[0].V.D;
  t_rowpass(pass64(B, B.u, ux, M1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  t_rowpass(pass64(B, B.w, wx, M1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  colmat_body<double>(Dm, M1, M1, B.u, us, nc, 0, 0, 1, sm);
  colmat_body<double>(Dm, M1, M1, B.w, ws, nc, 0, 0, 1, sm);
  stage_forcing_body(t0, ts, sa, B.u, nullptr, B.w, ux, nullptr, nullptr, nullptr, wx, nullptr, B.eta_x,
                     B.zero_s, B.f_eta, B.Ku, nullptr, B.Kw, us, nullptr, ws);
  __syncthreads();
  // right-hand side of the mixed-stage Poisson problem
  t_rowpass(pass64(B, us, usx, M1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  colmat_body<double>(Dm, M1, M1, us, Dus, nc, 0, 0, 1, sm);
  colmat_body<double>(Dm, M1, M1, ws, Dws, nc, 0, 0, 1, sm);
  stage_rhs_body(t0, ts, sa, us, nullptr, ws, usx, nullptr, Dus, nullptr, Dws, rhs);
  __syncthreads();
  solve_cta<MODE>(B, rhs, B.p, smem, sm, K);
  // projection
  t_rowpass(pass64(B, B.p, px, M1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  colmat_body<double>(Dm, M1, M1, B.p, Dp, nc, 0, 0, 1, sm);
  stage_project_body(t0, ts, sa, px, nullptr, Dp, B.Ku, nullptr, B.Kw, B.u, nullptr, B.w, B.flag);
  __syncthreads();
  for (int c = t0; c < nc; c += ts) B.eta[c] = B.eta_new[c];
  __syncthreads();
  (void)n;
}

template <int MODE>
__global__ void __launch_bounds__(512) k_batch_step(const BatchTankDesc* descs, const int* order,
                                                    const double* dt, int nsteps, int smem) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ KrylovSmem K;
  const int tank = order[blockIdx.x];
  const BatchTankDesc& B = descs[tank];
  for (int s = 0; s < nsteps; ++s)
    for (int k = 1; k <= 5; ++k) stage_cta<MODE>(B, k, dt[tank], smem, sm, K);
}

template <int MODE>
static cudaError_t launch_mode(const BatchTankDesc* descs, const int* order, int ntanks, const double* dt,
                               int nsteps, int smem, cudaStream_t s) {
  cudaError_t e = ensure_dyn_smem((const void*)k_batch_step<MODE>, (size_t)smem);
  if (e != cudaSuccess) return e;
  k_batch_step<MODE><<<ntanks, 512, smem, s>>>(descs, order, dt, nsteps, smem);
  return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchTankDesc* descs, const int* order, int ntanks, const double* dt,
                              int nsteps, int smem, int mode, cudaStream_t s) {
  if (mode == WT_FP64) return launch_mode<1>(descs, order, ntanks, dt, nsteps, smem, s);
  if (mode == WT_REFINE) return launch_mode<2>(descs, order, ntanks, dt, nsteps, smem, s);
  return launch_mode<0>(descs, order, ntanks, dt, nsteps, smem, s);
}

}  // namespace wt
