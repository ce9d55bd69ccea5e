// Batched uneven 2D tanks in one persistent launch.
//
// One CTA owns one tank for the whole launch and runs every Runge-Kutta step
// of it: the exponential filter, the kinematic free-surface update
// (Eq. kinematicFS), the sigma metric of every multigrid level (Eq. 1_Scoef),
// the smoother's block inverses and the coarsest inverse, the forcing and
// right-hand side (Eq. forc1, poissonp, bcpdneu), the mixed-stage Poisson
// solve - FP64 flexible GMRES (Sec. 4.4) preconditioned by the p-multigrid
// V-cycle (Algorithm 1) in FP32 (mixed form) or in FP64 (plain form: every
// level, smoother block and transfer in FP64) - and the projection
// (Eq. rkforc1).
// Tanks are launched in decreasing order of size (longest-processing-time
// first) so the large ones start first.  The phases are the device bodies of
// wt_dev.cuh / wt_cta.cuh; no CTA waits on another.
#define WT_DEV_RESTRICT
#include "wt_cta.cuh"

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

// out[i] = sum_e w[e] V_i[e] for i < nvec (and out[nvec] = ||w||^2 if norm).
__device__ void cta_dots(const double* w, const double* V, long ld, int nvec, long n, bool norm,
                         KrylovSmem& K) {
  double acc[33];
#pragma unroll
  for (int i = 0; i < 33; ++i) acc[i] = 0.0;
  for (long e = threadIdx.x; e < n; e += blockDim.x) {
    const double wv = w[e];
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < nvec) acc[i] += wv * V[i * ld + e];
    acc[32] += wv * wv;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 33; ++i) {
    if (!(i < nvec || (i == 32 && norm))) continue;
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) K.red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 33) {
    const int i = threadIdx.x;
    if (i < nvec || (i == 32 && norm)) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += K.red[k][i];
      K.h[i] = s;
    }
  }
  __syncthreads();
}

// w -= sum_i c_i V_i (c from K.h), optionally scaled into out.
__device__ void cta_update(double* w, const double* V, long ld, int nvec, long n, const double* c,
                           double scale, double* out) {
  for (long e = threadIdx.x; e < n; e += blockDim.x) {
    double wv = w[e];
    for (int i = 0; i < nvec; ++i) wv -= c[i] * V[i * ld + e];
    out[e] = wv * scale;
  }
  __syncthreads();
}

// FP64 flexible GMRES(m) with the V-cycle as preconditioner, in this CTA:
// the FP32 V-cycle on the rounded Arnoldi vector (P64 = false) or the FP64
// V-cycle on the vector itself (P64 = true).
template <bool P64>
__device__ void fgmres_cta(const BatchTankDesc& B, const double* b, double* x, int smem,
                           unsigned char* sm, KrylovSmem& K) {
  const TailLevel<double>& F = B.lv64[0];
  const long n = B.n;
  const int m = B.restart;
  double* V = B.V64;
  double* Z = B.Z64;
  TailArgs<float> A;
  A.lv = B.lv32;
  A.l0 = 0;
  A.nl = B.nl;
  A.f0 = B.b32;
  A.x0 = B.e32;
  A.f0_nyq = 1;
  A.omega = (float)B.omega;
  A.nu1 = B.nu1;
  A.nu2 = B.nu2;
  A.AinvT = B.AinvT;
  A.smem = smem;
  cta_dots(b, nullptr, 0, 0, n, true, K);
  const double bn = sqrt(K.h[32]);
  int its = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    for (long e = threadIdx.x; e < n; e += blockDim.x) x[e] = 0.0;
    __syncthreads();
  } else {
    for (;;) {
      t_apply_op<double, 2>(F, x, V, b, false, smem, sm);       // r = b - A x
      cta_dots(V, nullptr, 0, 0, n, true, K);
      const double beta = sqrt(K.h[32]);
      rel = beta / bn;
      if (rel <= B.tol || its >= B.max_it) break;
      for (long e = threadIdx.x; e < n; e += blockDim.x) V[e] /= beta;
      if (threadIdx.x == 0) {
        for (int i = 0; i <= m; ++i) K.g[i] = 0.0;
        K.g[0] = beta;
      }
      __syncthreads();
      int k = 0;
      bool done = false;
      for (int j = 0; j < m; ++j) {
        double* vj = V + (long)j * n;
        double* zj = Z + (long)j * n;
        double* w = V + (long)(j + 1) * n;
        if (P64) {
          TailArgs<double> A64;
          A64.lv = B.lv64;
          A64.l0 = 0;
          A64.nl = B.nl;
          A64.f0 = vj;
          A64.x0 = zj;
          A64.f0_nyq = 1;
          A64.omega = B.omega;
          A64.nu1 = B.nu1;
          A64.nu2 = B.nu2;
          A64.AinvT = B.AinvT;
          A64.smem = smem;
          vcycle_cta<double, 2>(A64, sm);                         // z_j = M^{-1} v_j (FP64)
          __syncthreads();
        } else {
          for (long e = threadIdx.x; e < n; e += blockDim.x) B.b32[e] = (float)vj[e];
          __syncthreads();
          vcycle_cta<float, 2>(A, sm);                            // e32 = M^{-1} v_j (FP32)
          for (long e = threadIdx.x; e < n; e += blockDim.x) zj[e] = (double)B.e32[e];
          __syncthreads();
        }
        t_apply_op<double, 2>(F, zj, w, nullptr, false, smem, sm);   // w = A z_j
        cta_dots(w, V, n, j + 1, n, false, K);                    // classical Gram-Schmidt, twice
        if (threadIdx.x <= j) K.H[j * (m + 1) + threadIdx.x] = K.h[threadIdx.x];
        __syncthreads();
        cta_update(w, V, n, j + 1, n, K.h, 1.0, w);
        cta_dots(w, V, n, j + 1, n, true, K);
        double hh = 0.0;
        if (threadIdx.x == 0) {
          double* H = K.H + j * (m + 1);
          hh = K.h[32];
          for (int i = 0; i <= j; ++i) {
            H[i] += K.h[i];
            hh -= K.h[i] * K.h[i];
          }
          const double hn = hh > 0 ? sqrt(hh) : 0.0;
          for (int i = 0; i < j; ++i) {
            const double t = K.cs[i] * H[i] + K.sn[i] * H[i + 1];
            H[i + 1] = -K.sn[i] * H[i] + K.cs[i] * H[i + 1];
            H[i] = t;
          }
          const double den = hypot(H[j], hn);
          const double c = den > 0 ? H[j] / den : 1.0, s = den > 0 ? hn / den : 0.0;
          K.cs[j] = c;
          K.sn[j] = s;
          H[j] = den;
          const double gj = K.g[j];
          K.g[j + 1] = -s * gj;
          K.g[j] = c * gj;
          const bool breakdown = !(hn > 1e-14 * den);
          K.scal[0] = breakdown ? 0.0 : 1.0 / hn;
          K.scal[1] = (fabs(K.g[j + 1]) <= B.tol * bn || breakdown) ? 1.0 : 0.0;
        }
        __syncthreads();
        cta_update(w, V, n, j + 1, n, K.h, K.scal[0], w);        // v_{j+1}
        ++its;
        k = j + 1;
        done = K.scal[1] != 0.0;
        if (done || its >= B.max_it) break;
      }
      if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
          double s = K.g[i];
          for (int l = i + 1; l < k; ++l) s -= K.H[l * (m + 1) + i] * K.y[l];
          K.y[i] = s / K.H[i * (m + 1) + i];
        }
      }
      __syncthreads();
      for (long e = threadIdx.x; e < n; e += blockDim.x) {
        double acc = x[e];
        for (int i = 0; i < k; ++i) acc += K.y[i] * Z[(long)i * n + e];
        x[e] = acc;
      }
      __syncthreads();
    }
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
template <bool P64>
__device__ void stage_cta(const BatchTankDesc& B, int k, double dt, int smem, unsigned char* sm,
                          KrylovSmem& K) {
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
  fgmres_cta<P64>(B, rhs, B.p, smem, sm, K);
  // projection
  t_rowpass(pass64(B, B.p, px, M1, Nx, lx, Nx, lx, XOP_DERIV), smem, sm);
  colmat_body<double>(Dm, M1, M1, B.p, Dp, nc, 0, 0, 1, sm);
  stage_project_body(t0, ts, sa, px, nullptr, Dp, B.Ku, nullptr, B.Kw, B.u, nullptr, B.w, B.flag);
  __syncthreads();
  for (int c = t0; c < nc; c += ts) B.eta[c] = B.eta_new[c];
  __syncthreads();
  (void)n;
}

template <bool P64>
__global__ void __launch_bounds__(512) k_batch_step(const BatchTankDesc* descs, const int* order,
                                                    const double* dt, int nsteps, int smem) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ KrylovSmem K;
  const int tank = order[blockIdx.x];
  const BatchTankDesc& B = descs[tank];
  for (int s = 0; s < nsteps; ++s)
    for (int k = 1; k <= 5; ++k) stage_cta<P64>(B, k, dt[tank], smem, sm, K);
}

cudaError_t launch_batch_step(const BatchTankDesc* descs, const int* order, int ntanks, const double* dt,
                              int nsteps, int smem, int fp64, cudaStream_t s) {
  const void* fn = fp64 ? (const void*)k_batch_step<true> : (const void*)k_batch_step<false>;
  cudaError_t e = ensure_dyn_smem(fn, (size_t)smem);
  if (e != cudaSuccess) return e;
  if (fp64)
    k_batch_step<true><<<ntanks, 512, smem, s>>>(descs, order, dt, nsteps, smem);
  else
    k_batch_step<false><<<ntanks, 512, smem, s>>>(descs, order, dt, nsteps, smem);
  return cudaGetLastError();
}

}  // namespace wt
