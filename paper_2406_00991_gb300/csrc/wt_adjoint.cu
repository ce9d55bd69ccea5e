// Adjoint (reverse-mode derivative) of one Runge-Kutta stage of a 2D tank
// (the paper has no adjoint; the forward stage is Sec. 3.1-3.3 with
// Eq. kinematicFS, forc1, poissonp, bcpdneu, rkforc1 and the filter of
// Sec. 3.6 on the stage input).
//
// Forward stage k (alpha, beta), c = 1 / (beta dt), with the filtered input
// (eta~, u~, w~), metric a of eta^(k) and b of eta~ (still water for both in
// the linearised model):
//   eta_x = D_x eta~,  f = -u~_0 eta_x + w~_0,  K_eta' = alpha K_eta + dt f,
//   eta^(k) = eta~ + beta K_eta'
//   F_u = -g eta_x - u~ D_x u~ - w_s D u~,  F_w = -u~ D_x w~ - w_s D w~,
//   w_s = -sigma f / d_b + u~ sx_b + w~ Z_b
//   K_q' = alpha K_q + dt F_q,  q* = q~ + beta K_q'
//   rhs = c (Div_a (u*, w*)) inside, c (h_x u* + w*) at the bottom, 0 on top
//   p = A_{a,b}^{-1} rhs
//   K_u'' = K_u' - dt (D_x p + sx_b D p),  K_w'' = K_w' - dt Z_b D p,
//   q^(k) = q~ + beta K_q''
// The reverse sweep below takes the adjoints of (eta^(k), u^(k), w^(k),
// K_eta', K_u'', K_w'') to those of the stage input and adds the stage's
// contribution to dJ/dh.  The pressure adjoint is the transposed problem
// A^T lam = (adjoint of p), solved with the same p-multigrid on A^T; the
// operator's dependence on the metric enters as -lam^T (dA/dtheta) p.
// D_x^T = -D_x (antisymmetric, Nyquist coefficient zeroed); D^T is the
// transposed sigma matrix.  Kernels here are one thread per column.
#include "wt_solver.h"

#include <algorithm>

namespace wt {

namespace {

constexpr int MM = kMaxM1;

__device__ inline void colvec(const double* f, long nc, long c, int M1, double* v) {
  for (int m = 0; m < M1; ++m) v[m] = f[m * nc + c];
}
__device__ inline void matvec(const double* D, int M1, const double* in, double* out) {
  for (int m = 0; m < M1; ++m) {
    double a = 0.0;
    for (int k = 0; k < M1; ++k) a += D[m * M1 + k] * in[k];
    out[m] = a;
  }
}
__device__ inline void matvecT(const double* D, int M1, const double* in, double* out) {
  for (int m = 0; m < M1; ++m) {
    double a = 0.0;
    for (int k = 0; k < M1; ++k) a += D[k * M1 + m] * in[k];
    out[m] = a;
  }
}

struct AdjArgs {
  int M1;
  long nc;
  const double* D;
  const double* sigma;
  const double* meta;
  double alpha, beta, dt, g;
  int linear;
};

// Projection (rkforc1) reversed: adjoints of K_u'', K_w'' -> grad_b p -> p.
__global__ void k_adj_proj(AdjArgs A, const double* __restrict__ Lu, const double* __restrict__ Lw,
                           const double* __restrict__ LKu, const double* __restrict__ LKw,
                           const double* __restrict__ p, double* __restrict__ LKu1,
                           double* __restrict__ LKw1, double* __restrict__ LGx, double* __restrict__ q,
                           double* __restrict__ lut, double* __restrict__ lwt, double* __restrict__ gB) {
  pdl_enter();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nc = A.nc;
  if (c >= nc) return;
  const int M1 = A.M1;
  const double AXb = A.meta[M_AXb * nc + c], BXb = A.meta[M_BXb * nc + c], Zb = A.meta[M_Zb * nc + c];
  double pv[MM], ps[MM], qv[MM], qo[MM];
  colvec(p, nc, c, M1, pv);
  matvec(A.D, M1, pv, ps);
  double gax = 0, gbx = 0, gz = 0;
  for (int m = 0; m < M1; ++m) {
    const long e = m * nc + c;
    const double ku = LKu[e] + A.beta * Lu[e], kw = LKw[e] + A.beta * Lw[e];
    LKu1[e] = ku;
    LKw1[e] = kw;
    lut[e] = Lu[e];
    lwt[e] = Lw[e];
    const double gx = -A.dt * ku, gzv = -A.dt * kw;
    LGx[e] = gx;
    const double s = A.sigma[m];
    qv[m] = (AXb - s * BXb) * gx + Zb * gzv;
    gax += gx * ps[m];
    gbx -= s * gx * ps[m];
    gz += gzv * ps[m];
  }
  matvecT(A.D, M1, qv, qo);
  for (int m = 0; m < M1; ++m) q[m * nc + c] = qo[m];
  gB[0 * nc + c] += gax;
  gB[1 * nc + c] += gbx;
  gB[2 * nc + c] += gz;
}

// Poisson problem (poissonp, bcpdneu) reversed: lam = A^{-T} (adjoint of p)
// gives -lam^T (dA/dtheta) p for the metric, lam -> adjoint of (u*, w*) and
// the rhs's own metric terms; then q* = q~ + beta K', K' = alpha K + dt F.
__global__ void k_adj_rhs(AdjArgs A, const double* __restrict__ lam, const double* __restrict__ Dxlam,
                          const double* __restrict__ p, const double* __restrict__ px,
                          const double* __restrict__ us, const double* __restrict__ ws,
                          double* __restrict__ LKu1, double* __restrict__ LKw1, double* __restrict__ lut,
                          double* __restrict__ lwt, double* __restrict__ LKu, double* __restrict__ LKw,
                          double* __restrict__ lFu, double* __restrict__ lFw, double* __restrict__ gA,
                          double* __restrict__ gB, double* __restrict__ gHX) {
  pdl_enter();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nc = A.nc;
  if (c >= nc) return;
  const int M1 = A.M1, N = M1 - 1;
  const double* meta = A.meta;
  const double AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c], Za = meta[M_Za * nc + c];
  const double AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c], Zb = meta[M_Zb * nc + c];
  const double HX = meta[M_HX * nc + c];
  const double cc = 1.0 / (A.beta * A.dt);
  double l[MM], v[MM], ps[MM], G[MM], DG[MM], a[MM], Dta[MM], mux[MM], muz[MM];
  colvec(lam, nc, c, M1, l);
  const double lN = l[N];
  // operator metric terms, geometry a: -lam_int . d(Div_a G)/dtheta_a
  colvec(p, nc, c, M1, v);
  matvec(A.D, M1, v, ps);
  for (int m = 0; m < M1; ++m) G[m] = px[m * nc + c] + (AXb - A.sigma[m] * BXb) * ps[m];
  matvec(A.D, M1, G, DG);
  double gAx = 0, gAb = 0, gAz = 0, gH = 0;
  for (int m = 1; m < N; ++m) {
    gAx -= l[m] * DG[m];
    gAb += A.sigma[m] * l[m] * DG[m];
  }
  gH -= lN * G[N];
  for (int m = 0; m < M1; ++m) G[m] = Zb * ps[m];                // G_z
  matvec(A.D, M1, G, DG);
  for (int m = 1; m < N; ++m) gAz -= l[m] * DG[m];
  // mu = adjoint of (G_x, G_z) for the weight lam
  for (int m = 0; m < M1; ++m) a[m] = (m > 0 && m < N) ? (AXa - A.sigma[m] * BXa) * l[m] : 0.0;
  matvecT(A.D, M1, a, Dta);
  for (int m = 0; m < M1; ++m) mux[m] = ((m > 0 && m < N) ? -Dxlam[m * nc + c] : 0.0) + Dta[m] + (m == N ? HX * lN : 0.0);
  for (int m = 0; m < M1; ++m) a[m] = (m > 0 && m < N) ? Za * l[m] : 0.0;
  matvecT(A.D, M1, a, Dta);
  for (int m = 0; m < M1; ++m) muz[m] = Dta[m] + (m == N ? lN : 0.0);
  double gBx = 0, gBb = 0, gBz = 0;
  for (int m = 0; m < M1; ++m) {
    gBx -= mux[m] * ps[m];
    gBb += A.sigma[m] * mux[m] * ps[m];
    gBz -= muz[m] * ps[m];
  }
  // rhs metric terms: + c lam_int . d(Div_a u*)/dtheta_a, bottom row h_x u*
  colvec(us, nc, c, M1, v);
  matvec(A.D, M1, v, DG);
  for (int m = 1; m < N; ++m) {
    gAx += cc * l[m] * DG[m];
    gAb -= cc * A.sigma[m] * l[m] * DG[m];
  }
  gH += cc * lN * v[N];
  colvec(ws, nc, c, M1, v);
  matvec(A.D, M1, v, DG);
  for (int m = 1; m < N; ++m) gAz += cc * l[m] * DG[m];
  // adjoint of (u*, w*) = c mu; then the 2N registers and the forcing
  for (int m = 0; m < M1; ++m) {
    const long e = m * nc + c;
    const double lu = cc * mux[m], lw = cc * muz[m];
    const double ku = LKu1[e] + A.beta * lu, kw = LKw1[e] + A.beta * lw;
    lut[e] += lu;
    lwt[e] += lw;
    lFu[e] = A.dt * ku;
    lFw[e] = A.dt * kw;
    LKu[e] = A.alpha * ku;
    LKw[e] = A.alpha * kw;
  }
  gA[0 * nc + c] += gAx;
  gA[1 * nc + c] += gAb;
  gA[2 * nc + c] += gAz;
  gB[0 * nc + c] += gBx;
  gB[1 * nc + c] += gBb;
  gB[2 * nc + c] += gBz;
  gHX[c] += gH;
}

// Momentum forcing (forc1) reversed.  lex = adjoint of eta_x, lfe = of f,
// ldb = direct adjoint of d_b (through sigma_t); lux, lwx are the adjoints of
// D_x u~, D_x w~ (the caller applies D_x^T = -D_x to them).
__global__ void k_adj_forcing(AdjArgs A, const double* __restrict__ ut, const double* __restrict__ wt,
                              const double* __restrict__ ux, const double* __restrict__ wx,
                              const double* __restrict__ fe, const double* __restrict__ lFu,
                              const double* __restrict__ lFw, double* __restrict__ lut,
                              double* __restrict__ lwt, double* __restrict__ lux, double* __restrict__ lwx,
                              double* __restrict__ lex, double* __restrict__ lfe, double* __restrict__ ldb,
                              double* __restrict__ gB) {
  pdl_enter();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nc = A.nc;
  if (c >= nc) return;
  const int M1 = A.M1;
  double sum = 0.0;
  for (int m = 0; m < M1; ++m) sum += lFu[m * nc + c];
  lex[c] = -A.g * sum;
  if (A.linear) {
    lfe[c] = 0.0;
    ldb[c] = 0.0;
    return;
  }
  const double* meta = A.meta;
  const double AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c], Zb = meta[M_Zb * nc + c];
  const double db = meta[M_D_B * nc + c];
  const double f = fe[c];
  double u[MM], w[MM], us[MM], wsv[MM], lus[MM], lws[MM], o[MM];
  colvec(ut, nc, c, M1, u);
  colvec(wt, nc, c, M1, w);
  matvec(A.D, M1, u, us);
  matvec(A.D, M1, w, wsv);
  double gax = 0, gbx = 0, gz = 0, lf = 0, ld = 0;
  for (int m = 0; m < M1; ++m) {
    const long e = m * nc + c;
    const double s = A.sigma[m];
    const double sxb = AXb - s * BXb;
    const double wsig = -s * f / db + u[m] * sxb + w[m] * Zb;
    const double fu = lFu[e], fw = lFw[e];
    const double lwsig = -fu * us[m] - fw * wsv[m];
    lut[e] += -fu * ux[e] - fw * wx[e] + lwsig * sxb;
    lwt[e] += lwsig * Zb;
    lux[e] = -fu * u[m];
    lwx[e] = -fw * u[m];
    lus[m] = -fu * wsig;
    lws[m] = -fw * wsig;
    lf -= s * lwsig / db;
    ld += s * lwsig * f / (db * db);
    gax += lwsig * u[m];
    gbx -= s * lwsig * u[m];
    gz += lwsig * w[m];
  }
  matvecT(A.D, M1, lus, o);
  for (int m = 0; m < M1; ++m) lut[m * nc + c] += o[m];
  matvecT(A.D, M1, lws, o);
  for (int m = 0; m < M1; ++m) lwt[m * nc + c] += o[m];
  lfe[c] = lf;
  ldb[c] = ld;
  gB[0 * nc + c] += gax;
  gB[1 * nc + c] += gbx;
  gB[2 * nc + c] += gz;
}

// Metric (Eq. 1_Scoef) reversed for both geometries: AX = h_x / d,
// BX = d_x / d, Z = 1 / d, d = h + e, d_x = h_x + e_x.  Outputs the direct
// adjoints of e_a, e_b and h, and those of e_a,x, e_b,x and h_x (the caller
// applies D_x^T = -D_x).
__global__ void k_adj_metric(long nc, const double* __restrict__ meta, const double* __restrict__ gA,
                             const double* __restrict__ gB, const double* __restrict__ gHX,
                             const double* __restrict__ ldb, double* __restrict__ lea,
                             double* __restrict__ leax, double* __restrict__ leb, double* __restrict__ lebx,
                             double* __restrict__ lh0, double* __restrict__ lhx) {
  pdl_enter();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double hx = meta[M_HX * nc + c];
  const double da = meta[M_D_A * nc + c], db = meta[M_D_B * nc + c];
  const double dxa = meta[M_BXa * nc + c] * da, dxb = meta[M_BXb * nc + c] * db;
  const double aX = gA[c], aB = gA[nc + c], aZ = gA[2 * nc + c];
  const double bX = gB[c], bB = gB[nc + c], bZ = gB[2 * nc + c];
  const double lda = -(aX * hx + aB * dxa + aZ) / (da * da);
  const double ldbv = -(bX * hx + bB * dxb + bZ) / (db * db) + ldb[c];
  lea[c] = lda;
  leb[c] = ldbv;
  leax[c] = aB / da;
  lebx[c] = bB / db;
  lh0[c] = lda + ldbv;
  lhx[c] = (aX + aB) / da + (bX + bB) / db + gHX[c];
}

// Free surface (kinematicFS) reversed; adds the stage's dJ/dh.
__global__ void k_adj_eta(AdjArgs A, const double* __restrict__ Le, double* __restrict__ LKe,
                          const double* __restrict__ lea, const double* __restrict__ tA,
                          const double* __restrict__ leb, const double* __restrict__ tB,
                          const double* __restrict__ lh0, const double* __restrict__ tH,
                          const double* __restrict__ lfe, const double* __restrict__ lexf,
                          const double* __restrict__ ex, const double* __restrict__ ut,
                          double* __restrict__ lut, double* __restrict__ lwt, double* __restrict__ lh,
                          double* __restrict__ let, double* __restrict__ lex) {
  pdl_enter();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.nc) return;
  const double LN = Le[c] + (A.linear ? 0.0 : lea[c] - tA[c]);      // adjoint of eta^(k)
  let[c] = LN + (A.linear ? 0.0 : leb[c] - tB[c]);
  lh[c] += lh0[c] - tH[c];
  const double k1 = LKe[c] + A.beta * LN;
  LKe[c] = A.alpha * k1;
  const double lf = lfe[c] + A.dt * k1;
  lwt[c] += lf;                                                      // surface row of w~
  if (A.linear) {
    lex[c] = lexf[c];
  } else {
    lut[c] += -lf * ex[c];
    lex[c] = lexf[c] - lf * ut[c];
  }
}

inline int blocks(long n) { return (int)std::max<long>(1, (n + 127) / 128); }

__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, long n) {
  pdl_enter();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

}  // namespace

cudaError_t launch_add(double* y, const double* x, long n, cudaStream_t s) {
  return launch_k(k_add, dim3(blocks(n)), dim3(128), 0, s, y, x, n);
}

// One stage reversed.  The forward stage k was recorded in t.adj->st[k-1].
int adjoint_stage(wt_tank& t, int k, double dt, const double* alpha, const double* beta) {
  AdjBufs& B = *t.adj;
  const AdjStage& R = B.st[k - 1];
  const long n = t.n, nc = t.ncols;
  const int M1 = t.M1;
  cudaStream_t s = t.s;
  const bool lin = t.opt.linear != 0;
  // geometry of the stage: a = eta^(k), b = eta~ (still water when linear)
  const int prec = t.opt.mode == WT_FP64 ? WT_FP64 : WT_FP32;
  setup_geometry(t, lin ? t.zero_s : R.eta_n, lin ? t.zero_s : R.eta_f, prec, true, true);
  AdjArgs A;
  A.M1 = M1;
  A.nc = nc;
  A.D = t.L64[0].D;
  A.sigma = t.L64[0].sigma;
  A.meta = t.L64[0].meta;
  A.alpha = alpha[k - 1];
  A.beta = beta[k - 1];
  A.dt = dt;
  A.g = t.g;
  A.linear = lin ? 1 : 0;
  auto pass = [&](const double* in, double* out, int rows, int op) {
    RowPass<double> a;
    a.in = in;
    a.out = out;
    a.nrows = rows;
    a.Nin = a.Nout = t.Nx;
    int lg = 0;
    while ((1 << lg) < t.Nx) ++lg;
    a.logNin = a.logNout = lg;
    a.op = op;
    a.kscale = 2.0 * M_PI / t.L;
    a.tw = t.tw64;
    a.logNtw = t.logNtw;
    return a;
  };
  WT_CK(cudaMemsetAsync(B.cols, 0, sizeof(double) * nc * kAdjCols, s));
  double* gA = B.col(0);
  double* gB = B.col(3);
  double* gHX = B.col(6);
  double *ldb = B.col(7), *lexf = B.col(8), *lfe = B.col(9), *lea = B.col(10), *leax = B.col(11),
         *leb = B.col(12), *lebx = B.col(13), *lh0 = B.col(14), *lhx = B.col(15), *tA = B.col(16),
         *tB = B.col(17), *tH = B.col(18), *ex = B.col(19), *let = B.col(20), *lex = B.col(21);
  // projection
  WT_LAUNCH(t, K_STAGE, 8.0 * n * 10, 8.0 * n * 4 * M1, launch_k(k_adj_proj, dim3(blocks(nc)), dim3(128), 0, s, A, B.Lu, B.Lw, B.LKu, B.LKw, R.p, B.LKu1, B.LKw1, B.LGx, B.q, B.lut, B.lwt, gB));
  {
    RowPass<double> a = pass(B.LGx, B.lp, M1, XOP_DERIV);
    a.scale = -1.0;
    a.add = B.q;
    a.epi = EPI_ADD;
    run_rowpass(t, a);
  }
  // the transposed pressure problem
  WT_CK(cudaMemsetAsync(B.lrhs, 0, sizeof(double) * n, s));
  wt_solve_info info{};
  const int st = poisson_solve_device(t, B.lp, B.lrhs, t.opt.tol, &info, true);
  B.last_its = info.iterations;
  B.last_rel = info.rel_residual;
  if (st != WT_OK && st != WT_ENOCONV) return st;
  run_rowpass(t, pass(B.lrhs, B.t1, M1, XOP_DERIV));
  run_rowpass(t, pass(R.p, B.px, M1, XOP_DERIV));
  WT_LAUNCH(t, K_STAGE, 8.0 * n * 16, 8.0 * n * 12 * M1, launch_k(k_adj_rhs, dim3(blocks(nc)), dim3(128), 0, s, A, B.lrhs, B.t1, R.p, B.px, R.us, R.ws, B.LKu1, B.LKw1, B.lut, B.lwt, B.LKu, B.LKw, B.lFu, B.lFw, gA, gB, gHX));
  // forcing
  if (!lin) {
    run_rowpass(t, pass(R.u_f, B.ux, M1, XOP_DERIV));
    run_rowpass(t, pass(R.w_f, B.wx, M1, XOP_DERIV));
  }
  WT_LAUNCH(t, K_STAGE, 8.0 * n * 12, 8.0 * n * 4 * M1, launch_k(k_adj_forcing, dim3(blocks(nc)), dim3(128), 0, s, A, R.u_f, R.w_f, B.ux, B.wx, R.f_eta, B.lFu, B.lFw, B.lut, B.lwt, B.lux, B.lwx, lexf, lfe, ldb, gB));
  if (!lin) {
    RowPass<double> a = pass(B.lux, B.lut, M1, XOP_DERIV);
    a.scale = -1.0;
    a.epi = EPI_ACC;
    run_rowpass(t, a);
    RowPass<double> b = pass(B.lwx, B.lwt, M1, XOP_DERIV);
    b.scale = -1.0;
    b.epi = EPI_ACC;
    run_rowpass(t, b);
  }
  // metric of both geometries, then the free surface
  WT_LAUNCH(t, K_STAGE, 8.0 * nc * 20, 0.0, launch_k(k_adj_metric, dim3(blocks(nc)), dim3(128), 0, s, nc, A.meta, gA, gB, gHX, ldb, lea, leax, leb, lebx, lh0, lhx));
  run_rowpass(t, pass(leax, tA, 1, XOP_DERIV));
  run_rowpass(t, pass(lebx, tB, 1, XOP_DERIV));
  run_rowpass(t, pass(lhx, tH, 1, XOP_DERIV));
  run_rowpass(t, pass(R.eta_f, ex, 1, XOP_DERIV));
  WT_LAUNCH(t, K_STAGE, 8.0 * nc * 16, 0.0, launch_k(k_adj_eta, dim3(blocks(nc)), dim3(128), 0, s, A, B.Le, B.LKe, lea, tA, leb, tB, lh0, tH, lfe, lexf, ex, R.u_f, B.lut, B.lwt, B.lh, let, lex));
  {
    RowPass<double> a = pass(lex, let, 1, XOP_DERIV);
    a.scale = -1.0;
    a.epi = EPI_ACC;
    run_rowpass(t, a);
  }
  // filter on the stage input (symmetric in x; the sigma matrix transposed)
  if (t.opt.filter) {
    RowPass<double> f1 = pass(let, B.Le, 1, XOP_FILTER);
    f1.filt = t.filt_x;
    run_rowpass(t, f1);
    run_col_matrix<double>(t, B.FchebT, M1, M1, B.lut, B.ux, (int)nc, 0);
    RowPass<double> f2 = pass(B.ux, B.Lu, M1, XOP_FILTER);
    f2.filt = t.filt_x;
    run_rowpass(t, f2);
    run_col_matrix<double>(t, B.FchebT, M1, M1, B.lwt, B.wx, (int)nc, 0);
    RowPass<double> f3 = pass(B.wx, B.Lw, M1, XOP_FILTER);
    f3.filt = t.filt_x;
    run_rowpass(t, f3);
  } else {
    WT_CK(cudaMemcpyAsync(B.Le, let, sizeof(double) * nc, cudaMemcpyDeviceToDevice, s));
    WT_CK(cudaMemcpyAsync(B.Lu, B.lut, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    WT_CK(cudaMemcpyAsync(B.Lw, B.lwt, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  return st == WT_ENOCONV ? WT_ENOCONV : WT_OK;
}

}  // namespace wt
