// Host orchestration of the pressure solve (paper Sec. 4): geometry set-up of
// every level, the matrix-free operator, the p-multigrid V-cycle
// (Algorithm 1), flexible GMRES (Sec. 4.4) and the FP64 iterative
// refinement wrapped around the FP32 solver.  Every step runs in the kernels
// of wt_fft.cu / wt_col.cu / wt_coarse.cu / wt_krylov.cu / wt_rk.cu; the host
// only sequences launches and reads one scalar per Krylov iteration.
#include "wt_host.h"
#include "wt_solver.h"

#include <algorithm>
#include <utility>
#include <cmath>
#include <cstring>

namespace wt {

template <> std::vector<Level<double>>& levels<double>(wt_tank& t) { return t.L64; }
template <> std::vector<Level<float>>& levels<float>(wt_tank& t) { return t.L32; }
template <> const c2_t<double>* twiddles<double>(wt_tank& t) { return t.tw64; }
template <> const c2_t<float>* twiddles<float>(wt_tank& t) { return t.tw32; }

static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename T>
static RowPass<T> xpass(wt_tank& t, const T* in, T* out, int nrows, int Nin, int Nout, int op) {
  RowPass<T> a;
  a.in = in;
  a.out = out;
  a.nrows = nrows;
  a.Nin = Nin;
  a.Nout = Nout;
  a.logNin = ilog2(Nin);
  a.logNout = ilog2(Nout);
  a.op = op;
  a.kscale = (T)(2.0 * M_PI / t.L);
  a.tw = twiddles<T>(t);
  a.logNtw = t.logNtw;
  a.warp = t.opt.warp_fft;
  a.df = df_level(t);
  return a;
}

template <typename T>
static RowPass<T> ypass(wt_tank& t, const T* in, T* out, int planes, int Nxl, int Nin, int Nout, int op) {
  RowPass<T> a = xpass<T>(t, in, out, planes * Nxl, Nin, Nout, op);
  a.ylines = 1;
  a.Nxl = Nxl;
  return a;
}

// ------------------------------------------------------------------ geometry
// Fourier truncation of a fine surface array to level l plus its derivatives.
static void surface_level(wt_tank& t, int l, const double* fine, double* out, double* outx,
                          double* outy) {
  cudaStream_t s = t.s;
  const auto& Lf = t.L64[0];
  const auto& Ll = t.L64[l];
  double* tmp = t.S[l].tmp;
  if (l == 0) {
    WT_CK(cudaMemcpyAsync(out, fine, sizeof(double) * Lf.ncols, cudaMemcpyDeviceToDevice, s));
  } else if (Ll.Ny == 1) {
    run_rowpass(t, xpass<double>(t, fine, out, 1, Lf.Nx, Ll.Nx, XOP_RESAMPLE));
  } else {
    run_rowpass(t, xpass<double>(t, fine, tmp, Lf.Ny, Lf.Nx, Ll.Nx, XOP_RESAMPLE));
    run_rowpass(t, ypass<double>(t, tmp, out, 1, Ll.Nx, Lf.Ny, Ll.Ny, XOP_RESAMPLE));
  }
  if (outx) run_rowpass(t, xpass<double>(t, out, outx, Ll.Ny, Ll.Nx, Ll.Nx, XOP_DERIV));
  if (outy && Ll.Ny > 1)
    run_rowpass(t, ypass<double>(t, out, outy, 1, Ll.Nx, Ll.Ny, Ll.Ny, XOP_DERIV));
}

void setup_bathymetry(wt_tank& t, const double* h_fine) {
  for (size_t l = 0; l < t.L64.size(); ++l)
    surface_level(t, (int)l, h_fine, t.S[l].h, t.S[l].hx, t.L64[l].Ny > 1 ? t.S[l].hy : nullptr);
}

void setup_geometry(wt_tank& t, const double* ea, const double* eb, int precision, bool blocks,
                    bool coarse) {
  const int nl = (int)t.L64.size();
  if (t.Ny == 1) {
    // 2D: every level's truncated surfaces and slopes read only the fine
    // surfaces, so all of them are independent passes of one launch; then
    // one launch fills every level's metric (and its FP32 copy)
    MultiPass<double> mp;
    auto flush = [&]() {
      WT_LAUNCH(t, K_ROWPASS, 0.0, 0.0, launch_rowpass_multi<double>(mp, t.s));
      mp.n = 0;
    };
    auto add = [&](const double* in, double* out, int Nout, int op) {
      if (mp.n == kMaxPasses) flush();
      mp.d[mp.n++] = xpass<double>(t, in, out, 1, t.Nx, Nout, op);
    };
    MetricMulti mm;
    mm.flag = t.dflag;
    for (int l = 0; l < nl; ++l) {
      auto& S = t.S[l];
      auto& L = t.L64[l];
      if (l == 0) {
        add(ea, S.eax, t.Nx, XOP_DERIV);
        add(eb, S.ebx, t.Nx, XOP_DERIV);
      } else {
        add(ea, S.ea, L.Nx, XOP_RESAMPLE);
        add(ea, S.eax, L.Nx, XOP_RESAMPLE_DERIV);
        add(eb, S.eb, L.Nx, XOP_RESAMPLE);
        add(eb, S.ebx, L.Nx, XOP_RESAMPLE_DERIV);
      }
      MetricLevel& M = mm.lv[mm.n++];
      M.ncols = L.ncols;
      M.h = S.h;
      M.hx = S.hx;
      M.hy = nullptr;
      M.ea = l == 0 ? ea : S.ea;
      M.eax = S.eax;
      M.eay = nullptr;
      M.eb = l == 0 ? eb : S.eb;
      M.ebx = S.ebx;
      M.eby = nullptr;
      M.meta = L.meta;
      M.meta32 = precision == WT_FP32 ? t.L32[l].meta : nullptr;
    }
    flush();
    WT_LAUNCH(t, K_STAGE, 8.0 * t.ncols * 23, 20.0 * t.ncols, launch_metric_multi(mm, t.s));
  }
  for (int l = 0; l < nl && t.Ny > 1; ++l) {
    auto& S = t.S[l];
    auto& L = t.L64[l];
    const bool y = L.Ny > 1;
    surface_level(t, l, ea, S.ea, S.eax, y ? S.eay : nullptr);
    surface_level(t, l, eb, S.eb, S.ebx, y ? S.eby : nullptr);
    WT_LAUNCH(t, K_STAGE, 8.0 * L.ncols * 23, 20.0 * L.ncols, launch_metric_fill(L.ncols, S.h, S.hx, y ? S.hy : nullptr, S.ea, S.eax, y ? S.eay : nullptr,
                             S.eb, S.ebx, y ? S.eby : nullptr, L.meta, t.dflag, t.s));
    if (precision == WT_FP32)
      WT_LAUNCH(t, K_STAGE, 12.0 * kMeta * L.ncols, 0.0, (launch_cast<double, float>(L.meta, t.L32[l].meta, (long)kMeta * L.ncols, t.s)));
  }
  setup_blocks(t, precision, blocks, coarse, t.s);
}

void setup_blocks(wt_tank& t, int precision, bool blocks, bool coarse, cudaStream_t s) {
  const int nl = (int)t.L64.size();
  // the spectral smoother alone (smoother = 1) needs column-block inverses
  // only on the levels that smooth by block-Jacobi (the one-launch tail and
  // the levels below spectral_min unknowns), if any
  int l0 = 0;
  if (t.opt.smoother == 1) {
    l0 = nl - 1;
    for (int l = 0; l < nl - 1; ++l)
      if ((t.opt.tail_max > 0 && t.L64[l].n <= t.opt.tail_max) || t.L64[l].n < t.opt.spectral_min) {
        l0 = l;
        break;
      }
  }
  if (blocks && l0 < nl - 1) {
    // the levels' column blocks in one launch
    auto fill = [&](auto& lev, auto tw, auto& m, double wbytes) {
      double bytes = 0.0, flops = 0.0;
      m.nlev = nl - 1 - l0;
      m.start[0] = 0;
      for (int i = 0; i < m.nlev; ++i) {
        auto& L = lev[l0 + i];
        const int l = i;
        m.L[l] = L.view(tw, t.logNtw, t.L);
        m.Binv[l] = L.Binv;
        m.nclass[l] = L.nclass;
        m.cxx[l] = L.cxx;
        m.cyy[l] = L.cyy;
        m.start[l + 1] = m.start[l] + (long)L.ncols * L.nclass;
        m.maxM1 = std::max(m.maxM1, L.M1);
        bytes += wbytes * L.ncols * (L.nclass * L.M1 * L.M1 + kMeta);
        flops += 2.0 * L.nclass * L.ncols * L.M1 * L.M1 * L.M1;
      }
      return std::make_pair(bytes, flops);
    };
    if (precision == WT_FP32) {
      BlockInvMulti<float> m;
      const auto bf = fill(t.L32, t.tw32, m, 4.0);
      WT_LAUNCH(t, K_BLOCKINV, bf.first, bf.second, launch_block_inverse_multi<float>(m, t.dflag, s));
    } else {
      BlockInvMulti<double> m;
      const auto bf = fill(t.L64, t.tw64, m, 8.0);
      WT_LAUNCH(t, K_BLOCKINV, bf.first, bf.second, launch_block_inverse_multi<double>(m, t.dflag, s));
    }
  }
  if (coarse) {
    auto& C = t.L64[nl - 1];
    WT_LAUNCH(t, K_COARSE, 8.0 * t.ncoarse * t.ncoarse, 2.0 / 3.0 * t.ncoarse * t.ncoarse * t.ncoarse, launch_coarse_factor(C.view(t.tw64, t.logNtw, t.L), t.cDx, t.cDy, t.cLU, t.cpiv, t.dflag, s));
  }
}

// ------------------------------------------------------------------ operator
// out = A x (f == nullptr) or out = f - A x; nyq: Nyquist coefficients of out.
template <typename T>
void apply_op(wt_tank& t, int l, const T* x, T* out, const T* f, bool nyq, bool tr, const OpExtra<T>& ex) {
  auto& L = levels<T>(t)[l];
  cudaStream_t s = t.s;
  const auto V = L.view(twiddles<T>(t), t.logNtw, t.L);
  auto extra = [&](RowPass<T>& a) {
    if (!ex.out2) return;
    a.out2 = ex.out2;
    a.Nout2 = ex.Nout2;
    a.logNout2 = ilog2(ex.Nout2);
    a.op2 = ex.op2;
    a.write_out = ex.write_out ? 1 : 0;
  };
  if (tr) {
    // A^T lam = part - D_x mu_x (2D): D_x lam, the column kernel, then the
    // x-derivative of mu_x subtracted in the epilogue of the last row pass
    if (L.Ny != 1) throw WtError{WT_ENOTSUP, "the transposed operator is 2D only"};
    if (!ex.have_dx) run_rowpass(t, xpass<T>(t, x, L.t1, L.M1, L.Nx, L.Nx, XOP_DERIV));
    WT_LAUNCH(t, K_OPCOLS, sizeof(T) * (4.0 * L.n + 7.0 * L.ncols), 6.0 * L.M1 * L.M1 * L.ncols, launch_op_cols_T<T>(V, x, L.t1, L.t2, L.t3, s));
    RowPass<T> a = xpass<T>(t, L.t2, out, L.M1, L.Nx, L.Nx, XOP_DERIV);
    a.scale = T(-1);
    a.add = L.t3;
    a.rhs = f;
    a.epi = f ? EPI_RESID : EPI_ADD;
    a.nyq = nyq ? L.rhoX : nullptr;
    extra(a);
    run_rowpass(t, a);
    return;
  }
  if (L.Ny == 1) {
    if (!ex.have_dx) run_rowpass(t, xpass<T>(t, x, L.t1, L.M1, L.Nx, L.Nx, XOP_DERIV));
    WT_LAUNCH(t, K_OPCOLS, sizeof(T) * (4.0 * L.n + 7.0 * L.ncols), 6.0 * L.M1 * L.M1 * L.ncols, launch_op_cols<T>(V, x, L.t1, nullptr, L.t2, nullptr, L.t3, s, df_level(t)));
    RowPass<T> a = xpass<T>(t, L.t2, out, L.M1, L.Nx, L.Nx, XOP_DERIV);
    a.skip_bc = 1;
    a.Ny = 1;
    a.M1 = L.M1;
    a.add = L.t3;
    a.rhs = f;
    a.epi = f ? EPI_RESID : EPI_ADD;
    a.nyq = nyq ? L.rhoX : nullptr;
    extra(a);
    run_rowpass(t, a);
  } else {
    run_rowpass(t, xpass<T>(t, x, L.t1, L.M1 * L.Ny, L.Nx, L.Nx, XOP_DERIV));
    run_rowpass(t, ypass<T>(t, x, L.t4, L.M1, L.Nx, L.Ny, L.Ny, XOP_DERIV));
    WT_LAUNCH(t, K_OPCOLS, sizeof(T) * (6.0 * L.n + 12.0 * L.ncols), 8.0 * L.M1 * L.M1 * L.ncols, launch_op_cols<T>(V, x, L.t1, L.t4, L.t2, L.t5, L.t3, s, df_level(t)));
    RowPass<T> a = xpass<T>(t, L.t2, L.t6, L.M1 * L.Ny, L.Nx, L.Nx, XOP_DERIV);
    a.skip_bc = 1;
    a.Ny = L.Ny;
    a.M1 = L.M1;
    a.add = L.t3;
    a.epi = EPI_ADD;
    run_rowpass(t, a);
    RowPass<T> b = ypass<T>(t, L.t5, out, L.M1, L.Nx, L.Ny, L.Ny, XOP_DERIV);
    b.skip_bc = 1;
    b.M1 = L.M1;
    b.add = L.t6;
    b.rhs = f;
    b.epi = f ? EPI_RESID : EPI_ADD;
    b.nyq = nyq ? L.rhoY : nullptr;
    run_rowpass(t, b);
    if (nyq) {
      WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (double)(L.M1 * L.Ny) * (L.Nx), 2.0 * (L.M1 * L.Ny) * (L.Nx), launch_nyquist_coef(out, sizeof(T) == 8, L.M1 * L.Ny, L.Nx, L.logNx, L.rhoX, s));
      WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (double)(L.M1) * (L.Ny), 2.0 * (L.M1) * (L.Ny), launch_nyquist_coef(L.rhoX, sizeof(T) == 8, L.M1, L.Ny, L.logNy, L.rhoXY, s));
    }
  }
}

// Nyquist coefficients of an arbitrary field (first sweep on the finest level).
template <typename T>
static void nyquist_of(wt_tank& t, Level<T>& L, const T* f) {
  cudaStream_t s = t.s;
  if (L.Ny == 1) {
    WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (double)(L.M1) * (L.Nx), 2.0 * (L.M1) * (L.Nx), launch_nyquist_coef(f, sizeof(T) == 8, L.M1, L.Nx, L.logNx, L.rhoX, s));
  } else {
    // y-Nyquist per (m, jx) line via a y-pass with an identity spectrum
    RowPass<T> b = ypass<T>(t, f, L.t6, L.M1, L.Nx, L.Ny, L.Ny, XOP_NONE);
    b.nyq = L.rhoY;
    run_rowpass(t, b);
    WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (double)(L.M1 * L.Ny) * (L.Nx), 2.0 * (L.M1 * L.Ny) * (L.Nx), launch_nyquist_coef(f, sizeof(T) == 8, L.M1 * L.Ny, L.Nx, L.logNx, L.rhoX, s));
    WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (double)(L.M1) * (L.Ny), 2.0 * (L.M1) * (L.Ny), launch_nyquist_coef(L.rhoX, sizeof(T) == 8, L.M1, L.Ny, L.logNy, L.rhoXY, s));
  }
}

// ------------------------------------------------------------------ V-cycle
// One sweep of the mean-depth spectral smoother: x = omega_s S f from x = 0
// (first) or x += omega_s S (f - A x) (wt_spec.cu).
template <typename T>
static void spectral_sweep(wt_tank& t, int l, T* x, const T* f, bool first, bool tr, bool have_dx) {
  auto& L = levels<T>(t)[l];
  if (!L.Stab) throw WtError{WT_EINVAL, "spectral smoother tables are not built"};
  const T* r = f;
  if (!first) {
    OpExtra<T> ex;
    ex.have_dx = have_dx;
    apply_op<T>(t, l, x, L.r, f, false, tr, ex);
    r = L.r;
  }
  SpecArgs<T> a;
  a.Nx = L.Nx; a.Ny = L.Ny; a.M1 = L.M1; a.logNx = L.logNx; a.logNy = L.logNy;
  a.r = r; a.x = x; a.spec = L.spec; a.tab = L.Stab; a.sidx = L.sidx;
  a.scale = (T)(t.opt.omega_s / ((double)L.Nx * L.Ny));
  a.first = first ? 1 : 0;
  a.tr = tr ? 1 : 0;
  a.tw = twiddles<T>(t);
  a.logNtw = t.logNtw;
  const double nh = (double)L.M1 * L.Ny * (L.Nx / 2 + 1);
  WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (3.0 * L.n + 8.0 * nh), 2.0 * 8.0 * nh * L.M1,
            launch_spectral_smooth<T>(a, t.s));
  // kernels of the pass: x forward, y forward and inverse (3D), columns, x inverse
  t.prof.launches += (L.Ny > 1 ? 5 : 3) - 1;
}

template <typename T>
static void smooth_bj(wt_tank& t, int l, T* x, const T* f, bool first, bool f_has_nyq, bool tr,
                      bool have_dx);

// One smoothing sweep of the kind the options select: damped block-Jacobi
// (0), the mean-depth spectral smoother (1), or a block-Jacobi sweep then a
// spectral sweep (2).  first: x = 0 on entry.
template <typename T>
static void smooth(wt_tank& t, int l, T* x, const T* f, bool first, bool f_has_nyq, bool tr,
                   bool have_dx = false) {
  // levels below spectral_min unknowns smooth by block-Jacobi alone
  const int kind = levels<T>(t)[l].n < t.opt.spectral_min ? 0 : t.opt.smoother;
  if (kind == 1) {
    spectral_sweep<T>(t, l, x, f, first, tr, have_dx);
    return;
  }
  smooth_bj<T>(t, l, x, f, first, f_has_nyq, tr, have_dx);
  if (kind == 2) spectral_sweep<T>(t, l, x, f, false, tr, false);
}

template <typename T>
static void smooth_bj(wt_tank& t, int l, T* x, const T* f, bool first, bool f_has_nyq, bool tr,
                      bool have_dx) {
  auto& L = levels<T>(t)[l];
  const auto V = L.view(twiddles<T>(t), t.logNtw, t.L);
  const T om = (T)t.opt.omega;
  if (first) {
    const bool y = L.Ny > 1;
    if (f_has_nyq) nyquist_of<T>(t, L, f);
    WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (2.0 * L.n + (double)L.nclass * L.M1 * L.M1 * L.ncols), 2.0 * L.nclass * L.M1 * L.M1 * L.ncols, launch_smooth_cols<T>(V, f, f_has_nyq ? L.rhoX : nullptr, (f_has_nyq && y) ? L.rhoY : nullptr,
                                (f_has_nyq && y) ? L.rhoXY : nullptr, L.Binv, L.nclass, x, om, 1, tr, t.s));
  } else {
    OpExtra<T> ex;
    ex.have_dx = have_dx;
    apply_op<T>(t, l, x, L.r, f, true, tr, ex);
    WT_LAUNCH(t, K_SMOOTH, sizeof(T) * (3.0 * L.n + (double)L.nclass * L.M1 * L.M1 * L.ncols), 2.0 * L.nclass * L.M1 * L.M1 * L.ncols, launch_smooth_cols<T>(V, L.r, L.rhoX, L.Ny > 1 ? L.rhoY : nullptr, L.Ny > 1 ? L.rhoXY : nullptr,
                                L.Binv, L.nclass, x, om, 0, tr, t.s));
  }
}

template <typename T>
static void restrict_to(wt_tank& t, int l, const T* r) {
  auto& F = levels<T>(t)[l];
  auto& C = levels<T>(t)[l + 1];
  cudaStream_t s = t.s;
  const T* cur = r;
  if (C.Nx != F.Nx) {
    // with identity sigma transfers the last Fourier truncation writes C.f
    const bool direct = F.sig_id;
    T* dx = (direct && F.Ny == 1) ? C.f : F.t4;
    run_rowpass(t, xpass<T>(t, cur, dx, F.M1 * F.Ny, F.Nx, C.Nx, XOP_RESAMPLE));
    cur = dx;
    if (F.Ny > 1) {
      T* dy = direct ? C.f : F.t5;
      run_rowpass(t, ypass<T>(t, cur, dy, F.M1, C.Nx, F.Ny, C.Ny, XOP_RESAMPLE));
      cur = dy;
    }
    if (direct) return;
  }
  run_col_matrix<T>(t, F.Rsig, C.M1, F.M1, cur, C.f, C.ncols, 0);
}

// x += P e_c.  With dx_out (2D, Fourier-refined levels) the same row pass
// also writes D_x of the corrected x there (for the next smoothing sweep);
// returns whether it did.
template <typename T>
static bool prolong_add(wt_tank& t, int l, T* x, T* dx_out = nullptr) {
  auto& F = levels<T>(t)[l];
  auto& C = levels<T>(t)[l + 1];
  cudaStream_t s = t.s;
  if (C.Nx == F.Nx) {
    run_col_matrix<T>(t, F.Psig, F.M1, C.M1, C.x, x, F.ncols, 1);
    return false;
  }
  const T* cur = C.x;                       // identity sigma transfer: read e_c itself
  if (!F.sig_id) {
    run_col_matrix<T>(t, F.Psig, F.M1, C.M1, C.x, F.t4, C.ncols, 0);
    cur = F.t4;
  }
  if (F.Ny > 1) {
    run_rowpass(t, ypass<T>(t, cur, F.t5, F.M1, C.Nx, C.Ny, F.Ny, XOP_RESAMPLE));
    cur = F.t5;
  }
  RowPass<T> a = xpass<T>(t, cur, x, F.M1 * F.Ny, C.Nx, F.Nx, XOP_RESAMPLE);
  a.epi = EPI_ACC;
  const bool fuse = dx_out && F.Ny == 1;
  if (fuse) {
    a.out2 = dx_out;
    a.Nout2 = F.Nx;
    a.logNout2 = ilog2(F.Nx);
    a.op2 = XOP_DERIV;
  }
  run_rowpass(t, a);
  return fuse;
}

template <typename T> static TailLevel<T>* tail_desc(wt_tank& t);
template <> TailLevel<double>* tail_desc<double>(wt_tank& t) { return t.tl64; }
template <> TailLevel<float>* tail_desc<float>(wt_tank& t) { return t.tl32; }

// First level handled by the single-launch tail of the V-cycle (one CTA, or
// one thread-block cluster with tail_cluster >= 2); -1: none.
// The tail smooths by block-Jacobi; with the spectral smoother (1 or 2) the
// levels above it keep the spectral sweeps.
template <typename T>
static int tail_level(wt_tank& t, bool tr) {
  if (t.opt.tail_max <= 0 || tr) return -1;
  auto& lev = levels<T>(t);
  for (size_t l = 0; l < lev.size(); ++l)
    if (lev[l].n <= t.opt.tail_max) return (int)l;
  return -1;
}

// x0_given: x holds an initial state (the full-multigrid cycle), so the
// first smoothing sweep works on the residual f - A x instead of assuming
// x = 0, and the one-launch schedules (which assume x = 0) are not used at
// this level.
template <typename T>
void vcycle(wt_tank& t, int l, const T* f, T* x, bool tr, bool x0_given) {
  static const char* const kLevelNames[kMaxLevels] = {
      "wt vcycle level 0",  "wt vcycle level 1",  "wt vcycle level 2",  "wt vcycle level 3",
      "wt vcycle level 4",  "wt vcycle level 5",  "wt vcycle level 6",  "wt vcycle level 7",
      "wt vcycle level 8",  "wt vcycle level 9",  "wt vcycle level 10", "wt vcycle level 11",
      "wt vcycle level 12", "wt vcycle level 13", "wt vcycle level 14", "wt vcycle level 15"};
  NvtxRange range(kLevelNames[l < kMaxLevels ? l : kMaxLevels - 1]);
  auto& lev = levels<T>(t);
  const int nl = (int)lev.size();
  auto& L = lev[l];
  if (l == 0 && !tr && t.opt.vcycle_grid && !x0_given && t.opt.smoother == 0) {
    // the whole cycle in one cooperative launch; the dynamic shared memory
    // holds the largest unprefetched row pair (twice the finest row plus
    // half a row of twiddles) and the small per-phase tables
    const int Nmax = std::max(L.Nx, L.Ny);
    const size_t need = (size_t)(2 * Nmax + Nmax / 2) * sizeof(c2_t<T>);
    const size_t smem = std::max<size_t>(need, 48 * 1024);
    if (smem <= 200 * 1024) {
      TailArgs<T> a;
      a.lv = tail_desc<T>(t);
      a.l0 = 0;
      a.nl = nl;
      a.f0 = f;
      a.x0 = x;
      a.f0_nyq = 1;
      a.omega = (T)t.opt.omega;
      a.nu1 = t.opt.nu1;
      a.nu2 = t.opt.nu2;
      a.AinvT = t.cLU;
      a.smem = (int)smem;
      WT_LAUNCH(t, K_TAIL, 0.0, 0.0, launch_vcycle_grid<T>(a, L.Ny > 1 ? 3 : 2, t.gbar, t.dflag, t.s));
      return;
    }
  }
  if (l == tail_level<T>(t, tr) && !x0_given) {
    TailArgs<T> a;
    a.lv = tail_desc<T>(t);
    a.l0 = l;
    a.nl = nl;
    a.f0 = f;
    a.x0 = x;
    a.f0_nyq = (l == 0) || (lev[l - 1].Nx == L.Nx);
    a.omega = (T)t.opt.omega;
    a.nu1 = t.opt.nu1;
    a.nu2 = t.opt.nu2;
    a.AinvT = t.cLU;
    a.smem = 96 * 1024;
    double bytes = 0.0;
    for (int k = l; k < nl; ++k)
      bytes += sizeof(T) * (double)lev[k].n * (14.0 * (t.opt.nu1 + t.opt.nu2) + 16.0) +
               sizeof(T) * (double)lev[k].nclass * lev[k].M1 * lev[k].M1 * lev[k].ncols *
                   (t.opt.nu1 + t.opt.nu2);
    if (t.opt.tail_cluster >= 2)
      WT_LAUNCH(t, K_TAIL, bytes, 0.0, launch_vcycle_cluster<T>(a, L.Ny > 1 ? 3 : 2, t.opt.tail_cluster, t.s));
    else
      WT_LAUNCH(t, K_TAIL, bytes, 0.0, launch_vcycle_tail<T>(a, L.Ny > 1 ? 3 : 2, t.s));
    return;
  }
  if (l == nl - 1) {
    WT_LAUNCH(t, K_COARSE, 8.0 * L.n * L.n + 2.0 * sizeof(T) * L.n, 2.0 * L.n * L.n, launch_coarse_solve<T>((int)L.n, t.cLU, t.cpiv, tr ? 1 : 0, f, x, t.s));
    return;
  }
  // pre-smoothing (nu1 sweeps from a zero initial state).  A right-hand side
  // that arrived through a Fourier truncation has no x- (y-) Nyquist content;
  // the finest level and levels reached by sigma-only coarsening may have some.
  const bool f_nyq = (l == 0) || (lev[l - 1].Nx == L.Nx);
  if (t.opt.nu1 > 0) {
    smooth<T>(t, l, x, f, !x0_given, f_nyq, tr);
    for (int i = 1; i < t.opt.nu1; ++i) smooth<T>(t, l, x, f, false, false, tr);
    auto& C = lev[l + 1];
    if (L.Ny == 1 && C.Nx != L.Nx) {
      // r = f - A u and its Fourier truncation in the same row pass; only the
      // truncated rows are stored, then the Chebyshev truncation
      OpExtra<T> ex;
      ex.out2 = L.sig_id ? C.f : L.t4;          // identity sigma transfer: straight to C.f
      ex.Nout2 = C.Nx;
      ex.op2 = XOP_RESAMPLE;
      ex.write_out = false;
      apply_op<T>(t, l, x, L.r, f, false, tr, ex);
      if (!L.sig_id) run_col_matrix<T>(t, L.Rsig, C.M1, L.M1, L.t4, C.f, C.ncols, 0);
    } else {
      apply_op<T>(t, l, x, L.r, f, false, tr);  // r = f - A u
      restrict_to<T>(t, l, L.r);
    }
  } else if (x0_given) {
    apply_op<T>(t, l, x, L.r, f, false, tr);  // r = f - A u
    restrict_to<T>(t, l, L.r);
  } else {
    WT_CK(cudaMemsetAsync(x, 0, sizeof(T) * L.n, t.s));
    restrict_to<T>(t, l, f);
  }
  vcycle<T>(t, l + 1, lev[l + 1].f, lev[l + 1].x, tr, false);
  const bool dx = prolong_add<T>(t, l, x, t.opt.nu2 > 0 ? L.t1 : nullptr);   // u = u + P e_c
  for (int i = 0; i < t.opt.nu2; ++i) smooth<T>(t, l, x, f, false, false, tr, dx && i == 0);
}

// Full multigrid (Algorithm 2): the right-hand side restricted to every
// level, the coarsest level solved, then on each finer level the prolongated
// coarse result as the initial state of one V-cycle.  Linear in f, so it is
// a fixed preconditioner like the V-cycle.
template <typename T>
void fmg(wt_tank& t, const T* f, T* x, bool tr) {
  auto& lev = levels<T>(t);
  const int nl = (int)lev.size();
  if (nl == 1) {
    vcycle<T>(t, 0, f, x, tr, false);
    return;
  }
  restrict_to<T>(t, 0, f);                                   // f_1 = R f_0
  for (int l = 1; l < nl - 1; ++l) restrict_to<T>(t, l, lev[l].f);   // f_{l+1} = R f_l
  vcycle<T>(t, nl - 1, lev[nl - 1].f, lev[nl - 1].x, tr, false);   // coarsest: direct solve
  for (int l = nl - 2; l >= 0; --l) {
    T* xl = l == 0 ? x : lev[l].x;
    const T* fl = l == 0 ? f : lev[l].f;
    WT_CK(cudaMemsetAsync(xl, 0, sizeof(T) * lev[l].n, t.s));
    prolong_add<T>(t, l, xl);                                // u_l = P u_{l+1}
    vcycle<T>(t, l, fl, xl, tr, true);                       // u_l = Vcycle(l, u_l, f_l)
  }
}

// The preconditioner of the Krylov solver: one V-cycle (Algorithm 1) or one
// full-multigrid cycle (Algorithm 2), as the options select.
template <typename T>
void mg_cycle(wt_tank& t, const T* f, T* x, bool tr) {
  if (t.opt.cycle == 1) fmg<T>(t, f, x, tr);
  else vcycle<T>(t, 0, f, x, tr, false);
}

// ------------------------------------------------------------------ norms
template <typename T>
static double norm2(wt_tank& t, const T* v, long n) {
  WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n * ((0) + 1), 2.0 * n * ((0) + 1), launch_dots<T>(v, nullptr, 0, 0, n, t.partial, t.nblk, 1, t.s));
  WT_LAUNCH(t, K_KRYLOV, 8.0 * t.nblk, 0.0, launch_gmres_init(t.stN, t.partial, t.nblk, 1, 1.0, 0.0, t.s));
  WT_CK(cudaMemcpyAsync(t.hst, t.stN, sizeof(double) * 4, cudaMemcpyDeviceToHost, t.s));
  WT_CK(cudaStreamSynchronize(t.s));
  return t.hst[0];
}

// ------------------------------------------------------------------ FGMRES
template <typename T> static T* Vbuf(wt_tank& t);
template <> double* Vbuf<double>(wt_tank& t) { return t.V64; }
template <> float* Vbuf<float>(wt_tank& t) { return t.V32; }
template <typename T> static T* Zbuf(wt_tank& t);
template <> double* Zbuf<double>(wt_tank& t) { return t.Z64; }
template <> float* Zbuf<float>(wt_tank& t) { return t.Z32; }

// Preconditioner z = M^{-1} v: one V-cycle in the precision of the Krylov
// vectors, or (pre32 with T = double) an FP32 V-cycle on the rounded vector
// t.b32 = (float)v, which the kernel that produced v has already written,
// with the correction widened back to FP64.
template <typename T>
static void precondition(wt_tank& t, const T* v, T* z, bool pre32, bool tr);
template <>
void precondition<float>(wt_tank& t, const float* v, float* z, bool, bool tr) {
  mg_cycle<float>(t, v, z, tr);
}
template <>
void precondition<double>(wt_tank& t, const double* v, double* z, bool pre32, bool tr) {
  if (!pre32) {
    mg_cycle<double>(t, v, z, tr);
    return;
  }
  const long n = t.n;
  mg_cycle<float>(t, t.b32, t.e32, tr);
  WT_LAUNCH(t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<float, double>(t.e32, z, n, nullptr, 0, t.s)));
}

// Drop every captured Arnoldi-step graph (new options, possibly a new
// hierarchy, or the tank's end): the next solve captures them again.
void destroy_graphs(wt_tank& t) {
  for (auto& v : t.graphs) {
    for (auto& g : v)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    v.clear();
  }
}

// Arnoldi step j: z_j = M^{-1} v_j, w = A z_j, CGS2 against v_0..v_j,
// Givens update, v_{j+1} = w / h_{j+1,j}.  Device-only: capturable.
template <typename T>
static void arnoldi_step(wt_tank& t, int j, bool pre32, bool tr) {
  const long n = levels<T>(t)[0].n;
  const int m = t.opt.restart;
  T* V = Vbuf<T>(t);
  T* Z = Zbuf<T>(t);
  T* vj = V + (long)j * n;
  T* zj = Z + (long)j * n;
  T* w = V + (long)(j + 1) * n;
  precondition<T>(t, vj, zj, pre32, tr);                 // z_j = M^{-1} v_j
  apply_op<T>(t, 0, zj, w, nullptr, false, tr);          // w = A z_j
  // CGS2: h1 = V^T w (one launch, summed by its last CTA), then w -= V h1,
  // h2 = V^T w, ||w|| and the Givens update of column j (one launch)
  WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n * (j + 2), 2.0 * n * (j + 1),
            launch_dots_sum<T>(w, V, n, j + 1, n, t.partial, t.nblk, 0, t.st + 8, t.tickets, t.s));
  WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n * (j + 3), 4.0 * n * (j + 2),
            launch_update_dots_arnoldi<T>(w, V, n, j + 1, n, t.st, t.partial, t.nblk, j, m, t.tickets + 1, t.s));
  WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n * (j + 3) + (pre32 ? 4.0 * n : 0.0), 2.0 * n * (j + 2),
            launch_update_normalize<T>(w, V, n, j + 1, n, t.st + 72, t.st + 2, w, pre32 ? t.b32 : nullptr, t.s));
}

// Run Arnoldi step j, replaying its CUDA graph (captured at first use) unless
// per-launch timing is on.
template <typename T>
static void arnoldi_step_graph(wt_tank& t, int j, bool pre32, bool tr) {
  const int key = (sizeof(T) == 4 ? 2 : (pre32 ? 1 : 0)) + (tr ? 3 : 0);
  if (!t.use_graphs || t.prof.mask != 0) {
    arnoldi_step<T>(t, j, pre32, tr);
    return;
  }
  auto& gv = t.graphs[key];
  if ((int)gv.size() < t.opt.restart) gv.resize(t.opt.restart);
  IterGraph& g = gv[j];
  if (!g.exec) {
    const long l0 = t.prof.launches;
    cudaGraph_t graph = nullptr;
    WT_CK(cudaStreamBeginCapture(t.s, cudaStreamCaptureModeThreadLocal));
    try {
      arnoldi_step<T>(t, j, pre32, tr);
    } catch (...) {
      cudaStreamEndCapture(t.s, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    WT_CK(cudaStreamEndCapture(t.s, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    WT_CK(e);
    g.kernels = t.prof.launches - l0;
    t.prof.launches = l0;
  }
  WT_CK(cudaGraphLaunch(g.exec, t.s));
  t.prof.launches += g.kernels;
}

// Right-preconditioned flexible GMRES(m) on the finest level of precision T:
// x is the initial guess and the result; returns the last true relative
// residual ||b - A x|| / bnorm computed in precision T.  With pre32 the
// preconditioner is the FP32 V-cycle: every Arnoldi step then refines the
// FP64 iterate with an FP32 correction (flexible Krylov iterative refinement).
template <typename T>
double fgmres(wt_tank& t, const T* b, T* x, double bnorm, double tol, int maxit, int* its_out,
              bool pre32, bool tr) {
  auto& L0 = levels<T>(t)[0];
  const long n = L0.n;
  const int m = t.opt.restart;
  T* V = Vbuf<T>(t);
  T* Z = Zbuf<T>(t);
  int its = 0;
  double rel = 1.0;
  for (;;) {
    {
      ResidualScope rs(t);                                     // the true residual
      apply_op<T>(t, 0, x, V, b, false, tr);                   // r = b - A x -> V_0
    }
    WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n, 2.0 * n,
              launch_dots<T>(V, nullptr, 0, 0, n, t.partial, t.nblk, 1, t.s));
    WT_LAUNCH(t, K_KRYLOV, 8.0 * t.nblk, 0.0,
              launch_gmres_init(t.st, t.partial, t.nblk, m, bnorm, tol, t.s));
    WT_CK(cudaMemcpyAsync(t.hst, t.st, sizeof(double) * 6, cudaMemcpyDeviceToHost, t.s));
    WT_CK(cudaStreamSynchronize(t.s));
    rel = bnorm > 0 ? t.hst[0] / bnorm : 0.0;
    if (rel <= tol || its >= maxit || t.hst[0] == 0.0 || !std::isfinite(rel)) break;
    // v_0 = r / beta (and its FP32 rounding for the FP32 V-cycle)
    WT_LAUNCH(t, K_KRYLOV, 2.0 * sizeof(T) * n + (pre32 ? 4.0 * n : 0.0), (double)n,
              launch_update_normalize<T>(V, V, n, 0, n, t.st + 72, t.st + 2, V, pre32 ? t.b32 : nullptr, t.s));
    int k = 0;
    for (int j = 0; j < m; ++j) {
      arnoldi_step_graph<T>(t, j, pre32, tr);
      WT_CK(cudaMemcpyAsync(t.hst, t.st, sizeof(double) * 6, cudaMemcpyDeviceToHost, t.s));
      WT_CK(cudaStreamSynchronize(t.s));
      ++its;
      k = j + 1;
      if (t.hst[3] != 0.0 || its >= maxit) break;
    }
    WT_LAUNCH(t, K_KRYLOV, 8.0 * k * k, (double)k * k, launch_gmres_solve_y(t.st, k, m, t.s));
    WT_LAUNCH(t, K_KRYLOV, sizeof(T) * (double)n * (k + 2), 2.0 * n * k,
              launch_lincomb<T>(x, Z, n, k, n, t.st + 328, t.s));
  }
  if (its_out) *its_out = its;
  return rel;
}

// The grid barrier's wait bound from the options (0: the compiled default).
void write_barrier_limit(wt_tank& t) {
  const long long lim = t.opt.barrier_cycles;
  WT_CK(cudaMemcpyAsync(&t.gbar->limit, &lim, sizeof(lim), cudaMemcpyHostToDevice, t.s));
  WT_CK(cudaStreamSynchronize(t.s));
}

// ------------------------------------------------------------------ solves
int poisson_solve_device(wt_tank& t, const double* b, double* x, double tol, wt_solve_info* info,
                         bool tr) {
  NvtxRange range("wt poisson solve");
  const long n = t.n;
  const double bn = norm2<double>(t, b, n);
  int its_total = 0, refinements = 0;
  double rel = 0.0;
  int status = WT_OK;
  if (!std::isfinite(bn)) {
    // a non-finite right-hand side (state or input): nothing to iterate on
    status = WT_EBREAK;
    rel = bn;
  } else if (bn == 0.0) {
    WT_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, t.s));
    rel = 0.0;
  } else {
    // WT_FP64: FP64 V-cycle.  WT_MIXED: FP32 V-cycle inside the FP64 flexible
    // GMRES, i.e. FP64 residuals and Krylov basis, FP32 preconditioner.
    if (t.opt.mode == WT_REFINE) {
      // FP64 iterative refinement: r = b - A x (FP64); A e = r / |r| solved by
      // FP32 flexible GMRES with the FP32 V-cycle to inner_tol; x += |r| e.
      for (;;) {
        {
          ResidualScope rs(t);                                 // the true residual
          apply_op<double>(t, 0, x, t.r64, b, false, tr);
        }
        const double rn = norm2<double>(t, t.r64, n);      // |r| also left in stN[0]
        rel = rn / bn;
        if (rel <= tol || refinements >= t.opt.max_ir || its_total >= t.opt.max_it || !std::isfinite(rel))
          break;
        WT_LAUNCH(t, K_KRYLOV, 12.0 * n, (double)n,
                  (launch_convert<double, float>(t.r64, t.b32, n, t.stN, 1, t.s)));
        WT_CK(cudaMemsetAsync(t.e32, 0, sizeof(float) * n, t.s));
        int its = 0;
        fgmres<float>(t, t.b32, t.e32, 1.0, t.opt.inner_tol,
                      std::min(t.opt.restart, t.opt.max_it - its_total), &its, false, tr);
        its_total += its;
        WT_LAUNCH(t, K_KRYLOV, 20.0 * n, 2.0 * n, launch_axpy_from<float>(x, t.e32, n, t.stN, t.s));
        ++refinements;
      }
    } else {
      int its = 0;
      rel = fgmres<double>(t, b, x, bn, tol, t.opt.max_it, &its, t.opt.mode == WT_MIXED, tr);
      its_total = its;
    }
    if (!(rel <= tol)) status = WT_ENOCONV;
    // a non-finite residual cannot improve: both loops stop on it
    if (!std::isfinite(rel)) status = WT_EBREAK;
  }
  WT_CK(cudaMemcpyAsync(t.hflag, t.dflag, sizeof(int), cudaMemcpyDeviceToHost, t.s));
  WT_CK(cudaStreamSynchronize(t.s));
  const int fl = *t.hflag;
  if (fl & 7) status = WT_EBREAK;
  if (fl & 32) {
    status = WT_ETIMEOUT;                 // a grid barrier gave up: reset it
    WT_CK(cudaMemsetAsync(t.gbar, 0, sizeof(GridBar), t.s));
    write_barrier_limit(t);
  }
  if (fl) {                               // reported once; the next call starts clean
    WT_CK(cudaMemsetAsync(t.dflag, 0, sizeof(int), t.s));
    WT_CK(cudaStreamSynchronize(t.s));
  }
  t.solves += 1;
  t.iterations += its_total;
  if (info) {
    info->iterations = its_total;
    info->rel_residual = rel;
    info->status = status;
    info->refinements = refinements;
  }
  return status;
}

template void apply_op<double>(wt_tank&, int, const double*, double*, const double*, bool, bool,
                               const OpExtra<double>&);
template void apply_op<float>(wt_tank&, int, const float*, float*, const float*, bool, bool,
                              const OpExtra<float>&);
template void vcycle<double>(wt_tank&, int, const double*, double*, bool, bool);
template void vcycle<float>(wt_tank&, int, const float*, float*, bool, bool);
template void mg_cycle<double>(wt_tank&, const double*, double*, bool);
template void mg_cycle<float>(wt_tank&, const float*, float*, bool);

}  // namespace wt
