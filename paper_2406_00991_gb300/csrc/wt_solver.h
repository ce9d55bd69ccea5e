// Solver entry points used by the C ABI (wt_capi.cu); defined in wt_solver.cu.
#pragma once

#include "wt_host.h"

namespace wt {

// Launch bookkeeping: every kernel launch is counted; launches of the classes
// selected by prof.mask are bracketed by CUDA events on the tank's stream and
// recorded with their algorithmic bytes and flops.
inline int prof_event(wt_tank& t) {
  auto& P = t.prof;
  if (P.used == P.pool.size()) {
    cudaEvent_t e;
    WT_CK(cudaEventCreate(&e));
    P.pool.push_back(e);
  }
  return (int)P.used++;
}
inline int prof_begin(wt_tank& t, int cat) {
  t.prof.launches++;
  if (!(t.prof.mask & (1u << cat))) return -1;
  const int i = prof_event(t);
  WT_CK(cudaEventRecord(t.prof.pool[i], t.s));
  return i;
}
inline void prof_end(wt_tank& t, int cat, int i0, double bytes, double flops) {
  if (i0 < 0) return;
  const int i1 = prof_event(t);
  WT_CK(cudaEventRecord(t.prof.pool[i1], t.s));
  t.prof.rec.push_back(ProfRec{i0, i1, cat, bytes, flops});
}
#define WT_LAUNCH(t, cat, bytes, flops, call)            \
  do {                                                   \
    const int i0_ = ::wt::prof_begin((t), (cat));        \
    WT_CK(call);                                         \
    ::wt::prof_end((t), (cat), i0_, (bytes), (flops));   \
  } while (0)

// Algorithmic bytes / flops of a spectral row pass: read Nin and write Nout
// per row (plus the epilogue operands); complex FFT 5 N log2 N per row pair.
template <typename T>
inline double rowpass_bytes(const RowPass<T>& a) {
  const double rows = a.nrows;
  double b = rows * a.Nin + rows * a.Nout;
  if (a.epi == EPI_ADD || a.epi == EPI_ACC) b += rows * a.Nout;
  if (a.epi == EPI_RESID) b += 2.0 * rows * a.Nout;
  return b * sizeof(T);
}
template <typename T>
inline double rowpass_flops(const RowPass<T>& a) {
  const double pairs = (a.nrows + 1) / 2;
  return pairs * 5.0 * ((double)a.Nin * a.logNin + (double)a.Nout * a.logNout);
}

template <typename T>
inline void run_rowpass(wt_tank& t, const RowPass<T>& a) {
  WT_LAUNCH(t, K_ROWPASS, rowpass_bytes(a), rowpass_flops(a), launch_rowpass(a, t.s));
}
// sigma-direction matrix applied to every column: read Mi, write Mo values
template <typename T>
inline void run_col_matrix(wt_tank& t, const T* M, int Mo, int Mi, const T* in, T* out, int ncols,
                           int acc) {
  WT_LAUNCH(t, K_COLMAT, (double)sizeof(T) * ncols * (Mi + Mo * (acc ? 2 : 1)),
            2.0 * Mo * Mi * ncols, launch_col_matrix<T>(M, Mo, Mi, in, out, ncols, acc, t.s, df_level(t)));
}

template <typename T> std::vector<Level<T>>& levels(wt_tank& t);
template <typename T> const c2_t<T>* twiddles(wt_tank& t);

void setup_bathymetry(wt_tank& t, const double* h_fine);
// Metric of every level for the surfaces ea (geometry a) and eb (geometry b),
// then (optionally) the smoother's block inverses in `precision` and the
// FP64 LU of the coarsest level.
void setup_geometry(wt_tank& t, const double* ea, const double* eb, int precision, bool blocks,
                    bool coarse);
// The block inverses of every level but the coarsest and the coarsest FP64
// inverse, from the current metric, on stream s.
void setup_blocks(wt_tank& t, int precision, bool blocks, bool coarse, cudaStream_t s);

// tr: the transposed operator A^T (2D) and the V-cycle of A^T (transposed
// smoother blocks and coarsest inverse, the same transfers).
// Options of one operator apply: out2 / Nout2 / op2 give a second transform
// of the last row pass's result (x-rows; write_out = false skips `out`);
// have_dx: L.t1 already holds D_x x.
template <typename T>
struct OpExtra {
  T* out2 = nullptr;
  int Nout2 = 0;
  int op2 = XOP_RESAMPLE;
  bool write_out = true;
  bool have_dx = false;
};
template <typename T> void apply_op(wt_tank& t, int l, const T* x, T* out, const T* f, bool nyq,
                                    bool tr = false, const OpExtra<T>& ex = OpExtra<T>());
template <typename T> void vcycle(wt_tank& t, int l, const T* f, T* x, bool tr = false, bool x0_given = false);
// The preconditioner cycle the options select (V-cycle or full multigrid).
template <typename T> void mg_cycle(wt_tank& t, const T* f, T* x, bool tr = false);
template <typename T>
double fgmres(wt_tank& t, const T* b, T* x, double bnorm, double tol, int maxit, int* its_out,
              bool pre32, bool tr = false);

// Release the captured Arnoldi-step graphs (after option / hierarchy changes).
void destroy_graphs(wt_tank& t);
// Copy the options' grid-barrier wait bound into the tank's barrier state.
void write_barrier_limit(wt_tank& t);

// Solve A p = b on the finest level (device pointers, FP64) with the tank's
// options; x holds the initial guess.  Geometry must be set up already.
int poisson_solve_device(wt_tank& t, const double* b, double* x, double tol, wt_solve_info* info,
                         bool tr = false);

// Reverse one recorded Runge-Kutta stage k of a 2D tank (wt_adjoint.cu):
// adjoints in t.adj (Le, Lu, Lw, LKe, LKu, LKw) go from the stage output to
// its input; t.adj->lh accumulates dJ/dh.  alpha, beta: the 2N coefficients.
int adjoint_stage(wt_tank& t, int k, double dt, const double* alpha, const double* beta);
// y += x (n values, device pointers).
cudaError_t launch_add(double* y, const double* x, long n, cudaStream_t s);

}  // namespace wt
