// Internal declarations shared by the CUDA translation units of libwt.
//
// Device data of one multigrid level is described by LevelView<T>, passed by
// value to kernels.  Field arrays are [M1][Ny][Nx] (x fastest), M1 = Nz + 1,
// sigma index 0 = free surface.  Per-column metric data is struct-of-arrays:
// meta[f * ncols + c] for field f of column c = jy * Nx + jx.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace wt {

// ------------------------------------------------------------ metric fields
// sigma_x^g(m) = AX_g - sigma_m BX_g, sigma_y^g(m) = AY_g - sigma_m BY_g and
// sigma_z^g = Z_g (Eq. 1_Scoef) with AX = h_x/d, BX = d_x/d, AY = h_y/d,
// BY = d_y/d, Z = 1/d for geometry g in {a, b}; HX, HY = bottom slope.
enum MetaField {
  M_AXa = 0, M_BXa, M_AYa, M_BYa, M_Za,
  M_AXb, M_BXb, M_AYb, M_BYb, M_Zb,
  M_HX, M_HY, M_D_A, M_D_B,   // d^a, d^b (for sigma_t and checks)
  kMeta
};

constexpr int kMaxLevels = 16;
constexpr int kMaxM1 = 33;      // Nz <= 32

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2_t = typename C2<T>::type;

template <typename T>
struct LevelView {
  int Nx, Ny, Nz, M1;
  int logNx, logNy;
  int ncols;          // Nx * Ny
  long n;             // M1 * ncols
  T L;
  const T* sigma;     // [M1]
  const T* D;         // [M1*M1] d/dsigma on the CGL nodes
  const T* D2;        // [M1*M1] D*D
  const T* DSD;       // [M1*M1] D*diag(sigma)*D
  const T* meta;      // [kMeta * ncols]
  const c2_t<T>* tw;  // twiddles exp(-2 pi i t / Ntw), t < Ntw/2
  int logNtw;
};

// Nyquist classes of the column-block smoother: 2D uses {00, N0}; 3D uses
// {00, N0, 0N, NN} (x-Nyquist, y-Nyquist, both).
constexpr int kMaxClasses = 4;

// Record the calling thread's last error for wt_last_error (wt_capi.cu).
int set_error(int code, const char* msg);

// ------------------------------------------------------------------ launchers
// All launchers enqueue on `s` and return cudaGetLastError().

// Spectral x-row / y-line passes (wt_fft.cu).
enum XEpi { EPI_STORE = 0, EPI_ADD = 1, EPI_RESID = 2, EPI_ACC = 3 };
// XOP_RESAMPLE_DERIV: the derivative of the Fourier-resampled row (truncate or
// zero-pad to Nout, then multiply by i kappa) in one transform pair.
enum XOp { XOP_DERIV = 0, XOP_RESAMPLE = 1, XOP_FILTER = 2, XOP_NONE = 3, XOP_RESAMPLE_DERIV = 4 };

template <typename T>
struct RowPass {
  // rows of length Nin read from `in` (row stride Nin), written with length
  // Nout to `out` (row stride Nout).  Row r of a field is (m, jy) = (r / Ny, r % Ny)
  // for x-rows; for y-lines the pass runs along y with x as the batch index.
  const T* in = nullptr;
  T* out = nullptr;
  const T* add = nullptr;      // EPI_ADD / EPI_RESID addend
  const T* rhs = nullptr;      // EPI_RESID: out = rhs - (add + D in)
  int nrows = 0;               // rows (x) or planes*Nx (y)
  int Nin = 0, Nout = 0;       // transform sizes
  int logNin = 0, logNout = 0;
  int Ny = 1;                  // for the sigma index of a row (skip_bc)
  int M1 = 0;                  // sigma levels (skip_bc)
  int skip_bc = 0;             // derivative term is zero on sigma rows 0 and M1-1
  int op = XOP_DERIV;
  int epi = EPI_STORE;
  T kscale = 1;                // 2 pi / L
  T scale = 1;                 // extra factor on the transformed term
  const T* filt = nullptr;     // XOP_FILTER: response per |n|, size Nin/2+1
  T* nyq = nullptr;            // optional per-row Nyquist coefficient of the output
  const c2_t<T>* tw = nullptr;
  int logNtw = 0;
  // y-line geometry (ylines = 1): lines along y of a [planes][Ny][Nx] array
  int ylines = 0, Nxl = 0;     // x extent of each plane
  int prefetch = 1;            // fetch epilogue operands with the inputs (needs smem)
  // Optional second transform of the epilogue's result (x-rows only): out2
  // receives it resampled to Nout2 (op2 = XOP_RESAMPLE) or differentiated
  // (op2 = XOP_DERIV, Nout2 = Nout); write_out = 0 skips storing `out`.
  T* out2 = nullptr;
  int Nout2 = 0, logNout2 = 0;
  int op2 = XOP_RESAMPLE;
  int write_out = 1;
  int warp = 1;                // derivative passes over many lines may use the warp kernels
  int df = 0;                  // FP64 derivative passes may run in double-float arithmetic
};

// Raise kernel `fn`'s dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute belongs to (kernel, device), so the cache of
// what has been set is kept per pair (wt_launch.cu); thread-safe.
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes);
// Allow cluster sizes above the portable 8 for kernel `fn` on the current
// device (cached per (kernel, device) likewise).
cudaError_t ensure_nonportable_cluster(const void* fn);

// Streaming multiprocessors of the current device (cached per device): grid
// caps are multiples of it.
int sm_count();

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while its predecessor in
// the stream still runs; every kernel that launch_k starts therefore begins
// with pdl_enter(): griddepcontrol.wait (returns once every prerequisite grid
// has completed and its memory operations are visible, and at once when the
// kernel was launched without the attribute) before it touches global
// memory.  A grid of at most half as many CTAs as the device has SMs then
// signals griddepcontrol.launch_dependents, so that the next kernel's CTAs
// are made resident on the idle SMs while it runs; a wider grid does not
// (its dependent would be packed onto the SMs that free up first and share
// them with the primary's last CTAs: measured slower on 3D levels).  The
// stream's serialisation is kept either way: only launch latency overlaps.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  unsigned nsm;
  asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
  if (2ull * gridDim.x * gridDim.y * gridDim.z <= nsm) pdl_trigger();
}

// Whether launch_k sets the attribute on the calling host thread; the C-ABI
// entry points scope it from the tank's `pdl` option (off elsewhere).
bool pdl_enabled();
struct PdlScope {
  bool prev;
  explicit PdlScope(bool on);
  ~PdlScope();
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};

// Launch through cudaLaunchKernelEx (grid, block, dynamic shared memory,
// stream), with the programmatic-serialisation attribute when pdl_enabled();
// returns the launch status.  Every kernel started here calls pdl_enter()
// first.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl_enabled()) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T> cudaError_t launch_rowpass(const RowPass<T>& a, cudaStream_t s);
// Derivative passes with one warp per line pair and the transform in
// registers (wt_wfft.cu); warp_deriv_fits says whether a pass qualifies.
template <typename T> bool warp_deriv_fits(const RowPass<T>& a);
template <typename T> cudaError_t launch_deriv_warp(const RowPass<T>& a, cudaStream_t s);

// Independent row passes in one launch (one pair of rows per CTA): the
// passes must not read what another pass of the same launch writes.
constexpr int kMaxPasses = 32;
template <typename T>
struct MultiPass {
  RowPass<T> d[kMaxPasses];
  int start[kMaxPasses + 1];   // first CTA of each pass; start[n] = grid size
  int n = 0;
};
template <typename T> cudaError_t launch_rowpass_multi(const MultiPass<T>& m, cudaStream_t s);

// Metric of several levels in one launch (FP64, plus the FP32 copy when m32).
struct MetricLevel {
  int ncols;
  const double *h, *hx, *hy, *ea, *eax, *eay, *eb, *ebx, *eby;   // y slopes NULL in 2D
  double* meta;
  float* meta32;               // NULL: no FP32 copy
};
constexpr int kMaxMetricLevels = 16;
struct MetricMulti {
  MetricLevel lv[kMaxMetricLevels];
  int n = 0;
  int* flag = nullptr;
};
cudaError_t launch_metric_multi(const MetricMulti& m, cudaStream_t s);

// Column kernels (wt_col.cu).  df != 0: FP64 levels of many columns run the
// double-float kernels of wt_dfcol.cu where they fit.
template <typename T>
cudaError_t launch_op_cols(const LevelView<T>& L, const T* p, const T* Px, const T* Py,
                           T* Gx, T* Gy, T* part, cudaStream_t s, int df = 0);
// Column part of A^T (2D only): Mx = mu_x, part as in opcolsT_body.
template <typename T>
cudaError_t launch_op_cols_T(const LevelView<T>& L, const T* lam, const T* Dlam, T* Mx, T* part,
                             cudaStream_t s);
// tr != 0: the transposed blocks (smoother of A^T).
template <typename T>
cudaError_t launch_smooth_cols(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                               const T* rhoXY, const T* Binv, int nclass, T* x, T omega,
                               int first, int tr, cudaStream_t s);
// out[mo][c] = sum_mi M[mo][mi] in[mi][c] for c < ncols (sigma transfers, filter)
template <typename T>
cudaError_t launch_col_matrix(const T* M, int Mo, int Mi, const T* in, T* out, int ncols,
                              int accumulate, cudaStream_t s, int df = 0);
// Double-float FP64 column kernels (wt_dfcol.cu) for column lengths 5, 9, 13,
// 17 (col_df_fits).
bool col_df_fits(int M1);
cudaError_t launch_op_cols_df(const LevelView<double>& L, const double* p, const double* Px, const double* Py,
                              double* Gx, double* Gy, double* part, cudaStream_t s);
cudaError_t launch_col_matrix_df(const double* M, int Mo, int Mi, const double* in, double* out, int ncols,
                                 int accumulate, cudaStream_t s);
// The block inverses of several levels in one launch: the (column, class)
// tasks of level l are start[l] .. start[l+1]-1, one warp each.
template <typename T>
struct BlockInvMulti {
  int nlev = 0;
  int maxM1 = 0;
  LevelView<T> L[kMaxLevels];
  T* Binv[kMaxLevels];
  int nclass[kMaxLevels];
  T cxx[kMaxLevels], cyy[kMaxLevels];
  long start[kMaxLevels + 1];
};
template <typename T>
cudaError_t launch_block_inverse_multi(const BlockInvMulti<T>& m, int* flag, cudaStream_t s);

// Single-CTA V-cycle over the levels l0..nl-1 (wt_tail.cu): all small levels
// run in one launch with __syncthreads between the phases.
template <typename T>
struct TailLevel {
  LevelView<T> V;
  T *x, *f, *r, *t1, *t2, *t3, *t4, *t5, *t6;
  const T* Binv;
  T *rhoX, *rhoY, *rhoXY;
  const T *Rsig, *Psig;     // to / from the next coarser level
  int nclass;               // smoother block classes and their x / y diagonals
  T cxx, cyy;
};

// FP64 surfaces of one level (bathymetry, both free surfaces, slopes).
struct SurfDesc {
  double *h, *hx, *ea, *eax, *eb, *ebx, *tmp;
};

// Everything the persistent batch kernel needs about one 2D tank (device
// pointers into the tank's own buffers, options as values).
struct BatchTankDesc {
  int nl, Nx, logNx, Nz, M1, ncols;
  long n;
  double L, g;
  const TailLevel<float>* lv32;
  const TailLevel<double>* lv64;
  const SurfDesc* S;
  double *AinvT, *cDx, *cDy;
  double *V64, *Z64;
  float *V32, *Z32;         // FP32 Krylov vectors of the refinement form's inner solve
  double* r64;              // FP64 residual of the refinement form
  float *b32, *e32;
  double *eta, *eta_new, *Keta, *f_eta, *eta_x, *u, *w, *Ku, *Kw, *p, *zero_s;
  double* work[18];
  const double *filt_x, *Fcheb;
  int* flag;
  double* stats;            // [0] solves, [1] Krylov iterations, [2] last relative residual
  double tol, omega, inner_tol;
  int nu1, nu2, restart, max_it, max_ir, filter, linear;
};
// mode: WT_MIXED (FP64 GMRES, FP32 V-cycle), WT_FP64 (FP64 GMRES, FP64
// V-cycle) or WT_REFINE (FP64 refinement around FP32 GMRES + FP32 V-cycle).
cudaError_t launch_batch_step(const BatchTankDesc* descs, const int* order, int ntanks, const double* dt,
                              int nsteps, int smem, int mode, cudaStream_t s);
template <typename T>
struct TailArgs {
  const TailLevel<T>* lv;   // device array, all levels of the hierarchy
  int l0, nl;
  const T* f0;              // right-hand side of level l0
  T* x0;                    // result of level l0
  int f0_nyq;               // f0 may carry x- (y-) Nyquist content
  T omega;
  int nu1, nu2;
  const double* AinvT;      // coarsest inverse, transposed, FP64
  int smem;                 // dynamic shared memory of the launch
};
template <typename T> cudaError_t launch_vcycle_tail(const TailArgs<T>& a, int dim, cudaStream_t s);

// Grid-wide barrier state of the cooperative V-cycle (device memory, zeroed
// at creation): a monotonic arrival counter and the abort flag.
struct GridBar {
  unsigned long long count;   // arrivals since creation (monotonic)
  int abort;
  int pad;
  long long limit;            // SM cycles a CTA waits before giving up (0: kBarrierCycles)
};
// The whole V-cycle from level a.l0 in one cooperative launch (every CTA
// resident); phases separated by a bounded grid barrier.  A barrier that
// waits longer than about a second sets bit 32 of *flag and bar->abort, and
// every CTA returns at its next barrier.
template <typename T>
cudaError_t launch_vcycle_grid(const TailArgs<T>& a, int dim, GridBar* bar, int* flag, cudaStream_t s);
// The levels from a.l0 down and back up in one launch of a single
// thread-block cluster of csize CTAs (2..16), phases separated by the
// cluster's hardware barrier.  cudaErrorInvalidConfiguration if a cluster of
// that size with a.smem bytes per CTA cannot be resident on this device.
template <typename T>
cudaError_t launch_vcycle_cluster(const TailArgs<T>& a, int dim, int csize, cudaStream_t s);

// Mean-depth spectral smoother (wt_spec.cu): x = scale S r (first) or
// x += scale S r, S the exact solve of the flat reference problem mode by mode.
template <typename T>
struct SpecArgs {
  int Nx = 0, Ny = 1, M1 = 0, logNx = 0, logNy = 0;
  const T* r = nullptr;          // residual [M1][Ny][Nx]
  T* x = nullptr;                // iterate [M1][Ny][Nx]
  c2_t<T>* spec = nullptr;       // work: half spectra [M1][Ny][Nx/2+1]
  const T* tab = nullptr;        // inverses of the reference column matrices [ntab][M1][M1]
  const int* sidx = nullptr;     // 3D: table of each mode [Ny][Nx/2+1]; NULL in 2D (table = kx)
  T scale = 1;                   // omega_s / (Nx Ny)
  int first = 0, tr = 0;         // x = (first) or x += ; transposed tables (smoother of A^T)
  const c2_t<T>* tw = nullptr;
  int logNtw = 0;
};
template <typename T> cudaError_t launch_spectral_smooth(const SpecArgs<T>& a, cudaStream_t s);

// Dense coarsest level (wt_coarse.cu), always FP64 arithmetic.
cudaError_t launch_coarse_factor(const LevelView<double>& L, const double* Dx, const double* Dy,
                                 double* LU, int* piv, int* flag, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(int n, const double* LU, const int* piv, int tr, const T* f, T* x,
                                cudaStream_t s);

// Vector / Krylov kernels (wt_krylov.cu).
template <typename T>
cudaError_t launch_dots(const T* w, const T* V, long ldv, int nvec, long n, double* partial,
                        int nblk, int with_norm, cudaStream_t s);
// One-launch forms: the last CTA sums the partials (dots -> out), or sums
// them and performs the Arnoldi / Givens update of column j (update_dots_arnoldi);
// `ticket` is a zero-initialised device counter per call site.
template <typename T>
cudaError_t launch_dots_sum(const T* w, const T* V, long ldv, int nvec, long n, double* partial, int nblk,
                            int with_norm, double* out, unsigned* ticket, cudaStream_t s);
template <typename T>
cudaError_t launch_update_dots_arnoldi(T* w, const T* V, long ldv, int nvec, long n, double* st,
                                       double* partial, int nblk, int j, int m, unsigned* ticket,
                                       cudaStream_t s);
template <typename T>
cudaError_t launch_update_normalize(const T* w, const T* V, long ldv, int nvec, long n,
                                    const double* h, const double* inv_norm, T* vout, float* v32,
                                    cudaStream_t s);
template <typename T>
cudaError_t launch_lincomb(T* x, const T* Z, long ldz, int nvec, long n, const double* y,
                           cudaStream_t s);
template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* in, To* out, long n, const double* scale, int invert,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_axpy_from(double* x, const T* e, long n, const double* scale, cudaStream_t s);
cudaError_t launch_nyquist_coef(const void* r, int is_double, int nrows, int Nx, int logNx,
                                void* rho, cudaStream_t s);
// GMRES small dense part on one thread: see wt_krylov.cu for the state layout.
cudaError_t launch_gmres_init(double* st, const double* partial, int nblk, int m, double bnorm,
                              double tol, cudaStream_t s);
cudaError_t launch_gmres_solve_y(double* st, int k, int m, cudaStream_t s);

// Surface metric (wt_metric.cu).
cudaError_t launch_metric_fill(int ncols, const double* h, const double* hx, const double* hy,
                               const double* ea, const double* eax, const double* eay,
                               const double* eb, const double* ebx, const double* eby,
                               double* meta, int* flag, cudaStream_t s);
template <typename Ti, typename To>
cudaError_t launch_cast(const Ti* in, To* out, long n, cudaStream_t s);

// Runge-Kutta stage kernels (wt_rk.cu).
struct StageArgs {
  int Nx, Ny, M1, ncols;
  double g, alpha, beta, dt;
  int linear;
  const double* sigma;
  const double* D;        // d/dsigma [M1*M1]
  const double* meta;     // finest-level metric (a = new, b = old)
  // viscous term nu Div_b Grad_b q of each velocity component (NULL: none)
  double nu = 0.0;
  const double *lap_u = nullptr, *lap_v = nullptr, *lap_w = nullptr;
};
// Viscous term, two pointwise halves around the derivative passes (geometry
// b of the stage's metric): grad: Gx = qx + sigma_x qs, Gy = qy + sigma_y qs
// (Gy NULL in 2D), Gz = sigma_z qs except Gz = 0 on the surface row (the
// stress-free surface: no vertical viscous flux there); div: lap = dGx +
// sigma_x sGx + dGy + sigma_y sGy + sigma_z sGz (x- / y-derivatives d,
// sigma-derivatives s).
cudaError_t launch_visc_grad(const StageArgs& a, const double* qx, const double* qy, const double* qs,
                             double* Gx, double* Gy, double* Gz, cudaStream_t s);
cudaError_t launch_visc_div(const StageArgs& a, const double* dGx, const double* sGx, const double* dGy,
                            const double* sGy, const double* sGz, double* lap, cudaStream_t s);
// Relaxation zone: q = (1 - wgt) q + wgt q_target for eta (per column) and
// the velocity fields (every sigma row), wgt per column.
cudaError_t launch_relax(int ncols, int M1, const double* wgt, const double* eta_t, const double* u_t,
                         const double* v_t, const double* w_t, double* eta, double* u, double* v, double* w,
                         cudaStream_t s);
cudaError_t launch_stage_forcing(const StageArgs& a, const double* u, const double* v,
                                 const double* w, const double* ux, const double* uy,
                                 const double* vx, const double* vy, const double* wx,
                                 const double* wy, const double* eta_x, const double* eta_y,
                                 const double* f_eta, double* Ku, double* Kv, double* Kw,
                                 double* us, double* vs, double* ws, cudaStream_t s);
cudaError_t launch_stage_eta(int ncols, int M1, int linear, double alpha, double beta, double dt,
                             const double* u, const double* v, const double* w,
                             const double* eta_x, const double* eta_y, double* Keta,
                             const double* eta, double* eta_new, double* f_eta, int* flag,
                             cudaStream_t s);
cudaError_t launch_stage_rhs(const StageArgs& a, const double* us, const double* vs,
                             const double* ws, const double* usx, const double* vsy,
                             const double* Dus, const double* Dvs, const double* Dws, double* rhs,
                             cudaStream_t s);
cudaError_t launch_stage_project(const StageArgs& a, const double* px, const double* py,
                                 const double* Dp, double* Ku, double* Kv, double* Kw, double* u,
                                 double* v, double* w, int* flag, cudaStream_t s);

}  // namespace wt
