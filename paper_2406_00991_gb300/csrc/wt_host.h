// Host-side data of a tank (shared by wt_capi.cu and wt_solver.cu).
#pragma once

#include "../../include/wt.h"
#include "wt_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <array>
#include <stdexcept>
#include <string>
#include <memory>
#include <vector>

namespace wt {

struct WtError {
  int code;
  std::string msg;
};

// NVTX range for the lifetime of the object (stage, solve, V-cycle level,
// batch step): visible in a timeline profiler, no cost without one.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define WT_CK(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::wt::WtError{WT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};   \
  } while (0)

// Device allocations released together.
struct Arena {
  std::vector<void*> ptrs;
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() { release(); }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
  template <typename T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw WtError{WT_ENOMEM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed"};
    }
    ptrs.push_back(p);
    WT_CK(cudaMemset(p, 0, n * sizeof(T)));
    return static_cast<T*>(p);
  }
};

template <typename T>
struct Level {
  int Nx = 0, Ny = 0, Nz = 0, M1 = 0, ncols = 0, logNx = 0, logNy = 0;
  long n = 0;
  T *sigma = nullptr, *D = nullptr, *D2 = nullptr, *DSD = nullptr, *meta = nullptr;
  T *x = nullptr, *f = nullptr, *r = nullptr;
  T *t1 = nullptr, *t2 = nullptr, *t3 = nullptr, *t4 = nullptr, *t5 = nullptr, *t6 = nullptr;
  T *Binv = nullptr;
  int nclass = 0;
  T cxx = 0, cyy = 0;
  T *rhoX = nullptr, *rhoY = nullptr, *rhoXY = nullptr;
  T *Rsig = nullptr, *Psig = nullptr;   // to / from the next coarser level
  bool sig_id = false;                   // both are the identity (same sigma nodes)
  // mean-depth spectral smoother: reference column inverses, table index
  // per mode (3D), half-spectrum work array (built when the option asks)
  T* Stab = nullptr;
  int* sidx = nullptr;
  c2_t<T>* spec = nullptr;
  LevelView<T> view(const c2_t<T>* tw, int logNtw, double Ld) const {
    LevelView<T> v;
    v.Nx = Nx; v.Ny = Ny; v.Nz = Nz; v.M1 = M1; v.logNx = logNx; v.logNy = logNy;
    v.ncols = ncols; v.n = n; v.L = (T)Ld;
    v.sigma = sigma; v.D = D; v.D2 = D2; v.DSD = DSD; v.meta = meta;
    v.tw = tw; v.logNtw = logNtw;
    return v;
  }
};

// FP64 surface data of one level: bathymetry and the two free surfaces.
struct SurfLevel {
  double *h = nullptr, *hx = nullptr, *hy = nullptr;
  double *ea = nullptr, *eax = nullptr, *eay = nullptr;
  double *eb = nullptr, *ebx = nullptr, *eby = nullptr;
  double *tmp = nullptr;
};

// Kernel classes of the optional per-launch CUDA-event profiler.
enum KCat { K_ROWPASS = 0, K_OPCOLS, K_SMOOTH, K_COLMAT, K_BLOCKINV, K_COARSE, K_KRYLOV, K_STAGE,
            K_TAIL, K_NCAT };

struct ProfRec {
  int ev0, ev1, cat;
  double bytes, flops;
};

struct Prof {
  unsigned mask = 0;                 // bit k: time kernel class k with events
  std::vector<cudaEvent_t> pool;     // reused between profiling windows
  size_t used = 0;
  std::vector<ProfRec> rec;
  long launches = 0;                 // every kernel launch since creation
  ~Prof() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// One captured FGMRES Arnoldi step (preconditioner, operator, CGS2 and
// Givens kernels for basis index j), replayed with a single graph launch.
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  long kernels = 0;
};

}  // namespace wt

namespace wt {
// Forward values of one stage kept for its adjoint (FP64, fine level).
struct AdjStage {
  double *eta_f = nullptr, *u_f = nullptr, *w_f = nullptr;   // filtered stage input
  double *eta_n = nullptr, *f_eta = nullptr;                 // eta^(k), kinematic f
  double *us = nullptr, *ws = nullptr, *p = nullptr;         // u*, w*, p
};
constexpr int kAdjCols = 22;     // per-column accumulators of the reverse stage
// Buffers of the adjoint step (allocated at the first adjoint call).
struct AdjBufs {
  Arena ar;
  AdjStage st[5];
  double *Le = nullptr, *Lu = nullptr, *Lw = nullptr;        // adjoints of the stage outputs
  double *LKe = nullptr, *LKu = nullptr, *LKw = nullptr;
  double *LKu1 = nullptr, *LKw1 = nullptr, *LGx = nullptr, *q = nullptr, *lp = nullptr;
  double *lrhs = nullptr, *t1 = nullptr, *px = nullptr, *ux = nullptr, *wx = nullptr;
  double *lux = nullptr, *lwx = nullptr, *lut = nullptr, *lwt = nullptr, *lFu = nullptr, *lFw = nullptr;
  double *lh = nullptr;                                      // dJ/dh of this step
  double* cols = nullptr;                                    // kAdjCols x ncols
  double* FchebT = nullptr;                                  // transposed sigma filter
  long ncols = 0;
  int last_its = 0;
  double last_rel = 0.0;
  double* col(int i) { return cols + (long)i * ncols; }
};
// A solved stream-function wave (wt_sfwave.cu): wavenumber k, still depth d,
// height H, gravity g, N Fourier modes, speed c = U, flux Q, Bernoulli R,
// stream-function coefficients B_1..B_N, surface cosine coefficients E_0..E_N.
struct SfWave {
  double k = 0, d = 0, H = 0, g = 0;
  int N = 0;
  double c = 0, U = 0, Q = 0, R = 0;
  std::vector<double> B, E;
};
bool sf_solve(double k, double d, double H, double g, int N, SfWave& out);
double sf_eta(const SfWave& W, double x, double t);
// fixed-frame velocity at x, height z above the still water level, time t
void sf_velocity(const SfWave& W, double x, double z, double t, double& u, double& w);

}  // namespace wt

struct wt_tank {
  wt::Prof prof;
  // graphs[key][j], key = 0: FP64 V-cycle, 1: FP32 V-cycle in FP64 FGMRES,
  // 2: FP32 FGMRES; key + 3: the same for A^T; rebuilt after any option or
  // hierarchy change
  std::vector<wt::IterGraph> graphs[6];
  bool use_graphs = true;
  // > 0 while the solver evaluates a true residual (restart residual of the
  // flexible GMRES, refinement residual): with df64 = 1 the FP64 real-row
  // passes then stay in FP64 arithmetic (see df_level)
  int residual_scope = 0;
  cudaStream_t own_stream = nullptr;
  cudaEvent_t order_ev = nullptr;
  cudaStream_t side = nullptr;                 // stage set-up overlapped with the forcing:
  cudaStream_t side2 = nullptr;                //   block inverses on side, coarsest LU on side2
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
  int Nx = 0, Ny = 0, Nz = 0, M1 = 0, ncols = 0;
  long n = 0;
  double L = 0, g = 9.81, nu = 0;
  wt_options opt{};
  cudaStream_t s = nullptr;
  int device = 0;

  wt::Arena ar;       // sizes fixed at creation
  wt::Arena har;      // level hierarchy (rebuilt when coarsest_max changes)
  wt::Arena spar;     // spectral smoother tables (rebuilt with the hierarchy or the bathymetry)
  double hmin = 1.0;  // reference depth of the spectral smoother: min h of the fine bathymetry
  double hmax = 1.0;  // max h of the fine bathymetry (flat-bottom checks)
  wt::SfWave sf;      // last stream-function wave solved for this tank (cache)
  bool spec_ready = false;

  std::vector<std::array<int, 3>> dims;
  std::vector<wt::Level<double>> L64;
  std::vector<wt::Level<float>> L32;
  std::vector<wt::SurfLevel> S;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  int logNtw = 0;
  wt::TailLevel<double>* tl64 = nullptr;   // device descriptors of every level
  wt::TailLevel<float>* tl32 = nullptr;
  wt::SurfDesc* sd = nullptr;                 // per-level surfaces (device array)
  double *cLU = nullptr, *cDx = nullptr, *cDy = nullptr;
  int* cpiv = nullptr;
  int ncoarse = 0;
  double *filt_x = nullptr, *filt_y = nullptr, *Fcheb = nullptr;
  float* zeros32 = nullptr;

  // Krylov storage (finest level)
  double *V64 = nullptr, *Z64 = nullptr;
  float *V32 = nullptr, *Z32 = nullptr;
  double *st = nullptr, *stN = nullptr, *partial = nullptr;
  int nblk = 1;
  double *x64 = nullptr, *r64 = nullptr, *b64 = nullptr;
  float *b32 = nullptr, *e32 = nullptr;

  // model state and stage work arrays (finest level, FP64)
  double *eta = nullptr, *eta_new = nullptr, *Keta = nullptr, *f_eta = nullptr;
  double *eta_x = nullptr, *eta_y = nullptr, *zero_s = nullptr;
  double *u = nullptr, *v = nullptr, *w = nullptr, *Ku = nullptr, *Kv = nullptr, *Kw = nullptr;
  double *p = nullptr;
  std::vector<double*> work;       // fine-level FP64 temporaries
  std::vector<double*> visc;       // viscous term (nu != 0): laplacians of u, v, w and temporaries
  double* relax_w = nullptr;       // relaxation-zone weights per column (first wt_relax)
  double *io_s1 = nullptr, *io_s2 = nullptr, *io_f1 = nullptr, *io_f2 = nullptr;
  double time = 0;
  bool have_state = false;
  std::unique_ptr<wt::AdjBufs> adj;   // adjoint step buffers (first adjoint call)
  int* dflag = nullptr;
  int* hflag = nullptr;            // pinned
  double* hst = nullptr;           // pinned
  wt::GridBar* gbar = nullptr;     // barrier of the cooperative V-cycle
  unsigned* tickets = nullptr;     // last-CTA counters of the one-launch Krylov reductions
  long solves = 0, iterations = 0;
};

namespace wt {

// Double-float level of the FP64 kernels for the next launches (the
// RowPass.df / column-kernel df argument): 0 FP64 arithmetic; 1 the warp
// passes and sigma-column kernels over many lines / columns in double-float;
// 2 also the CTA-per-row passes.  Option df64 = 1 (default) gives 2, and 1
// inside a true-residual evaluation, so that the attainable residual of an
// FP64 solve stays FP64's; df64 = 2 gives 2 everywhere.
inline int df_level(const wt_tank& t) {
  const int d = t.opt.df64;
  if (d == 1) return t.residual_scope > 0 ? 1 : 2;
  return d;
}

// Marks a true-residual evaluation for df_level while it lives.
struct ResidualScope {
  wt_tank& t;
  explicit ResidualScope(wt_tank& tk) : t(tk) { ++t.residual_scope; }
  ~ResidualScope() { --t.residual_scope; }
  ResidualScope(const ResidualScope&) = delete;
  ResidualScope& operator=(const ResidualScope&) = delete;
};

}  // namespace wt
