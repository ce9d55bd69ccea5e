// Solver autotuner: times the tank's own pressure problem A_{a,b} p = rhs
// under a grid of solver settings and keeps the fastest one that reaches the
// tolerance.  The paper fixes neither the damping, the number of smoothing
// sweeps nor the size of the coarsest level (Sec. 4.1 leaves them open), and
// their best values depend on the tank's resolution and depth profile.
//
// Everything here goes through the public C ABI: wt_set_options and
// wt_poisson_solve on device copies of the inputs, timed on the host clock
// (each solve returns only after its result is on the device).
#include "../../include/wt.h"
#include "wt_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

namespace {

// ---- file of tuned options (JSON lines, one search result per line)
//   {"key": "step 1024x1x24 fp64=0 filter=1 linear=0 tol=1e-10", "mode": 1, "omega": 0.5, ...}
// keyed by the kind of search, the finest grid, whether the tank runs the
// all-FP64 form, the filter, the linearised model and the tolerance.
std::mutex g_cache_mu;
std::string g_cache_path;

struct CacheField {
  const char* name;
  double (*get)(const wt_options&);
  void (*set)(wt_options&, double);
};
#define WT_CF(F) {#F, [](const wt_options& o) { return (double)o.F; }, [](wt_options& o, double v) { o.F = (decltype(o.F))v; }}
const CacheField kCacheFields[] = {WT_CF(mode),     WT_CF(omega),        WT_CF(nu1),      WT_CF(nu2),
                                   WT_CF(coarsest_max), WT_CF(inner_tol), WT_CF(smoother), WT_CF(spectral_min),
                                   WT_CF(omega_s),  WT_CF(cycle),        WT_CF(tail_max), WT_CF(tail_cluster),
                                   WT_CF(vcycle_grid)};
#undef WT_CF

std::string cache_key(const char* kind, wt_tank* t, const wt_options& o) {
  int nl = 0;
  int dims[3 * 16] = {0};
  wt_get_levels(t, &nl, dims);
  char buf[200];
  std::snprintf(buf, sizeof buf, "%s %dx%dx%d fp64=%d filter=%d linear=%d tol=%.3g", kind, dims[0], dims[1],
                dims[2], o.mode == WT_FP64 ? 1 : 0, o.filter, o.linear, o.tol);
  return buf;
}

bool json_number(const std::string& line, const char* name, double* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return false;
  const char* p = line.c_str() + at + pat.size();
  char* end = nullptr;
  *v = std::strtod(p, &end);
  return end != p;
}

std::string line_key(const std::string& line) {
  const std::string pat = "\"key\": \"";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return "";
  const size_t b = at + pat.size(), e = line.find('"', b);
  return e == std::string::npos ? "" : line.substr(b, e - b);
}

// The stored options for key on top of o (true if found).
bool cache_lookup(const std::string& key, wt_options& o, double* best_ms, double* entry_ms) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (g_cache_path.empty()) return false;
  std::ifstream in(g_cache_path);
  std::string line;
  while (std::getline(in, line)) {
    if (line_key(line) != key) continue;
    wt_options r = o;
    for (const auto& f : kCacheFields) {
      double v;
      if (!json_number(line, f.name, &v)) return false;
      f.set(r, v);
    }
    double b = 0.0, e = 0.0;
    json_number(line, "best_ms", &b);
    json_number(line, "entry_ms", &e);
    o = r;
    if (best_ms) *best_ms = b;
    if (entry_ms) *entry_ms = e;
    return true;
  }
  return false;
}

// Replace (or add) the line of key, written to a temporary file and renamed.
void cache_store(const std::string& key, const wt_options& o, double best_ms, double entry_ms) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (g_cache_path.empty()) return;
  std::vector<std::string> keep;
  {
    std::ifstream in(g_cache_path);
    std::string line;
    while (std::getline(in, line))
      if (!line.empty() && line_key(line) != key) keep.push_back(line);
  }
  std::ostringstream os;
  os.precision(17);
  os << "{\"key\": \"" << key << "\"";
  for (const auto& f : kCacheFields) os << ", \"" << f.name << "\": " << f.get(o);
  os << ", \"best_ms\": " << best_ms << ", \"entry_ms\": " << entry_ms << "}";
  keep.push_back(os.str());
  const std::string tmp = g_cache_path + ".tmp";
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return;
    for (const auto& l : keep) out << l << "\n";
    if (!out) return;
  }
  std::rename(tmp.c_str(), g_cache_path.c_str());
}

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Second stage on the winner: the refinement form with inner tolerances
// 1e-4 and 1e-3, the spectral smoothers (on every level, or on the finest
// one to three levels; then their damping 0.8 / 1.2), the full-multigrid cycle instead of
// the V-cycle, then the launch schedule of the V-cycles - the levels below
// tail_max unknowns in one launch (one CTA, or a cluster of 16 CTAs), or (with
// block-Jacobi alone) the whole cycle as one cooperative launch - each kept
// only where it is faster.
// Unknowns of each level of the tank's hierarchy, finest first.
std::vector<long> level_sizes(const wt_tank* t) {
  int nl = 0;
  int dims[3 * 16] = {0};
  std::vector<long> n;
  if (wt_get_levels(t, &nl, dims) != WT_OK) return n;
  for (int l = 0; l < nl; ++l) n.push_back((long)dims[3 * l] * dims[3 * l + 1] * (dims[3 * l + 2] + 1));
  return n;
}

template <typename F>
void refine_schedule(wt_options& bo, double& bms, F&& measure, const std::vector<long>& sizes) {
  if (bo.mode != WT_FP64) {
    // the literal refinement form with looser inner solves: each refinement
    // then costs fewer FP32 iterations, and the FP64 operator (the costly
    // part on a GPU with a low FP64 rate) runs once per refinement only
    const wt_options base = bo;
    const double itols[] = {1e-4, 1e-3};
    for (double it : itols) {
      wt_options o = base;
      o.mode = WT_REFINE;
      o.inner_tol = it;
      const double ms = measure(o, bms);
      if (ms > 0 && ms < bms) {
        bms = ms;
        bo = o;
      }
    }
  }
  {
    // the mean-depth spectral smoother, alone or after block-Jacobi, with
    // one or two sweeps each way, on every level or on the finest one, two
    // or three levels only (block-Jacobi below: spectral_min)
    const wt_options base = bo;
    const int kinds[] = {1, 2};
    const int nus[] = {1, 2};
    std::vector<int> mins = {0};
    for (size_t k = 1; k <= 3 && k + 1 < sizes.size(); ++k)
      mins.push_back((int)std::min<long>(sizes[k] + 1, 1L << 30));
    for (int kind : kinds)
      for (int nu : nus)
        for (int mn : mins) {
          wt_options o = base;
          o.smoother = kind;
          o.nu1 = o.nu2 = nu;
          o.spectral_min = mn;
          o.tail_max = 0;
          o.tail_cluster = 0;
          o.vcycle_grid = 0;
          const double ms = measure(o, bms);
          if (ms > 0 && ms < bms) {
            bms = ms;
            bo = o;
          }
        }
  }
  if (bo.smoother != 0) {
    // the spectral sweep's damping around the undamped exact flat solve
    const wt_options base = bo;
    const double oms[] = {0.8, 1.2};
    for (double om : oms) {
      wt_options o = base;
      o.omega_s = om;
      const double ms = measure(o, bms);
      if (ms > 0 && ms < bms) {
        bms = ms;
        bo = o;
      }
    }
  }
  {
    // the full-multigrid cycle (Algorithm 2) as the preconditioner
    wt_options o = bo;
    o.cycle = 1;
    o.tail_max = 0;
    o.tail_cluster = 0;
    o.vcycle_grid = 0;
    const double ms = measure(o, bms);
    if (ms > 0 && ms < bms) {
      bms = ms;
      bo = o;
    }
  }
  // the levels at or below tail_max unknowns in one launch (block-Jacobi
  // inside it; with the spectral smoother the finer levels keep theirs)
  const wt_options base = bo;
  const int tails[] = {2048, 8192};
  const int clusters[] = {0, 16};
  for (int tm : tails)
    for (int cl : clusters) {
      wt_options o = base;
      o.tail_max = tm;
      o.tail_cluster = cl;
      o.vcycle_grid = 0;
      const double ms = measure(o, bms);
      if (ms > 0 && ms < bms) {
        bms = ms;
        bo = o;
      }
    }
  if (base.smoother != 0) return;          // the cooperative cycle smooths by block-Jacobi only
  wt_options o = base;
  o.vcycle_grid = 1;
  o.tail_max = 0;
  o.tail_cluster = 0;
  const double ms = measure(o, bms);
  if (ms > 0 && ms < bms) {
    bms = ms;
    bo = o;
  }
}

}  // namespace

extern "C" int wt_autotune(wt_tank* t, const double* eta_a, const double* eta_b, const double* rhs, int reps,
                           wt_options* best, double* best_ms, double* entry_ms) {
  if (!t || !eta_a || !eta_b || !rhs) return wt::set_error(WT_EINVAL, "wt_autotune: NULL argument");
  if (reps < 1 || reps > 100) return wt::set_error(WT_EINVAL, "wt_autotune: reps must be in [1, 100]");
  wt_options entry{};
  wt_get_options(t, &entry);
  const std::string key = cache_key("solve", t, entry);
  {
    wt_options o = entry;
    if (cache_lookup(key, o, best_ms, entry_ms)) {
      const int st = wt_set_options(t, &o);
      if (st == WT_OK && best) *best = o;
      return st;
    }
  }
  int nl = 0;
  int dims[3 * 16];
  if (wt_get_levels(t, &nl, dims) != WT_OK) return WT_EINVAL;
  const int Nx = dims[0], Ny = dims[1], Nz = dims[2];        // finest level
  const size_t ncols = (size_t)Nx * Ny, n = ncols * (Nz + 1);
  DevBuf ea, eb, b, p;
  cudaError_t e;
  if ((e = cudaMalloc(&ea.p, sizeof(double) * ncols)) != cudaSuccess ||
      (e = cudaMalloc(&eb.p, sizeof(double) * ncols)) != cudaSuccess ||
      (e = cudaMalloc(&b.p, sizeof(double) * n)) != cudaSuccess ||
      (e = cudaMalloc(&p.p, sizeof(double) * n)) != cudaSuccess) {
    cudaGetLastError();
    return wt::set_error(WT_ENOMEM, "wt_autotune: device buffers");
  }
  if ((e = cudaMemcpy(ea.p, eta_a, sizeof(double) * ncols, cudaMemcpyDefault)) != cudaSuccess ||
      (e = cudaMemcpy(eb.p, eta_b, sizeof(double) * ncols, cudaMemcpyDefault)) != cudaSuccess ||
      (e = cudaMemcpy(b.p, rhs, sizeof(double) * n, cudaMemcpyDefault)) != cudaSuccess)
    return wt::set_error(WT_ECUDA, cudaGetErrorString(e));

  // one candidate: a warm-up solve (captures its graphs), then the median of
  // reps solves from a zero initial guess; < 0 if it does not converge
  auto measure = [&](const wt_options& o, double prune_ms) -> double {
    if (wt_set_options(t, &o) != WT_OK) return -1.0;
    std::vector<double> ms;
    for (int r = 0; r <= reps; ++r) {
      if (cudaMemset(p.p, 0, sizeof(double) * n) != cudaSuccess) return -1.0;
      wt_solve_info info{};
      const double t0 = now_ms();
      const int st = wt_poisson_solve(t, ea.p, eb.p, b.p, p.p, 0.0, &info);
      const double dt = now_ms() - t0;
      if (st != WT_OK) return -1.0;
      if (r == 0) {
        if (prune_ms > 0 && dt > 3.0 * prune_ms) return -1.0;   // far slower than the best so far
        continue;
      }
      ms.push_back(dt);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };

  const double e_ms = measure(entry, 0.0);
  wt_options bo = entry;
  double bms = e_ms > 0 ? e_ms : 1e300;
  std::vector<int> modes;
  if (entry.mode == WT_FP64)
    modes = {WT_FP64};
  else
    modes = {WT_MIXED, WT_REFINE};
  const double omegas[] = {0.3, 0.4, 0.5, 0.6};
  const int nus[][2] = {{1, 1}, {2, 2}, {3, 3}};
  const int coarsest[] = {32, 64, 128};
  for (int mode : modes)
    for (double om : omegas)
      for (const auto& nu : nus)
        for (int cm : coarsest) {
          wt_options o = entry;
          o.mode = mode;
          o.omega = om;
          o.nu1 = nu[0];
          o.nu2 = nu[1];
          o.coarsest_max = cm;
          if (o.mode == entry.mode && o.omega == entry.omega && o.nu1 == entry.nu1 && o.nu2 == entry.nu2 &&
              o.coarsest_max == entry.coarsest_max)
            continue;                                  // measured above
          const double ms = measure(o, bms < 1e300 ? bms : 0.0);
          if (ms > 0 && ms < bms) {
            bms = ms;
            bo = o;
          }
        }
  if (bms < 1e300) refine_schedule(bo, bms, measure, level_sizes(t));
  if (bms >= 1e300) {
    wt_set_options(t, &entry);
    return wt::set_error(WT_ENOCONV, "wt_autotune: no candidate reached the tolerance");
  }
  const int st = wt_set_options(t, &bo);
  if (st != WT_OK) return st;
  cache_store(key, bo, bms, e_ms);
  if (best) *best = bo;
  if (best_ms) *best_ms = bms;
  if (entry_ms) *entry_ms = e_ms;
  return WT_OK;
}

// Step-level variant: the tank's own Runge-Kutta step (current state, dt) is
// the timed unit, so the choice covers every solve of a step and the stage
// work around it.  The state is restored after every trial.
extern "C" int wt_autotune_step(wt_tank* t, double dt, int reps, wt_options* best, double* best_ms,
                                double* entry_ms) {
  if (!t) return wt::set_error(WT_EINVAL, "wt_autotune_step: NULL tank");
  if (reps < 1 || reps > 100) return wt::set_error(WT_EINVAL, "wt_autotune_step: reps must be in [1, 100]");
  if (!(dt > 0)) return wt::set_error(WT_EINVAL, "wt_autotune_step: dt must be positive");
  wt_options entry{};
  wt_get_options(t, &entry);
  const std::string key = cache_key("step", t, entry);
  {
    wt_options o = entry;
    if (cache_lookup(key, o, best_ms, entry_ms)) {
      const int st = wt_set_options(t, &o);
      if (st == WT_OK && best) *best = o;
      return st;
    }
  }
  int nl = 0;
  int dims[3 * 16];
  if (wt_get_levels(t, &nl, dims) != WT_OK) return WT_EINVAL;
  const int Nx = dims[0], Ny = dims[1], Nz = dims[2];
  const size_t ncols = (size_t)Nx * Ny, n = ncols * (Nz + 1);
  DevBuf e0, u0, v0, w0;
  if (cudaMalloc(&e0.p, sizeof(double) * ncols) != cudaSuccess || cudaMalloc(&u0.p, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&v0.p, sizeof(double) * n) != cudaSuccess || cudaMalloc(&w0.p, sizeof(double) * n) != cudaSuccess) {
    cudaGetLastError();
    return wt::set_error(WT_ENOMEM, "wt_autotune_step: device buffers");
  }
  double time0 = 0.0;
  int st = wt_get_state(t, e0.p, u0.p, v0.p, w0.p, &time0);
  if (st != WT_OK) return st;
  auto restore = [&]() { return wt_set_state(t, e0.p, u0.p, v0.p, w0.p, time0); };
  auto measure = [&](const wt_options& o, double prune_ms) -> double {
    if (wt_set_options(t, &o) != WT_OK) return -1.0;
    if (restore() != WT_OK) return -1.0;
    std::vector<double> ms;
    for (int r = 0; r <= reps; ++r) {
      const double t0 = now_ms();
      const int s = wt_step(t, dt, 1);
      const double d = now_ms() - t0;
      if (s != WT_OK) return -1.0;
      if (r == 0) {
        if (prune_ms > 0 && d > 3.0 * prune_ms) return -1.0;
        continue;
      }
      ms.push_back(d);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };
  const double e_ms = measure(entry, 0.0);
  wt_options bo = entry;
  double bms = e_ms > 0 ? e_ms : 1e300;
  const std::vector<int> modes = entry.mode == WT_FP64 ? std::vector<int>{WT_FP64}
                                                       : std::vector<int>{WT_MIXED, WT_REFINE};
  const double omegas[] = {0.3, 0.4, 0.5, 0.6};
  const int nus[][2] = {{1, 1}, {2, 2}, {3, 3}};
  const int coarsest[] = {32, 64, 128};
  for (int mode : modes)
    for (double om : omegas)
      for (const auto& nu : nus)
        for (int cm : coarsest) {
          wt_options o = entry;
          o.mode = mode;
          o.omega = om;
          o.nu1 = nu[0];
          o.nu2 = nu[1];
          o.coarsest_max = cm;
          if (o.mode == entry.mode && o.omega == entry.omega && o.nu1 == entry.nu1 && o.nu2 == entry.nu2 &&
              o.coarsest_max == entry.coarsest_max)
            continue;
          const double ms = measure(o, bms < 1e300 ? bms : 0.0);
          if (ms > 0 && ms < bms) {
            bms = ms;
            bo = o;
          }
        }
  if (bms < 1e300) refine_schedule(bo, bms, measure, level_sizes(t));
  if (bms >= 1e300) {
    wt_set_options(t, &entry);
    restore();
    return wt::set_error(WT_ENOCONV, "wt_autotune_step: no candidate completed a step");
  }
  st = wt_set_options(t, &bo);
  if (st == WT_OK) st = restore();
  if (st != WT_OK) return st;
  cache_store(key, bo, bms, e_ms);
  if (best) *best = bo;
  if (best_ms) *best_ms = bms;
  if (entry_ms) *entry_ms = e_ms;
  return WT_OK;
}

// Batch autotuner: one option set for every tank of the batch, timed on one
// wt_batch_step of the batch itself (the makespan of the persistent launch,
// host clock: the call returns when every tank is done), from the batch's
// current states, which are restored before every trial and on return.
extern "C" int wt_batch_autotune(wt_batch* b, const double* dt, int reps, wt_options* best, double* best_ms,
                                 double* entry_ms) {
  if (!b || !dt) return wt::set_error(WT_EINVAL, "wt_batch_autotune: NULL argument");
  if (reps < 1 || reps > 20) return wt::set_error(WT_EINVAL, "wt_batch_autotune: reps must be in [1, 20]");
  int ntanks = 0, st = wt_batch_size(b, &ntanks);
  if (st != WT_OK) return st;
  struct Saved {
    std::vector<double> eta, u, w;
    double time = 0.0;
  };
  std::vector<Saved> saved(ntanks);
  for (int i = 0; i < ntanks; ++i) {
    int Nx = 0, Nz = 0;
    if ((st = wt_batch_tank_dims(b, i, &Nx, &Nz)) != WT_OK) return st;
    saved[i].eta.resize(Nx);
    saved[i].u.resize((size_t)(Nz + 1) * Nx);
    saved[i].w.resize((size_t)(Nz + 1) * Nx);
    if ((st = wt_batch_get_state(b, i, saved[i].eta.data(), saved[i].u.data(), saved[i].w.data(),
                                 &saved[i].time)) != WT_OK)
      return st;
  }
  wt_options entry{};
  if ((st = wt_batch_get_options(b, &entry)) != WT_OK) return st;
  auto restore = [&]() {
    for (int i = 0; i < ntanks; ++i) {
      const int s = wt_batch_set_state(b, i, saved[i].eta.data(), saved[i].u.data(), saved[i].w.data(),
                                       saved[i].time);
      if (s != WT_OK) return s;
    }
    return (int)WT_OK;
  };
  auto measure = [&](const wt_options& o) -> double {
    if (wt_batch_set_options(b, &o) != WT_OK) return -1.0;
    std::vector<double> ms;
    for (int r = 0; r < reps; ++r) {
      if (restore() != WT_OK) return -1.0;
      const double t0 = now_ms();
      const int s = wt_batch_step(b, dt, 1);
      const double d = now_ms() - t0;
      if (s != WT_OK) return -1.0;
      ms.push_back(d);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };
  const double e_ms = measure(entry);
  wt_options bo = entry;
  double bms = e_ms > 0 ? e_ms : 1e300;
  const double omegas[] = {0.3, 0.4, 0.5, 0.6};
  const int nus[][2] = {{1, 1}, {2, 2}};
  for (double om : omegas)
    for (const auto& nu : nus) {
      wt_options o = entry;
      o.omega = om;
      o.nu1 = nu[0];
      o.nu2 = nu[1];
      if (o.omega == entry.omega && o.nu1 == entry.nu1 && o.nu2 == entry.nu2) continue;
      const double ms = measure(o);
      if (ms > 0 && ms < bms) {
        bms = ms;
        bo = o;
      }
    }
  if (bms < 1e300 && entry.mode != WT_FP64) {
    const wt_options base = bo;
    const double itols[] = {1e-4, 1e-3};
    for (double it : itols) {
      wt_options o = base;
      o.mode = WT_REFINE;
      o.inner_tol = it;
      const double ms = measure(o);
      if (ms > 0 && ms < bms) {
        bms = ms;
        bo = o;
      }
    }
  }
  if (bms >= 1e300) {
    wt_batch_set_options(b, &entry);
    restore();
    return wt::set_error(WT_ENOCONV, "wt_batch_autotune: no candidate completed a step");
  }
  st = wt_batch_set_options(b, &bo);
  if (st == WT_OK) st = restore();
  if (st != WT_OK) return st;
  if (best) *best = bo;
  if (best_ms) *best_ms = bms;
  if (entry_ms) *entry_ms = e_ms;
  return WT_OK;
}

extern "C" int wt_autotune_cache(const char* path) {
  if (path && !*path) return wt::set_error(WT_EINVAL, "wt_autotune_cache: empty path");
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache_path = path ? path : "";
  return WT_OK;
}
