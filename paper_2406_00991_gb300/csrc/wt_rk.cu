// Pointwise kernels of the sigma metric and of the low-storage Runge-Kutta
// stage (paper Sec. 2.1, 3.1-3.3).  All FP64: the metric terms and the
// free-surface / RK accumulation stay in double precision in both solver
// modes.  Derivatives along x / y come from the spectral row passes and the
// sigma-derivatives from the column-matrix kernel; these kernels combine them.
#include "wt_dev.cuh"

#include <algorithm>

namespace wt {

static inline int blocks_n(long n) { return (int)std::min<long>(std::max<long>(1, (n + 255) / 256), (long)sm_count() * 8); }

#define GRID_LOOP(i, n) for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

#define TLOOP (long)blockIdx.x * blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x

__global__ void k_metric_fill(int ncols, const double* __restrict__ h, const double* __restrict__ hx,
                              const double* __restrict__ hy, const double* __restrict__ ea,
                              const double* __restrict__ eax, const double* __restrict__ eay,
                              const double* __restrict__ eb, const double* __restrict__ ebx,
                              const double* __restrict__ eby, double* __restrict__ meta, int* flag) {
  pdl_enter();
  metric_body(TLOOP, ncols, h, hx, hy, ea, eax, eay, eb, ebx, eby, meta, flag);
}

// Every level's metric in one launch: blockIdx.y = level.
__global__ void k_metric_multi(const __grid_constant__ MetricMulti m) {
  pdl_enter();
  const MetricLevel& L = m.lv[blockIdx.y];
  const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
  metric_body(t0, ts, L.ncols, L.h, L.hx, L.hy, L.ea, L.eax, L.eay, L.eb, L.ebx, L.eby, L.meta, m.flag);
  if (L.meta32) {
    // each thread converts the columns it wrote
    for (long c = t0; c < L.ncols; c += ts)
      for (int f = 0; f < kMeta; ++f) L.meta32[f * (long)L.ncols + c] = (float)L.meta[f * (long)L.ncols + c];
  }
}

template <typename Ti, typename To>
__global__ void k_cast(const Ti* __restrict__ in, To* __restrict__ out, long n) {
  pdl_enter();
  GRID_LOOP(i, n) out[i] = (To)in[i];
}

__global__ void k_stage_eta(int ncols, int linear, double alpha, double beta, double dt,
                            const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ w, const double* __restrict__ ex,
                            const double* __restrict__ ey, double* __restrict__ Keta,
                            const double* __restrict__ eta, double* __restrict__ eta_new,
                            double* __restrict__ f_eta, int* flag) {
  pdl_enter();
  stage_eta_body(TLOOP, ncols, linear, alpha, beta, dt, u, v, w, ex, ey, Keta, eta, eta_new, f_eta, flag);
}

__global__ void k_stage_forcing(StageArgs a, const double* __restrict__ u, const double* __restrict__ v,
                                const double* __restrict__ w, const double* __restrict__ ux,
                                const double* __restrict__ uy, const double* __restrict__ vx,
                                const double* __restrict__ vy, const double* __restrict__ wx,
                                const double* __restrict__ wy, const double* __restrict__ ex,
                                const double* __restrict__ ey, const double* __restrict__ f_eta,
                                double* __restrict__ Ku, double* __restrict__ Kv,
                                double* __restrict__ Kw, double* __restrict__ us,
                                double* __restrict__ vs, double* __restrict__ ws) {
  pdl_enter();
  stage_forcing_body(TLOOP, a, u, v, w, ux, uy, vx, vy, wx, wy, ex, ey, f_eta, Ku, Kv, Kw, us, vs, ws);
}

__global__ void k_stage_rhs(StageArgs a, const double* __restrict__ us, const double* __restrict__ vs,
                            const double* __restrict__ ws, const double* __restrict__ usx,
                            const double* __restrict__ vsy, const double* __restrict__ Dus,
                            const double* __restrict__ Dvs, const double* __restrict__ Dws,
                            double* __restrict__ rhs) {
  pdl_enter();
  stage_rhs_body(TLOOP, a, us, vs, ws, usx, vsy, Dus, Dvs, Dws, rhs);
}

__global__ void k_stage_project(StageArgs a, const double* __restrict__ px, const double* __restrict__ py,
                                const double* __restrict__ Dp, double* __restrict__ Ku,
                                double* __restrict__ Kv, double* __restrict__ Kw,
                                double* __restrict__ u, double* __restrict__ v, double* __restrict__ w,
                                int* flag) {
  pdl_enter();
  stage_project_body(TLOOP, a, px, py, Dp, Ku, Kv, Kw, u, v, w, flag);
}

__global__ void k_visc_grad(StageArgs a, const double* __restrict__ qx, const double* __restrict__ qy,
                            const double* __restrict__ qs, double* __restrict__ Gx, double* __restrict__ Gy,
                            double* __restrict__ Gz) {
  pdl_enter();
  const long nc = a.ncols;
  GRID_LOOP(e, (long)a.M1 * nc) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double* meta = a.meta;
    const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
    const double q = qs[e];
    Gx[e] = qx[e] + sxb * q;
    if (Gy) Gy[e] = qy[e] + (meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c]) * q;
    Gz[e] = m == 0 ? 0.0 : meta[M_Zb * nc + c] * q;     // stress-free surface: no vertical flux
  }
}

__global__ void k_visc_div(StageArgs a, const double* __restrict__ dGx, const double* __restrict__ sGx,
                           const double* __restrict__ dGy, const double* __restrict__ sGy,
                           const double* __restrict__ sGz, double* __restrict__ lap) {
  pdl_enter();
  const long nc = a.ncols;
  GRID_LOOP(e, (long)a.M1 * nc) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double* meta = a.meta;
    double v = dGx[e] + (meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c]) * sGx[e] + meta[M_Zb * nc + c] * sGz[e];
    if (dGy) v += dGy[e] + (meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c]) * sGy[e];
    lap[e] = v;
  }
}

__global__ void k_relax(int ncols, int M1, const double* __restrict__ wgt, const double* __restrict__ eta_t,
                        const double* __restrict__ u_t, const double* __restrict__ v_t,
                        const double* __restrict__ w_t, double* __restrict__ eta, double* __restrict__ u,
                        double* __restrict__ v, double* __restrict__ w) {
  pdl_enter();
  GRID_LOOP(e, (long)M1 * ncols) {
    const long c = e % ncols;
    const double g = wgt[c];
    if (g == 0.0) continue;
    if (e < ncols && eta_t) eta[c] = (1.0 - g) * eta[c] + g * eta_t[c];
    if (u_t) u[e] = (1.0 - g) * u[e] + g * u_t[e];
    if (v && v_t) v[e] = (1.0 - g) * v[e] + g * v_t[e];
    if (w_t) w[e] = (1.0 - g) * w[e] + g * w_t[e];
  }
}

cudaError_t launch_visc_grad(const StageArgs& a, const double* qx, const double* qy, const double* qs,
                             double* Gx, double* Gy, double* Gz, cudaStream_t s) {
  return launch_k(k_visc_grad, dim3(blocks_n((long)a.M1 * a.ncols)), dim3(256), 0, s, a, qx, qy, qs, Gx, Gy, Gz);
}
cudaError_t launch_visc_div(const StageArgs& a, const double* dGx, const double* sGx, const double* dGy,
                            const double* sGy, const double* sGz, double* lap, cudaStream_t s) {
  return launch_k(k_visc_div, dim3(blocks_n((long)a.M1 * a.ncols)), dim3(256), 0, s, a, dGx, sGx, dGy, sGy, sGz, lap);
}
cudaError_t launch_relax(int ncols, int M1, const double* wgt, const double* eta_t, const double* u_t,
                         const double* v_t, const double* w_t, double* eta, double* u, double* v, double* w,
                         cudaStream_t s) {
  return launch_k(k_relax, dim3(blocks_n((long)M1 * ncols)), dim3(256), 0, s, ncols, M1, wgt, eta_t, u_t, v_t, w_t, eta, u, v, w);
}

cudaError_t launch_metric_fill(int ncols, const double* h, const double* hx, const double* hy,
                               const double* ea, const double* eax, const double* eay,
                               const double* eb, const double* ebx, const double* eby, double* meta,
                               int* flag, cudaStream_t s) {
  return launch_k(k_metric_fill, dim3(blocks_n(ncols)), dim3(256), 0, s, ncols, h, hx, hy, ea, eax, eay, eb, ebx, eby, meta, flag);
}

cudaError_t launch_metric_multi(const MetricMulti& m, cudaStream_t s) {
  if (m.n <= 0) return cudaSuccess;
  if (m.n > kMaxMetricLevels) return cudaErrorInvalidValue;
  int maxc = 1;
  for (int i = 0; i < m.n; ++i) maxc = std::max(maxc, m.lv[i].ncols);
  return launch_k(k_metric_multi, dim3(blocks_n(maxc), m.n), dim3(256), 0, s, m);
}

template <typename Ti, typename To>
cudaError_t launch_cast(const Ti* in, To* out, long n, cudaStream_t s) {
  return launch_k(k_cast<Ti, To>, dim3(blocks_n(n)), dim3(256), 0, s, in, out, n);
}
template cudaError_t launch_cast<double, float>(const double*, float*, long, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, long, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, long, cudaStream_t);

cudaError_t launch_stage_eta(int ncols, int M1, int linear, double alpha, double beta, double dt,
                             const double* u, const double* v, const double* w, const double* eta_x,
                             const double* eta_y, double* Keta, const double* eta, double* eta_new,
                             double* f_eta, int* flag, cudaStream_t s) {
  (void)M1;
  return launch_k(k_stage_eta, dim3(blocks_n(ncols)), dim3(256), 0, s, ncols, linear, alpha, beta, dt, u, v, w, eta_x, eta_y,
                                              Keta, eta, eta_new, f_eta, flag);
}

cudaError_t launch_stage_forcing(const StageArgs& a, const double* u, const double* v, const double* w,
                                 const double* ux, const double* uy, const double* vx, const double* vy,
                                 const double* wx, const double* wy, const double* eta_x,
                                 const double* eta_y, const double* f_eta, double* Ku, double* Kv,
                                 double* Kw, double* us, double* vs, double* ws, cudaStream_t s) {
  return launch_k(k_stage_forcing, dim3(blocks_n((long)a.M1 * a.ncols)), dim3(256), 0, s, a, u, v, w, ux, uy, vx, vy, wx, wy,
                                                                  eta_x, eta_y, f_eta, Ku, Kv, Kw, us,
                                                                  vs, ws);
}

cudaError_t launch_stage_rhs(const StageArgs& a, const double* us, const double* vs, const double* ws,
                              const double* usx, const double* vsy, const double* Dus,
                              const double* Dvs, const double* Dws, double* rhs, cudaStream_t s) {
  return launch_k(k_stage_rhs, dim3(blocks_n((long)a.M1 * a.ncols)), dim3(256), 0, s, a, us, vs, ws, usx, vsy, Dus, Dvs, Dws, rhs);
}
cudaError_t launch_stage_project(const StageArgs& a, const double* px, const double* py,
                                  const double* Dp, double* Ku, double* Kv, double* Kw, double* u,
                                  double* v, double* w, int* flag, cudaStream_t s) {
  return launch_k(k_stage_project, dim3(blocks_n((long)a.M1 * a.ncols)), dim3(256), 0, s, a, px, py, Dp, Ku, Kv, Kw, u, v, w, flag);
}
}  // namespace wt
