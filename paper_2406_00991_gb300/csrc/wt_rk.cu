// Pointwise kernels of the sigma metric and of the low-storage Runge-Kutta
// stage (paper Sec. 2.1, 3.1-3.3).  All FP64: the metric terms and the
// free-surface / RK accumulation stay in double precision in both solver
// modes.  Derivatives along x / y come from the spectral row passes and the
// sigma-derivatives from the column-matrix kernel; these kernels combine them.
#include "wt_internal.h"

#include <algorithm>

namespace wt {

static inline int blocks_n(long n) { return (int)std::min<long>(std::max<long>(1, (n + 255) / 256), 152 * 8); }

#define GRID_LOOP(i, n) for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

// Metric of Eq. 1_Scoef per column for the geometries a (eta_a) and b (eta_b):
// d = h + eta, d_x = h_x + eta_x;  sigma_x = (h_x - sigma d_x)/d = AX - sigma BX.
__global__ void k_metric_fill(int ncols, const double* __restrict__ h, const double* __restrict__ hx,
                              const double* __restrict__ hy, const double* __restrict__ ea,
                              const double* __restrict__ eax, const double* __restrict__ eay,
                              const double* __restrict__ eb, const double* __restrict__ ebx,
                              const double* __restrict__ eby, double* __restrict__ meta, int* flag) {
  GRID_LOOP(c, ncols) {
    const double HX = hx[c], HY = hy ? hy[c] : 0.0;
    const double da = h[c] + ea[c], db = h[c] + eb[c];
    const double dxa = HX + eax[c], dxb = HX + ebx[c];
    const double dya = HY + (eay ? eay[c] : 0.0), dyb = HY + (eby ? eby[c] : 0.0);
    if (!(da > 0.0) || !(db > 0.0) || !isfinite(da) || !isfinite(db) || !isfinite(dxa) ||
        !isfinite(dxb) || !isfinite(dya) || !isfinite(dyb))
      atomicOr(flag, 4);
    const double ia = 1.0 / da, ib = 1.0 / db;
    meta[M_AXa * (long)ncols + c] = HX * ia;
    meta[M_BXa * (long)ncols + c] = dxa * ia;
    meta[M_AYa * (long)ncols + c] = HY * ia;
    meta[M_BYa * (long)ncols + c] = dya * ia;
    meta[M_Za * (long)ncols + c] = ia;
    meta[M_AXb * (long)ncols + c] = HX * ib;
    meta[M_BXb * (long)ncols + c] = dxb * ib;
    meta[M_AYb * (long)ncols + c] = HY * ib;
    meta[M_BYb * (long)ncols + c] = dyb * ib;
    meta[M_Zb * (long)ncols + c] = ib;
    meta[M_HX * (long)ncols + c] = HX;
    meta[M_HY * (long)ncols + c] = HY;
    meta[M_D_A * (long)ncols + c] = da;
    meta[M_D_B * (long)ncols + c] = db;
  }
}

template <typename Ti, typename To>
__global__ void k_cast(const Ti* __restrict__ in, To* __restrict__ out, long n) {
  GRID_LOOP(i, n) out[i] = (To)in[i];
}

// Kinematic free-surface condition (Eq. kinematicFS) and its 2N register:
// f_eta = -u~ eta_x - v~ eta_y + w~ (linear model: w~); K = alpha K + dt f;
// eta^(k) = eta^(k-1) + beta K.  u~ = surface node (sigma index 0).
__global__ void k_stage_eta(int ncols, int linear, double alpha, double beta, double dt,
                            const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ w, const double* __restrict__ ex,
                            const double* __restrict__ ey, double* __restrict__ Keta,
                            const double* __restrict__ eta, double* __restrict__ eta_new,
                            double* __restrict__ f_eta, int* flag) {
  GRID_LOOP(c, ncols) {
    const double ut = u[c], vt = v ? v[c] : 0.0, wt = w[c];
    const double fe = linear ? wt : (-ut * ex[c] - (v ? vt * ey[c] : 0.0) + wt);
    const double K = alpha * Keta[c] + dt * fe;
    Keta[c] = K;
    const double en = eta[c] + beta * K;
    eta_new[c] = en;
    f_eta[c] = fe;
    if (!isfinite(en)) atomicOr(flag, 8);
  }
}

// Momentum forcing without p_D (Eq. forc1 with the pressure split of Sec. 2):
//   F_q = -(u q_x + v q_y + w_sigma q_sigma) - g (eta_x, eta_y, 0)_q,
//   w_sigma = sigma_t + u sigma_x + v sigma_y + w sigma_z, sigma_t = -sigma f_eta / d,
// then K_q <- alpha K_q + dt F_q and q* = q + beta K_q (q* overwrites the
// sigma-derivative inputs Dq).
__global__ void k_stage_forcing(StageArgs a, const double* __restrict__ u, const double* __restrict__ v,
                                const double* __restrict__ w, const double* __restrict__ ux,
                                const double* __restrict__ uy, const double* __restrict__ vx,
                                const double* __restrict__ vy, const double* __restrict__ wx,
                                const double* __restrict__ wy, const double* __restrict__ ex,
                                const double* __restrict__ ey, const double* __restrict__ f_eta,
                                double* __restrict__ Ku, double* __restrict__ Kv,
                                double* __restrict__ Kw, double* __restrict__ us,
                                double* __restrict__ vs, double* __restrict__ ws) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  GRID_LOOP(e, n) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double uu = u[e], ww = w[e], vv = v ? v[e] : 0.0;
    double Fu = -a.g * ex[c], Fv = v ? -a.g * ey[c] : 0.0, Fw = 0.0;
    if (!a.linear) {
      const double* meta = a.meta;
      const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double Zb = meta[M_Zb * nc + c], db = meta[M_D_B * nc + c];
      const double wsig = -s * f_eta[c] / db + uu * sxb + vv * syb + ww * Zb;
      Fu -= uu * ux[e] + wsig * us[e];
      Fw -= uu * wx[e] + wsig * ws[e];
      if (v) {
        Fu -= vv * uy[e];
        Fw -= vv * wy[e];
        Fv -= uu * vx[e] + vv * vy[e] + wsig * vs[e];
      }
    }
    const double ku = a.alpha * Ku[e] + a.dt * Fu;
    const double kw = a.alpha * Kw[e] + a.dt * Fw;
    Ku[e] = ku;
    Kw[e] = kw;
    us[e] = uu + a.beta * ku;
    ws[e] = ww + a.beta * kw;
    if (v) {
      const double kv = a.alpha * Kv[e] + a.dt * Fv;
      Kv[e] = kv;
      vs[e] = vv + a.beta * kv;
    }
  }
}

// Poisson right-hand side in projection form (Eq. poissonp, bcpd, bcpdneu):
// interior Div_a u* / (beta dt), surface 0, bottom (h_x u* + h_y v* + w*)/(beta dt).
// Inputs: u*_x, v*_y and the sigma-derivatives D u*, D v*, D w* (in Dus, Dvs, Dws).
__global__ void k_stage_rhs(StageArgs a, const double* __restrict__ us, const double* __restrict__ vs,
                            const double* __restrict__ ws, const double* __restrict__ usx,
                            const double* __restrict__ vsy, const double* __restrict__ Dus,
                            const double* __restrict__ Dvs, const double* __restrict__ Dws,
                            double* __restrict__ rhs) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  const double ib = 1.0 / (a.beta * a.dt);
  GRID_LOOP(e, n) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double* meta = a.meta;
    double b;
    if (m == 0) {
      b = 0.0;
    } else if (m == a.M1 - 1) {
      b = (meta[M_HX * nc + c] * us[e] + (vs ? meta[M_HY * nc + c] * vs[e] : 0.0) + ws[e]) * ib;
    } else {
      const double s = a.sigma[m];
      const double sxa = meta[M_AXa * nc + c] - s * meta[M_BXa * nc + c];
      double d = usx[e] + sxa * Dus[e] + meta[M_Za * nc + c] * Dws[e];
      if (vs) {
        const double sya = meta[M_AYa * nc + c] - s * meta[M_BYa * nc + c];
        d += vsy[e] + sya * Dvs[e];
      }
      b = d * ib;
    }
    rhs[e] = b;
  }
}

// Projection (Eq. rkforc1): K_q <- K_q - dt (Grad_b p)_q, q^(k) = q^(k-1) + beta K_q.
__global__ void k_stage_project(StageArgs a, const double* __restrict__ px, const double* __restrict__ py,
                                const double* __restrict__ Dp, double* __restrict__ Ku,
                                double* __restrict__ Kv, double* __restrict__ Kw,
                                double* __restrict__ u, double* __restrict__ v, double* __restrict__ w,
                                int* flag) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  GRID_LOOP(e, n) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double* meta = a.meta;
    const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
    const double Zb = meta[M_Zb * nc + c];
    const double Gx = px[e] + sxb * Dp[e];
    const double Gz = Zb * Dp[e];
    const double ku = Ku[e] - a.dt * Gx, kw = Kw[e] - a.dt * Gz;
    Ku[e] = ku;
    Kw[e] = kw;
    const double un = u[e] + a.beta * ku, wn = w[e] + a.beta * kw;
    u[e] = un;
    w[e] = wn;
    bool bad = !isfinite(un) || !isfinite(wn);
    if (v) {
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double Gy = py[e] + syb * Dp[e];
      const double kv = Kv[e] - a.dt * Gy;
      Kv[e] = kv;
      const double vn = v[e] + a.beta * kv;
      v[e] = vn;
      bad = bad || !isfinite(vn);
    }
    if (bad) atomicOr(flag, 8);
  }
}

cudaError_t launch_metric_fill(int ncols, const double* h, const double* hx, const double* hy,
                               const double* ea, const double* eax, const double* eay,
                               const double* eb, const double* ebx, const double* eby, double* meta,
                               int* flag, cudaStream_t s) {
  k_metric_fill<<<blocks_n(ncols), 256, 0, s>>>(ncols, h, hx, hy, ea, eax, eay, eb, ebx, eby, meta, flag);
  return cudaGetLastError();
}

template <typename Ti, typename To>
cudaError_t launch_cast(const Ti* in, To* out, long n, cudaStream_t s) {
  k_cast<Ti, To><<<blocks_n(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_cast<double, float>(const double*, float*, long, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, long, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, long, cudaStream_t);

cudaError_t launch_stage_eta(int ncols, int M1, int linear, double alpha, double beta, double dt,
                             const double* u, const double* v, const double* w, const double* eta_x,
                             const double* eta_y, double* Keta, const double* eta, double* eta_new,
                             double* f_eta, int* flag, cudaStream_t s) {
  (void)M1;
  k_stage_eta<<<blocks_n(ncols), 256, 0, s>>>(ncols, linear, alpha, beta, dt, u, v, w, eta_x, eta_y,
                                              Keta, eta, eta_new, f_eta, flag);
  return cudaGetLastError();
}

cudaError_t launch_stage_forcing(const StageArgs& a, const double* u, const double* v, const double* w,
                                 const double* ux, const double* uy, const double* vx, const double* vy,
                                 const double* wx, const double* wy, const double* eta_x,
                                 const double* eta_y, const double* f_eta, double* Ku, double* Kv,
                                 double* Kw, double* us, double* vs, double* ws, cudaStream_t s) {
  k_stage_forcing<<<blocks_n((long)a.M1 * a.ncols), 256, 0, s>>>(a, u, v, w, ux, uy, vx, vy, wx, wy,
                                                                  eta_x, eta_y, f_eta, Ku, Kv, Kw, us,
                                                                  vs, ws);
  return cudaGetLastError();
}

cudaError_t launch_stage_rhs(const StageArgs& a, const double* us, const double* vs, const double* ws,
                              const double* usx, const double* vsy, const double* Dus,
                              const double* Dvs, const double* Dws, double* rhs, cudaStream_t s) {
  k_stage_rhs<<<blocks_n((long)a.M1 * a.ncols), 256, 0, s>>>(a, us, vs, ws, usx, vsy, Dus, Dvs, Dws, rhs);
  return cudaGetLastError();
}
cudaError_t launch_stage_project(const StageArgs& a, const double* px, const double* py,
                                  const double* Dp, double* Ku, double* Kv, double* Kw, double* u,
                                  double* v, double* w, int* flag, cudaStream_t s) {
  k_stage_project<<<blocks_n((long)a.M1 * a.ncols), 256, 0, s>>>(a, px, py, Dp, Ku, Kv, Kw, u, v, w, flag);
  return cudaGetLastError();
}
}  // namespace wt
