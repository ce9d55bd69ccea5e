// Steady nonlinear periodic waves by the Fourier stream-function method
// (Rienecker & Fenton 1981): the initial condition of the paper's nonlinear
// accuracy study (Sec. 5.2) and of its bar case (Sec. 5.5), which the paper
// cites without printing.  Host code (FP64): a Newton solve of 2N + 4
// unknowns, then the fields evaluated at the tank's nodes.
//
// In a frame moving with the wave speed c over a flat bed at y = 0 (still
// depth d), psi(X, y) = -U y + sum_j B_j sinh(j k y) / cosh(j k d) cos(j k X)
// satisfies Laplace's equation and the bed condition exactly; at the N + 1
// surface points X_m = m pi / (N k) (crest to trough) the surface y = d + eta_m
// is the streamline psi = -Q and Bernoulli's condition (u^2 + w^2)/2 + g eta_m
// = R holds; eta has zero mean (trapezoidal rule over the half wavelength,
// exact for the cosine series), eta_0 - eta_N = H, and c = U (no mean
// Eulerian current).  The Jacobian is analytic; the height is raised in
// steps of about 0.005 in steepness from linear theory, each start
// extrapolated from the last two solutions.
#include "wt_host.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace wt {

namespace {

// sinh(a y) / cosh(a d) and cosh(a y) / cosh(a d) without overflow
inline void sh_ch(double a, double y, double d, double& sh, double& ch) {
  const double e1 = std::exp(a * (y - d)), e2 = std::exp(-a * (y + d)), e3 = std::exp(-2.0 * a * d);
  sh = (e1 - e2) / (1.0 + e3);
  ch = (e1 + e2) / (1.0 + e3);
}

// F(z) and its Jacobian J (row-major n x n) for z = [U, Q, R, eta_0..N, B_1..N]
void residual(const std::vector<double>& z, double k, double d, double H, double g, int N,
              std::vector<double>& F, std::vector<double>& J) {
  const int n = 2 * N + 4;
  F.assign(n, 0.0);
  J.assign((size_t)n * n, 0.0);
  const double U = z[0], Q = z[1], R = z[2];
  const double* eta = z.data() + 3;
  const double* B = z.data() + 3 + N + 1;
  for (int m = 0; m <= N; ++m) {
    const double X = m * M_PI / (N * k), y = d + eta[m];
    double psi = -U * y, u = -U, w = 0.0, uy = 0.0, wy = 0.0;
    std::vector<double> dpsi(N), du(N), dw(N);
    for (int j = 1; j <= N; ++j) {
      const double jk = j * k;
      double sh, ch;
      sh_ch(jk, y, d, sh, ch);
      const double cs = std::cos(jk * X), sn = std::sin(jk * X);
      dpsi[j - 1] = sh * cs;
      du[j - 1] = jk * ch * cs;
      dw[j - 1] = jk * sh * sn;
      psi += B[j - 1] * dpsi[j - 1];
      u += B[j - 1] * du[j - 1];
      w += B[j - 1] * dw[j - 1];
      uy += B[j - 1] * jk * jk * sh * cs;
      wy += B[j - 1] * jk * jk * ch * sn;
    }
    // kinematic row m: psi + Q
    const int rk = m;
    F[rk] = psi + Q;
    J[(size_t)rk * n + 0] = -y;
    J[(size_t)rk * n + 1] = 1.0;
    J[(size_t)rk * n + 3 + m] = u;                       // d psi / d y
    for (int j = 0; j < N; ++j) J[(size_t)rk * n + 3 + N + 1 + j] = dpsi[j];
    // dynamic row: (u^2 + w^2)/2 + g eta - R
    const int rd = N + 1 + m;
    F[rd] = 0.5 * (u * u + w * w) + g * eta[m] - R;
    J[(size_t)rd * n + 0] = -u;
    J[(size_t)rd * n + 2] = -1.0;
    J[(size_t)rd * n + 3 + m] = u * uy + w * wy + g;
    for (int j = 0; j < N; ++j) J[(size_t)rd * n + 3 + N + 1 + j] = u * du[j] + w * dw[j];
  }
  // mean level and height
  const int rm = 2 * N + 2, rh = 2 * N + 3;
  double mean = 0.0;
  for (int m = 0; m <= N; ++m) {
    const double wt = (m == 0 || m == N) ? 0.5 : 1.0;
    mean += wt * eta[m] / N;
    J[(size_t)rm * n + 3 + m] = wt / N;
  }
  F[rm] = mean;
  F[rh] = eta[0] - eta[N] - H;
  J[(size_t)rh * n + 3] = 1.0;
  J[(size_t)rh * n + 3 + N] = -1.0;
}

// Solve A x = b in place (Gaussian elimination, partial pivoting); false if singular.
bool gauss_solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (!(std::fabs(A[(size_t)p * n + c]) > 0.0)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)p * n + j], A[(size_t)c * n + j]);
      std::swap(b[p], b[c]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < n; ++j) s -= A[(size_t)r * n + j] * b[j];
    b[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

}  // namespace

bool sf_solve(double k, double d, double H, double g, int N, SfWave& out) {
  const int n = 2 * N + 4;
  const double c0 = std::sqrt(g / k * std::tanh(k * d));
  const double steep = H * k / (2.0 * M_PI);
  const int steps = std::max(1, (int)std::ceil(steep / 0.005));
  std::vector<std::vector<double>> sols;
  std::vector<double> F, J;
  for (int s = 1; s <= steps; ++s) {
    const double Hs = H * s / steps;
    std::vector<double> z(n, 0.0);
    if (sols.empty()) {                          // linear theory
      z[0] = c0;
      z[1] = c0 * d;
      z[2] = 0.5 * c0 * c0;
      for (int m = 0; m <= N; ++m) z[3 + m] = 0.5 * Hs * std::cos(m * M_PI / N);
      z[3 + N + 1] = c0 * Hs / (2.0 * std::tanh(k * d));
    } else if (sols.size() == 1) {
      z = sols.back();
    } else {                                     // linear extrapolation in the height
      const auto& a = sols[sols.size() - 1];
      const auto& b = sols[sols.size() - 2];
      for (int i = 0; i < n; ++i) z[i] = 2.0 * a[i] - b[i];
    }
    bool ok = false;
    for (int it = 0; it < 50; ++it) {
      residual(z, k, d, Hs, g, N, F, J);
      std::vector<double> dz(F);
      for (double& v : dz) v = -v;
      if (!gauss_solve(J, dz, n)) return false;
      double dmax = 0.0, zmax = 1.0;
      for (int i = 0; i < n; ++i) {
        z[i] += dz[i];
        dmax = std::max(dmax, std::fabs(dz[i]));
        zmax = std::max(zmax, std::fabs(z[i]));
      }
      if (!std::isfinite(dmax)) return false;
      if (dmax <= 1e-14 * zmax) {
        ok = true;
        break;
      }
    }
    if (!ok) {                                   // accept if the residual is at rounding level
      residual(z, k, d, Hs, g, N, F, J);
      double fm = 0.0;
      for (double v : F) fm = std::max(fm, std::fabs(v));
      if (!(fm <= 1e-11 * std::max(1.0, g * Hs))) return false;
    }
    sols.push_back(z);
  }
  const auto& z = sols.back();
  out.k = k; out.d = d; out.H = H; out.g = g; out.N = N;
  out.U = z[0]; out.Q = z[1]; out.R = z[2];
  out.c = z[0];
  out.B.assign(z.begin() + 3 + N + 1, z.end());
  // cosine coefficients of the surface from its N + 1 node values
  out.E.assign(N + 1, 0.0);
  for (int j = 0; j <= N; ++j) {
    double a = 0.0;
    for (int m = 0; m <= N; ++m) {
      const double wt = (m == 0 || m == N) ? 0.5 : 1.0;
      a += wt * z[3 + m] * std::cos(j * m * M_PI / N);
    }
    a *= 2.0 / N;
    if (j == 0 || j == N) a *= 0.5;
    out.E[j] = a;
  }
  return true;
}

double sf_eta(const SfWave& W, double x, double t) {
  const double X = x - W.c * t;
  double e = 0.0;
  for (int j = 0; j <= W.N; ++j) e += W.E[j] * std::cos(j * W.k * X);
  return e;
}

void sf_velocity(const SfWave& W, double x, double z, double t, double& u, double& w) {
  const double X = x - W.c * t, y = z + W.d;
  u = 0.0;
  w = 0.0;
  for (int j = 1; j <= W.N; ++j) {
    const double jk = j * W.k;
    double sh, ch;
    sh_ch(jk, y, W.d, sh, ch);
    u += jk * W.B[j - 1] * ch * std::cos(jk * X);
    w += jk * W.B[j - 1] * sh * std::sin(jk * X);
  }
}

}  // namespace wt
