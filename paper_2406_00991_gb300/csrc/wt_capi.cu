// C ABI of libwt (declared in include/wt.h): tank creation (grids, level
// hierarchy, Chebyshev matrices and twiddles built on the host in FP64),
// options, state transfer, the solve / operator test hooks and the
// low-storage Runge-Kutta stage (paper Sec. 3.1-3.3).
#include "wt_host.h"
#include "wt_solver.h"

#include <algorithm>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <utility>

using namespace wt;

namespace {

thread_local std::string g_err;
thread_local int g_code = WT_OK;

int fail(int code, const std::string& msg) {
  g_err = msg;
  g_code = code;
  return code;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ------------------------------------------------------------ host matrices
// CGL nodes xi_m = cos(m pi / Nz); sigma = (xi + 1) / 2 (m = 0: surface).
std::vector<double> cgl_xi(int Nz) {
  std::vector<double> x(Nz + 1);
  for (int m = 0; m <= Nz; ++m) x[m] = std::cos(M_PI * m / Nz);
  return x;
}
// d/dsigma on the CGL nodes: 2 x the textbook CGL matrix on [-1, 1]
// (c_0 = c_Nz = 2; off-diagonal c_i (-1)^(i+j) / (c_j (xi_i - xi_j)); diagonal = -row sum).
std::vector<double> cheb_D(int Nz) {
  const int M1 = Nz + 1;
  auto x = cgl_xi(Nz);
  std::vector<double> D(M1 * M1, 0.0);
  for (int i = 0; i < M1; ++i) {
    double rs = 0.0;
    for (int j = 0; j < M1; ++j) {
      if (i == j) continue;
      const double ci = (i == 0 || i == Nz) ? 2.0 : 1.0;
      const double cj = (j == 0 || j == Nz) ? 2.0 : 1.0;
      const double sgn = ((i + j) & 1) ? -1.0 : 1.0;
      const double v = ci / cj * sgn / (x[i] - x[j]);
      D[i * M1 + j] = 2.0 * v;
      rs += v;
    }
    D[i * M1 + i] = -2.0 * rs;
  }
  return D;
}
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int n, int k, int m) {
  std::vector<double> C((size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < k; ++l)
      for (int j = 0; j < m; ++j) C[(size_t)i * m + j] += A[(size_t)i * k + l] * B[(size_t)l * m + j];
  return C;
}
// nodal -> modal Chebyshev coefficients on the CGL nodes (discrete Chebyshev
// transform): a_k = 2/(Nz c_k) sum_j f_j cos(k j pi / Nz) / c_j.
std::vector<double> cheb_modal(int Nz) {
  const int M1 = Nz + 1;
  std::vector<double> W(M1 * M1);
  for (int k = 0; k <= Nz; ++k)
    for (int j = 0; j <= Nz; ++j) {
      const double ck = (k == 0 || k == Nz) ? 2.0 : 1.0;
      const double cj = (j == 0 || j == Nz) ? 2.0 : 1.0;
      W[k * M1 + j] = 2.0 / (Nz * ck * cj) * std::cos(M_PI * k * j / Nz);
    }
  return W;
}
double chebT(int k, double xi) { return std::cos(k * std::acos(std::max(-1.0, std::min(1.0, xi)))); }
// Chebyshev truncation Nzf -> Nzc evaluated at the coarse nodes (Sec. 4.2).
std::vector<double> cheb_restrict(int Nzf, int Nzc, bool inject) {
  auto Wf = cheb_modal(Nzf);
  auto xc = cgl_xi(Nzc);
  const int Mf = Nzf + 1, Mc = Nzc + 1;
  std::vector<double> R(Mc * Mf, 0.0);
  for (int i = 0; i < Mc; ++i)
    for (int j = 0; j < Mf; ++j) {
      double s = 0.0;
      for (int k = 0; k <= Nzc; ++k) s += chebT(k, xc[i]) * Wf[k * Mf + j];
      R[i * Mf + j] = s;
    }
  if (inject) {
    for (int j = 0; j < Mf; ++j) {
      R[0 * Mf + j] = (j == 0) ? 1.0 : 0.0;
      R[(Mc - 1) * Mf + j] = (j == Mf - 1) ? 1.0 : 0.0;
    }
  }
  return R;
}
// Interpolation of the degree-Nzc polynomial at the fine nodes (Sec. 4.2).
std::vector<double> cheb_prolong(int Nzc, int Nzf) {
  auto Wc = cheb_modal(Nzc);
  auto xf = cgl_xi(Nzf);
  const int Mf = Nzf + 1, Mc = Nzc + 1;
  std::vector<double> P(Mf * Mc, 0.0);
  for (int i = 0; i < Mf; ++i)
    for (int j = 0; j < Mc; ++j) {
      double s = 0.0;
      for (int k = 0; k <= Nzc; ++k) s += chebT(k, xf[i]) * Wc[k * Mc + j];
      P[i * Mc + j] = s;
    }
  return P;
}
// Exponential cut-off F_S(i, Nc, alpha = 36, s = 2) with the damping sign (Sec. 3.6).
double filter_resp(int i, int N, int Nc) {
  if (i <= Nc) return 1.0;
  const double r = double(i - Nc) / double(N + 1 - Nc);
  return std::exp(-36.0 * r * r);
}
// Nodal matrix of the Chebyshev exponential filter (Sec. 3.6): modal
// transform, damping of mode m by F_S(m, Nc = floor(0.9 Nz)), evaluation.
std::vector<double> cheb_filter(int Nz) {
  const int M1 = Nz + 1;
  auto W = cheb_modal(Nz);
  auto x = cgl_xi(Nz);
  const int Nc = (int)std::floor(0.9 * Nz);
  std::vector<double> VF(M1 * M1);
  for (int i = 0; i < M1; ++i)
    for (int k = 0; k < M1; ++k) VF[i * M1 + k] = chebT(k, x[i]) * filter_resp(k, Nz, Nc);
  return matmul(VF, W, M1, M1, M1);
}
// Dense periodic first derivative (Nyquist coefficient zero) and its square.
std::vector<double> fourier_D_and_DD(int N, double L) {
  std::vector<double> D(N * N, 0.0);
  if (N > 1) {
    const double h = 2.0 * M_PI / N;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        if (i == j) continue;
        const int k = i - j;
        const double sgn = (k & 1) ? -1.0 : 1.0;
        D[i * N + j] = 0.5 * sgn / std::tan(k * h / 2.0) * (2.0 * M_PI / L);
      }
  }
  auto DD = matmul(D, D, N, N, N);
  std::vector<double> out(D);
  out.insert(out.end(), DD.begin(), DD.end());
  return out;
}
// Diagonal of the composite second derivative: -(1/N) sum_{n != N/2} kappa_n^2.
double second_diag(int N, double L) {
  if (N <= 1) return 0.0;
  double s = 0.0;
  for (int n = -N / 2 + 1; n < N / 2; ++n) {
    const double k = 2.0 * M_PI * n / L;
    s += k * k;
  }
  return -s / N;
}

// p-multigrid hierarchy (Sec. 4.1, reading in the oracle): halve Nx (and Ny)
// if Nx > Nz, halve Nz if Nz > Nx, both if equal; stop at <= coarsest_max
// unknowns or when Nx < 4 / Nz < 2 would follow.
std::vector<std::array<int, 3>> hierarchy(int Nx, int Ny, int Nz, int coarsest_max) {
  std::vector<std::array<int, 3>> lv{{Nx, Ny, Nz}};
  for (;;) {
    auto [nx, ny, nz] = lv.back();
    if ((long)nx * ny * (nz + 1) <= coarsest_max) break;
    int cx = nx, cy = ny, cz = nz;
    if (nx > nz) { cx = nx / 2; cy = ny > 1 ? ny / 2 : 1; }
    else if (nz > nx) { cz = std::max(2, (nz + 1) / 2); }
    else { cx = nx / 2; cy = ny > 1 ? ny / 2 : 1; cz = std::max(2, (nz + 1) / 2); }
    if (cx < 4 || cz < 2 || (Ny > 1 && cy < 4) || (cx == nx && cy == ny && cz == nz)) break;
    lv.push_back({cx, cy, cz});
  }
  return lv;
}

template <typename T>
T* upload(Arena& ar, const std::vector<double>& h) {
  std::vector<T> tmp(h.begin(), h.end());
  T* d = ar.alloc<T>(h.size());
  WT_CK(cudaMemcpy(d, tmp.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return d;
}

template <typename T>
void alloc_level(Arena& ar, Level<T>& L, int Nx, int Ny, int Nz, double Ldom, bool coarsest) {
  L.Nx = Nx; L.Ny = Ny; L.Nz = Nz; L.M1 = Nz + 1; L.ncols = Nx * Ny; L.n = (long)L.M1 * L.ncols;
  L.logNx = ilog2(Nx); L.logNy = ilog2(Ny);
  auto x = cgl_xi(Nz);
  std::vector<double> sig(L.M1);
  for (int m = 0; m < L.M1; ++m) sig[m] = 0.5 * (x[m] + 1.0);
  auto D = cheb_D(Nz);
  auto D2 = matmul(D, D, L.M1, L.M1, L.M1);
  std::vector<double> SD(D);
  for (int i = 0; i < L.M1; ++i)
    for (int j = 0; j < L.M1; ++j) SD[i * L.M1 + j] *= sig[i];
  auto DSD = matmul(D, SD, L.M1, L.M1, L.M1);
  L.sigma = upload<T>(ar, sig);
  L.D = upload<T>(ar, D);
  L.D2 = upload<T>(ar, D2);
  L.DSD = upload<T>(ar, DSD);
  L.meta = ar.alloc<T>((size_t)kMeta * L.ncols);
  L.x = ar.alloc<T>(L.n); L.f = ar.alloc<T>(L.n); L.r = ar.alloc<T>(L.n);
  L.t1 = ar.alloc<T>(L.n); L.t2 = ar.alloc<T>(L.n); L.t3 = ar.alloc<T>(L.n);
  L.t4 = ar.alloc<T>(L.n); L.t5 = ar.alloc<T>(L.n); L.t6 = ar.alloc<T>(L.n);
  L.rhoX = ar.alloc<T>((size_t)L.M1 * Ny);
  L.rhoY = ar.alloc<T>((size_t)L.M1 * Nx);
  L.rhoXY = ar.alloc<T>(L.M1);
  L.nclass = Ny > 1 ? 4 : 2;
  L.cxx = (T)second_diag(Nx, Ldom);
  L.cyy = (T)second_diag(Ny, Ldom);
  if (!coarsest) L.Binv = ar.alloc<T>((size_t)L.nclass * L.M1 * L.M1 * L.ncols);
}

// In-place inverse of the n x n row-major matrix A (Gauss-Jordan with
// partial pivoting, FP64); false if A is singular.
bool invert_host(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * n + c]) > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)piv * n + j], A[(size_t)c * n + j]);
        std::swap(I[(size_t)piv * n + j], I[(size_t)c * n + j]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      A[(size_t)c * n + j] *= d;
      I[(size_t)c * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

// Tables of the mean-depth spectral smoother on every level above the
// coarsest: for each distinct kappa^2 = (2 pi / L)^2 (n^2 + m^2) (n, m the
// x and y mode numbers, 0 at an axis' Nyquist mode) the inverse of the flat
// reference column matrix of depth dref = min h:
//   rows 1..Nz-1: D D / dref^2 - kappa^2 I,  row 0: e_0,  row Nz: D[Nz, :] / dref.
// 2D: table n for kx = n (the Nyquist column uses table 0).  3D: an index
// per mode (ky, kx), kx <= Nx/2.
void build_spectral(wt_tank& t) {
  t.spar.release();
  t.spec_ready = false;
  const int nl = (int)t.L64.size();
  const double dref = t.hmin;
  const double k0 = 2.0 * M_PI / t.L;
  for (int l = 0; l + 1 < nl; ++l) {
    auto& L64 = t.L64[l];
    auto& L32 = t.L32[l];
    const int Nx = L64.Nx, Ny = L64.Ny, M1 = L64.M1, Nz = L64.Nz;
    const int H = Nx / 2, Nh = H + 1;
    auto D = cheb_D(Nz);
    auto D2 = matmul(D, D, M1, M1, M1);
    auto modeno = [](int k, int N) {            // |mode number|, 0 at Nyquist
      if (N == 1) return 0;
      const int m = k <= N / 2 ? k : N - k;
      return m == N / 2 ? 0 : m;
    };
    std::vector<long> keys;                     // n^2 + m^2 of each table
    std::vector<int> idx;
    if (Ny == 1) {
      for (int n = 0; n < H; ++n) keys.push_back((long)n * n);
    } else {
      std::map<long, int> where;
      idx.resize((size_t)Ny * Nh);
      for (int ky = 0; ky < Ny; ++ky)
        for (int kx = 0; kx < Nh; ++kx) {
          const long mx = modeno(kx, Nx), my = modeno(ky, Ny);
          const long key = mx * mx + my * my;
          auto it = where.find(key);
          if (it == where.end()) {
            it = where.emplace(key, (int)keys.size()).first;
            keys.push_back(key);
          }
          idx[(size_t)ky * Nh + kx] = it->second;
        }
    }
    std::vector<double> tab(keys.size() * (size_t)M1 * M1);
    for (size_t q = 0; q < keys.size(); ++q) {
      const double kap2 = k0 * k0 * (double)keys[q];
      std::vector<double> A((size_t)M1 * M1, 0.0);
      for (int i = 1; i < Nz; ++i)
        for (int j = 0; j < M1; ++j)
          A[(size_t)i * M1 + j] = D2[(size_t)i * M1 + j] / (dref * dref) - (i == j ? kap2 : 0.0);
      A[0] = 1.0;
      for (int j = 0; j < M1; ++j) A[(size_t)Nz * M1 + j] = D[(size_t)Nz * M1 + j] / dref;
      if (!invert_host(A, M1)) throw WtError{WT_EINVAL, "singular reference column matrix"};
      std::copy(A.begin(), A.end(), tab.begin() + q * (size_t)M1 * M1);
    }
    L64.Stab = upload<double>(t.spar, tab);
    L32.Stab = upload<float>(t.spar, tab);
    int* di = nullptr;
    if (Ny > 1) {
      di = t.spar.alloc<int>(idx.size());
      WT_CK(cudaMemcpy(di, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
    }
    L64.sidx = L32.sidx = di;
    L64.spec = t.spar.alloc<double2>((size_t)M1 * Ny * Nh);
    L32.spec = t.spar.alloc<float2>((size_t)M1 * Ny * Nh);
  }
  t.spec_ready = true;
}

// Build the spectral tables if the options use the spectral smoother.
void ensure_spectral(wt_tank& t) {
  if (t.opt.smoother != 0 && !t.spec_ready) build_spectral(t);
}

void build_hierarchy(wt_tank& t) {
  t.spar.release();
  t.spec_ready = false;
  for (auto& L : t.L64) L.Stab = nullptr, L.sidx = nullptr, L.spec = nullptr;
  for (auto& L : t.L32) L.Stab = nullptr, L.sidx = nullptr, L.spec = nullptr;
  t.har.release();
  t.L64.clear();
  t.L32.clear();
  t.S.clear();
  t.dims = hierarchy(t.Nx, t.Ny, t.Nz, t.opt.coarsest_max);
  const int nl = (int)t.dims.size();
  if (nl > kMaxLevels) throw WtError{WT_EINVAL, "too many multigrid levels"};
  t.L64.resize(nl);
  t.L32.resize(nl);
  t.S.resize(nl);
  for (int l = 0; l < nl; ++l) {
    auto [nx, ny, nz] = t.dims[l];
    alloc_level<double>(t.har, t.L64[l], nx, ny, nz, t.L, l == nl - 1);
    alloc_level<float>(t.har, t.L32[l], nx, ny, nz, t.L, l == nl - 1);
    auto& S = t.S[l];
    const size_t nc = (size_t)nx * ny;
    S.h = t.har.alloc<double>(nc); S.hx = t.har.alloc<double>(nc); S.hy = t.har.alloc<double>(nc);
    S.ea = t.har.alloc<double>(nc); S.eax = t.har.alloc<double>(nc); S.eay = t.har.alloc<double>(nc);
    S.eb = t.har.alloc<double>(nc); S.ebx = t.har.alloc<double>(nc); S.eby = t.har.alloc<double>(nc);
    S.tmp = t.har.alloc<double>((size_t)t.Ny * nx);
  }
  const bool inject = t.opt.bc_transfer == 0;
  for (int l = 0; l + 1 < nl; ++l) {
    const int Nzf = t.dims[l][2], Nzc = t.dims[l + 1][2];
    auto R = cheb_restrict(Nzf, Nzc, inject);
    auto P = cheb_prolong(Nzc, Nzf);
    t.L64[l].Rsig = upload<double>(t.har, R);
    t.L64[l].Psig = upload<double>(t.har, P);
    t.L32[l].Rsig = upload<float>(t.har, R);
    t.L32[l].Psig = upload<float>(t.har, P);
    // a step that coarsens in x only keeps the sigma nodes: both transfers
    // are then the identity (checked on the assembled matrices), and the
    // V-cycle skips their column passes
    bool id = Nzf == Nzc;
    for (int i = 0; id && i <= Nzf; ++i)
      for (int k = 0; k <= Nzf; ++k) {
        const double e = (i == k) ? 1.0 : 0.0;
        if (std::fabs(R[i * (Nzf + 1) + k] - e) > 1e-12 || std::fabs(P[i * (Nzf + 1) + k] - e) > 1e-12) {
          id = false;
          break;
        }
      }
    t.L64[l].sig_id = t.L32[l].sig_id = id;
  }
  // level descriptors for the one-launch V-cycle kernels (one CTA, one
  // cluster, the cooperative grid)
  {
    std::vector<TailLevel<double>> d64(nl);
    std::vector<TailLevel<float>> d32(nl);
    auto fill = [&](auto& v, auto& Lv, auto* tw) {
      for (int l = 0; l < nl; ++l) {
        auto& L = Lv[l];
        v[l].V = L.view(tw, t.logNtw, t.L);
        v[l].x = L.x; v[l].f = L.f; v[l].r = L.r;
        v[l].t1 = L.t1; v[l].t2 = L.t2; v[l].t3 = L.t3; v[l].t4 = L.t4; v[l].t5 = L.t5; v[l].t6 = L.t6;
        v[l].Binv = L.Binv;
        v[l].rhoX = L.rhoX; v[l].rhoY = L.rhoY; v[l].rhoXY = L.rhoXY;
        v[l].Rsig = L.Rsig; v[l].Psig = L.Psig;
        v[l].nclass = L.nclass; v[l].cxx = L.cxx; v[l].cyy = L.cyy;
      }
    };
    fill(d64, t.L64, t.tw64);
    fill(d32, t.L32, t.tw32);
    t.tl64 = t.har.alloc<TailLevel<double>>(nl);
    t.tl32 = t.har.alloc<TailLevel<float>>(nl);
    WT_CK(cudaMemcpy(t.tl64, d64.data(), sizeof(TailLevel<double>) * nl, cudaMemcpyHostToDevice));
    WT_CK(cudaMemcpy(t.tl32, d32.data(), sizeof(TailLevel<float>) * nl, cudaMemcpyHostToDevice));
    std::vector<SurfDesc> sd(nl);
    for (int l = 0; l < nl; ++l)
      sd[l] = SurfDesc{t.S[l].h, t.S[l].hx, t.S[l].ea, t.S[l].eax, t.S[l].eb, t.S[l].ebx, t.S[l].tmp};
    t.sd = t.har.alloc<SurfDesc>(nl);
    WT_CK(cudaMemcpy(t.sd, sd.data(), sizeof(SurfDesc) * nl, cudaMemcpyHostToDevice));
  }
  auto [cx, cy, cz] = t.dims.back();
  t.ncoarse = cx * cy * (cz + 1);
  if (t.ncoarse > 128)
    throw WtError{WT_ENOTSUP, "coarsest level has " + std::to_string(t.ncoarse) +
                                  " unknowns; the dense FP64 solve takes at most 128"};
  t.cLU = t.har.alloc<double>((size_t)t.ncoarse * t.ncoarse);
  t.cpiv = t.har.alloc<int>(t.ncoarse);
  t.cDx = upload<double>(t.har, fourier_D_and_DD(cx, t.L));
  t.cDy = upload<double>(t.har, fourier_D_and_DD(cy, t.L));
}

const double* in_dev(wt_tank& t, const double* user, double* staging, size_t count) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, user);
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaSuccess && (at.type == cudaMemoryTypeManaged ||
                           (at.type == cudaMemoryTypeDevice && at.device == t.device)))
    return user;
  if (e == cudaSuccess && at.type == cudaMemoryTypeDevice)
    throw WtError{WT_EINVAL, "an array lives on another GPU than the tank's"};
  WT_CK(cudaMemcpyAsync(staging, user, sizeof(double) * count, cudaMemcpyHostToDevice, t.s));
  return staging;
}
void out_copy(wt_tank& t, double* user, const double* dev, size_t count) {
  WT_CK(cudaMemcpyAsync(user, dev, sizeof(double) * count, cudaMemcpyDefault, t.s));
}

int check_options(const wt_options& o) {
  if (o.mode != WT_FP64 && o.mode != WT_MIXED && o.mode != WT_REFINE)
    return fail(WT_EINVAL, "mode must be WT_FP64, WT_MIXED or WT_REFINE");
  if (!(o.inner_tol > 0) || !(o.inner_tol < 1)) return fail(WT_EINVAL, "inner_tol must be in (0, 1)");
  if (o.max_ir < 1) return fail(WT_EINVAL, "max_ir must be >= 1");
  if (o.vcycle_grid != 0 && o.vcycle_grid != 1) return fail(WT_EINVAL, "vcycle_grid must be 0 or 1");
  if (o.tail_cluster < 0 || o.tail_cluster > 16) return fail(WT_EINVAL, "tail_cluster must be in [0, 16]");
  if (!(o.tol > 0) || !(o.tol < 1)) return fail(WT_EINVAL, "tol must be in (0, 1)");
  if (o.restart < 1 || o.restart > 31) return fail(WT_EINVAL, "restart must be in [1, 31]");
  if (o.nu1 < 0 || o.nu1 > 8 || o.nu2 < 0 || o.nu2 > 8 || o.nu1 + o.nu2 == 0)
    return fail(WT_EINVAL, "nu1, nu2 must be in [0, 8], not both 0");
  if (!(o.omega > 0) || !(o.omega < 2)) return fail(WT_EINVAL, "omega must be in (0, 2)");
  if (o.max_it < 1) return fail(WT_EINVAL, "max_it must be >= 1");
  if (o.coarsest_max < 1 || o.coarsest_max > 128) return fail(WT_EINVAL, "coarsest_max must be in [1, 128]");
  if (o.tail_max < 0) return fail(WT_EINVAL, "tail_max must be >= 0");
  if (o.barrier_cycles < 0) return fail(WT_EINVAL, "barrier_cycles must be >= 0");
  if (o.cycle != 0 && o.cycle != 1) return fail(WT_EINVAL, "cycle must be 0 (V-cycle) or 1 (full multigrid)");
  if (o.smoother < 0 || o.smoother > 2)
    return fail(WT_EINVAL, "smoother must be 0 (block-Jacobi), 1 (spectral) or 2 (both)");
  if (!(o.omega_s > 0) || !(o.omega_s < 2)) return fail(WT_EINVAL, "omega_s must be in (0, 2)");
  if (o.warp_fft != 0 && o.warp_fft != 1) return fail(WT_EINVAL, "warp_fft must be 0 or 1");
  if (o.pdl != 0 && o.pdl != 1) return fail(WT_EINVAL, "pdl must be 0 or 1");
  if (o.df64 < 0 || o.df64 > 2) return fail(WT_EINVAL, "df64 must be 0, 1 or 2");
  if (o.spectral_min < 0) return fail(WT_EINVAL, "spectral_min must be >= 0");
  if ((o.filter != 0 && o.filter != 1) || (o.linear != 0 && o.linear != 1) ||
      (o.bc_transfer != 0 && o.bc_transfer != 1))
    return fail(WT_EINVAL, "filter, linear, bc_transfer are 0 or 1");
  return WT_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const WtError& e) {
    return fail(e.code, e.msg);
  } catch (const std::exception& e) {
    return fail(WT_ENOMEM, e.what());
  }
}

// guarded() with the tank's programmatic-dependent-launch option in force for
// the launches of the call.
template <typename F>
int guarded_t(const wt_tank* t, F&& f) {
  PdlScope pdl(t->opt.pdl != 0);
  return guarded(std::forward<F>(f));
}

// Order the tank's own stream after work already queued on the legacy
// default stream (where callers usually produce their device inputs).
void enter(wt_tank& t) {
  if (t.s != t.own_stream) return;
  WT_CK(cudaEventRecord(t.order_ev, 0));
  WT_CK(cudaStreamWaitEvent(t.s, t.order_ev, 0));
}

int read_flags(wt_tank& t) {
  WT_CK(cudaMemcpyAsync(t.hflag, t.dflag, sizeof(int), cudaMemcpyDeviceToHost, t.s));
  WT_CK(cudaStreamSynchronize(t.s));
  WT_CK(cudaGetLastError());
  const int f = *t.hflag;
  if (f) {
    WT_CK(cudaMemsetAsync(t.dflag, 0, sizeof(int), t.s));
    WT_CK(cudaStreamSynchronize(t.s));
  }
  return f;
}

// Carpenter-Kennedy five-stage fourth-order 2N-storage coefficients.
const double kAlpha[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kBeta[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};

RowPass<double> dpass(wt_tank& t, const double* in, double* out, int nrows, int N, int op) {
  RowPass<double> a;
  a.in = in; a.out = out; a.nrows = nrows; a.Nin = N; a.Nout = N;
  a.logNin = ilog2(N); a.logNout = ilog2(N); a.op = op;
  a.kscale = 2.0 * M_PI / t.L; a.tw = t.tw64; a.logNtw = t.logNtw;
  a.warp = t.opt.warp_fft;
  a.df = df_level(t);
  return a;
}
// d/dx of a field with `planes` sigma levels (planes = 1: a surface)
void ddx(wt_tank& t, const double* in, double* out, int planes) {
  run_rowpass(t, dpass(t, in, out, planes * t.Ny, t.Nx, XOP_DERIV));
}
void ddy(wt_tank& t, const double* in, double* out, int planes) {
  RowPass<double> a = dpass(t, in, out, planes * t.Nx, t.Ny, XOP_DERIV);
  a.ylines = 1;
  a.Nxl = t.Nx;
  run_rowpass(t, a);
}
void dds(wt_tank& t, const double* in, double* out) {
  run_col_matrix<double>(t, t.L64[0].D, t.M1, t.M1, in, out, t.ncols, 0);
}
void filter_field(wt_tank& t, double* q, int planes, bool cheb) {
  RowPass<double> a = dpass(t, q, q, planes * t.Ny, t.Nx, XOP_FILTER);
  a.filt = t.filt_x;
  run_rowpass(t, a);
  if (t.Ny > 1) {
    RowPass<double> b = dpass(t, q, q, planes * t.Nx, t.Ny, XOP_FILTER);
    b.ylines = 1;
    b.Nxl = t.Nx;
    b.filt = t.filt_y;
    run_rowpass(t, b);
  }
  if (cheb) run_col_matrix<double>(t, t.Fcheb, t.M1, t.M1, q, q, t.ncols, 0);
}

int rk_stage(wt_tank& t, int k, double dt, AdjStage* rec = nullptr) {
  static const char* const kStageNames[5] = {"wt stage 1", "wt stage 2", "wt stage 3", "wt stage 4",
                                             "wt stage 5"};
  NvtxRange range(kStageNames[k - 1]);
  enter(t);
  const double a = kAlpha[k - 1], b = kBeta[k - 1];
  const bool y = t.Ny > 1;
  const int M1 = t.M1;
  auto& W = t.work;
  if (t.opt.filter) {
    filter_field(t, t.eta, 1, false);
    filter_field(t, t.u, M1, true);
    if (y) filter_field(t, t.v, M1, true);
    filter_field(t, t.w, M1, true);
  }
  auto keep = [&](double* dst, const double* src, long count) {
    WT_CK(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, t.s));
  };
  if (rec) {
    keep(rec->eta_f, t.eta, t.ncols);
    keep(rec->u_f, t.u, t.n);
    keep(rec->w_f, t.w, t.n);
  }
  // free-surface update (Eq. kinematicFS), independent of p_D
  ddx(t, t.eta, t.eta_x, 1);
  if (y) ddy(t, t.eta, t.eta_y, 1);
  WT_LAUNCH(t, K_STAGE, 8.0 * t.ncols * 9, 8.0 * t.ncols, launch_stage_eta(t.ncols, M1, t.opt.linear, a, b, dt, t.u, y ? t.v : nullptr, t.w, t.eta_x,
                         y ? t.eta_y : t.zero_s, t.Keta, t.eta, t.eta_new, t.f_eta, t.dflag, t.s));
  if (rec) {
    keep(rec->eta_n, t.eta_new, t.ncols);
    keep(rec->f_eta, t.f_eta, t.ncols);
  }
  // geometry a = eta^(k), b = eta^(k-1) (still water for the linear model)
  const int prec = t.opt.mode == WT_FP64 ? WT_FP64 : WT_FP32;
  // the smoother's block inverses and the coarsest inverse depend only on the
  // metric: they run on two side streams, concurrently with each other and
  // with the forcing and the right-hand side here (not while per-launch
  // timing is on)
  const bool overlap = t.side && t.side2 && t.prof.mask == 0;
  setup_geometry(t, t.opt.linear ? t.zero_s : t.eta_new, t.opt.linear ? t.zero_s : t.eta, prec, !overlap,
                 !overlap);
  if (overlap) {
    WT_CK(cudaEventRecord(t.ev_fork, t.s));
    WT_CK(cudaStreamWaitEvent(t.side, t.ev_fork, 0));
    WT_CK(cudaStreamWaitEvent(t.side2, t.ev_fork, 0));
    setup_blocks(t, prec, true, false, t.side);
    setup_blocks(t, prec, false, true, t.side2);
    WT_CK(cudaEventRecord(t.ev_join, t.side));
    WT_CK(cudaEventRecord(t.ev_join2, t.side2));
  }
  StageArgs sa;
  sa.Nx = t.Nx; sa.Ny = t.Ny; sa.M1 = M1; sa.ncols = t.ncols;
  sa.g = t.g; sa.alpha = a; sa.beta = b; sa.dt = dt; sa.linear = t.opt.linear;
  sa.sigma = t.L64[0].sigma; sa.D = t.L64[0].D; sa.meta = t.L64[0].meta;
  double *ux = W[0], *uy = W[1], *vx = W[2], *vy = W[3], *wx = W[4], *wy = W[5];
  double *us = W[6], *vs = W[7], *ws = W[8], *usx = W[9], *vsy = W[10], *Dus = W[11], *Dvs = W[12],
         *Dws = W[13], *rhs = W[14], *px = W[15], *py = W[16], *Dp = W[17];
  // forcing without p_D (Eq. forc1), 2N registers and u* = u + beta (alpha K + dt F)
  ddx(t, t.u, ux, M1);
  ddx(t, t.w, wx, M1);
  if (y) {
    ddx(t, t.v, vx, M1);
    ddy(t, t.u, uy, M1);
    ddy(t, t.v, vy, M1);
    ddy(t, t.w, wy, M1);
  }
  dds(t, t.u, us);
  dds(t, t.w, ws);
  if (y) dds(t, t.v, vs);
  if (t.nu != 0.0) {
    // nu Div_b Grad_b q for q = u, (v,) w with the derivatives just taken
    auto& Vb = t.visc;
    double *Gx = Vb[3], *Gy = Vb[4], *Gz = Vb[5], *dGx = Vb[6], *dGy = Vb[7], *sGx = Vb[8], *sGy = Vb[9],
           *sGz = Vb[10];
    auto lap = [&](const double* qx, const double* qy, const double* qs, double* out) {
      WT_LAUNCH(t, K_STAGE, 8.0 * t.n * (y ? 6 : 4), 6.0 * t.n, launch_visc_grad(sa, qx, y ? qy : nullptr, qs, Gx, y ? Gy : nullptr, Gz, t.s));
      ddx(t, Gx, dGx, M1);
      if (y) ddy(t, Gy, dGy, M1);
      dds(t, Gx, sGx);
      if (y) dds(t, Gy, sGy);
      dds(t, Gz, sGz);
      WT_LAUNCH(t, K_STAGE, 8.0 * t.n * (y ? 6 : 4), 8.0 * t.n, launch_visc_div(sa, dGx, sGx, y ? dGy : nullptr, y ? sGy : nullptr, sGz, out, t.s));
    };
    lap(ux, uy, us, Vb[0]);
    if (y) lap(vx, vy, vs, Vb[1]);
    lap(wx, wy, ws, Vb[2]);
    sa.nu = t.nu;
    sa.lap_u = Vb[0];
    sa.lap_v = y ? Vb[1] : nullptr;
    sa.lap_w = Vb[2];
  }
  WT_LAUNCH(t, K_STAGE, 8.0 * t.n * (y ? 24 : 14), 30.0 * t.n, launch_stage_forcing(sa, t.u, y ? t.v : nullptr, t.w, ux, uy, vx, vy, wx, wy, t.eta_x,
                             y ? t.eta_y : t.zero_s, t.f_eta, t.Ku, t.Kv, t.Kw, us, vs, ws, t.s));
  if (rec) {
    keep(rec->us, us, t.n);
    keep(rec->ws, ws, t.n);
  }
  // right-hand side of the mixed-stage Poisson problem (Eq. poissonp, bcpdneu)
  ddx(t, us, usx, M1);
  if (y) ddy(t, vs, vsy, M1);
  dds(t, us, Dus);
  dds(t, ws, Dws);
  if (y) dds(t, vs, Dvs);
  WT_LAUNCH(t, K_STAGE, 8.0 * t.n * (y ? 9 : 6), 10.0 * t.n, launch_stage_rhs(sa, us, y ? vs : nullptr, ws, usx, vsy, Dus, Dvs, Dws, rhs, t.s));
  if (overlap) {
    WT_CK(cudaStreamWaitEvent(t.s, t.ev_join, 0));
    WT_CK(cudaStreamWaitEvent(t.s, t.ev_join2, 0));
  }
  // solve with the previous stage's p_D as the initial guess
  wt_solve_info info{};
  int st = poisson_solve_device(t, rhs, t.p, t.opt.tol, &info);
  if (st != WT_OK && st != WT_ENOCONV) return fail(st, "pressure solve failed (depth <= 0 or non-finite)");
  if (rec) keep(rec->p, t.p, t.n);
  // projection (Eq. rkforc1)
  ddx(t, t.p, px, M1);
  if (y) ddy(t, t.p, py, M1);
  dds(t, t.p, Dp);
  WT_LAUNCH(t, K_STAGE, 8.0 * t.n * (y ? 12 : 9), 16.0 * t.n, launch_stage_project(sa, px, py, Dp, t.Ku, t.Kv, t.Kw, t.u, y ? t.v : nullptr, t.w, t.dflag, t.s));
  if (t.nu != 0.0) {
    // no-slip bed (Sec. 5.4): the velocity and its stage registers vanish on
    // the bottom nodes
    const size_t off = (size_t)(M1 - 1) * t.ncols, bytes = sizeof(double) * t.ncols;
    double* rows[] = {t.u, t.w, t.Ku, t.Kw, y ? t.v : nullptr, y ? t.Kv : nullptr};
    for (double* q : rows)
      if (q) WT_CK(cudaMemsetAsync(q + off, 0, bytes, t.s));
  }
  std::swap(t.eta, t.eta_new);
  if (k == 5) t.time += dt;
  const int fl = read_flags(t);
  if (fl) return fail(WT_EBREAK, "water depth d <= 0 or non-finite state after stage " + std::to_string(k));
  if (st == WT_ENOCONV) return fail(WT_ENOCONV, "pressure solve did not reach its tolerance");
  return WT_OK;
}

// Buffers of the adjoint step, allocated at its first use.
void alloc_adj(wt_tank& t) {
  if (t.adj) return;
  auto B = std::make_unique<AdjBufs>();
  const long n = t.n, nc = t.ncols;
  const int M1 = t.M1;
  auto& A = B->ar;
  B->ncols = nc;
  for (auto& S : B->st) {
    S.eta_f = A.alloc<double>(nc);
    S.u_f = A.alloc<double>(n);
    S.w_f = A.alloc<double>(n);
    S.eta_n = A.alloc<double>(nc);
    S.f_eta = A.alloc<double>(nc);
    S.us = A.alloc<double>(n);
    S.ws = A.alloc<double>(n);
    S.p = A.alloc<double>(n);
  }
  B->Le = A.alloc<double>(nc);
  B->LKe = A.alloc<double>(nc);
  B->lh = A.alloc<double>(nc);
  double** fields[] = {&B->Lu, &B->Lw, &B->LKu, &B->LKw, &B->LKu1, &B->LKw1, &B->LGx, &B->q, &B->lp,
                       &B->lrhs, &B->t1, &B->px, &B->ux, &B->wx, &B->lux, &B->lwx, &B->lut, &B->lwt,
                       &B->lFu, &B->lFw};
  for (double** f : fields) *f = A.alloc<double>(n);
  B->cols = A.alloc<double>((size_t)kAdjCols * nc);
  std::vector<double> F(M1 * M1), FT(M1 * M1);
  WT_CK(cudaMemcpy(F.data(), t.Fcheb, sizeof(double) * M1 * M1, cudaMemcpyDeviceToHost));
  for (int i = 0; i < M1; ++i)
    for (int j = 0; j < M1; ++j) FT[i * M1 + j] = F[j * M1 + i];
  B->FchebT = upload<double>(A, FT);
  t.adj = std::move(B);
}

}  // namespace

int wt::set_error(int code, const char* msg) { return fail(code, msg); }

// ====================================================================== C ABI
extern "C" {

int wt_default_options(wt_options* o) {
  if (!o) return fail(WT_EINVAL, "options pointer is NULL");
  o->mode = WT_MIXED;
  o->tol = 1e-10;
  o->restart = 30;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.4;
  o->max_it = 200;
  o->filter = 0;
  o->linear = 0;
  o->coarsest_max = 64;
  o->bc_transfer = 0;
  o->tail_max = 0;
  o->inner_tol = 1e-5;
  o->max_ir = 30;
  o->vcycle_grid = 0;
  o->tail_cluster = 0;
  o->barrier_cycles = 0;
  o->cycle = 0;
  o->smoother = 0;
  o->omega_s = 1.0;
  o->warp_fft = 1;
  o->pdl = 1;
  o->df64 = 1;
  o->spectral_min = 0;
  return WT_OK;
}

int wt_create(int Nx, int Ny, int Nz, double L, double g, double nu, const double* bathymetry,
              wt_tank** out) {
  if (!out) return fail(WT_EINVAL, "out pointer is NULL");
  *out = nullptr;
  if (!pow2(Nx) || Nx < 4 || Nx > 4096) return fail(WT_EINVAL, "Nx must be a power of two in [4, 4096]");
  if (!(Ny == 1 || (pow2(Ny) && Ny >= 4 && Ny <= 1024)))
    return fail(WT_EINVAL, "Ny must be 1 or a power of two in [4, 1024]");
  if (Nz < 2 || Nz > 32) return fail(WT_EINVAL, "Nz must be in [2, 32]");
  if (!(L > 0) || !std::isfinite(L)) return fail(WT_EINVAL, "L must be positive");
  if (!(g > 0) || !std::isfinite(g)) return fail(WT_EINVAL, "g must be positive");
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(WT_EINVAL, "nu must be >= 0 and finite");
  if (!bathymetry) return fail(WT_EINVAL, "bathymetry pointer is NULL");
  return guarded([&]() -> int {
    std::unique_ptr<wt_tank> t(new wt_tank());
    WT_CK(cudaGetDevice(&t->device));
    // a stream of its own (graph capture needs a non-legacy stream); every call
    // first orders itself after the work already queued on the legacy stream
    WT_CK(cudaStreamCreateWithFlags(&t->own_stream, cudaStreamNonBlocking));
    WT_CK(cudaEventCreateWithFlags(&t->order_ev, cudaEventDisableTiming));
    WT_CK(cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking));
    WT_CK(cudaStreamCreateWithFlags(&t->side2, cudaStreamNonBlocking));
    WT_CK(cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming));
    WT_CK(cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming));
    WT_CK(cudaEventCreateWithFlags(&t->ev_join2, cudaEventDisableTiming));
    t->s = t->own_stream;
    t->Nx = Nx; t->Ny = Ny; t->Nz = Nz; t->M1 = Nz + 1; t->ncols = Nx * Ny; t->n = (long)t->M1 * t->ncols;
    t->L = L; t->g = g; t->nu = nu;
    wt_default_options(&t->opt);
    auto& ar = t->ar;
    const long n = t->n;
    const int nc = t->ncols;
    // twiddles exp(-2 pi i j / Ntw), host FP64
    const int Ntw = std::max(Nx, Ny);
    t->logNtw = ilog2(Ntw);
    {
      std::vector<double2> tw(Ntw / 2);
      std::vector<float2> tf(Ntw / 2);
      for (int j = 0; j < Ntw / 2; ++j) {
        const double ang = 2.0 * M_PI * j / Ntw;
        tw[j] = make_double2(std::cos(ang), -std::sin(ang));
        tf[j] = make_float2((float)tw[j].x, (float)tw[j].y);
      }
      t->tw64 = ar.alloc<double2>(Ntw / 2);
      t->tw32 = ar.alloc<float2>(Ntw / 2);
      WT_CK(cudaMemcpy(t->tw64, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice));
      WT_CK(cudaMemcpy(t->tw32, tf.data(), sizeof(float2) * tf.size(), cudaMemcpyHostToDevice));
    }
    {
      std::vector<double> fx(Nx / 2 + 1), fy(std::max(1, Ny / 2 + 1), 1.0);
      for (int i = 0; i <= Nx / 2; ++i) fx[i] = filter_resp(i, Nx / 2, Nx / 4);
      if (Ny > 1)
        for (int i = 0; i <= Ny / 2; ++i) fy[i] = filter_resp(i, Ny / 2, Ny / 4);
      t->filt_x = upload<double>(ar, fx);
      t->filt_y = upload<double>(ar, fy);
      t->Fcheb = upload<double>(ar, cheb_filter(Nz));
    }
    // Krylov storage for restart <= 31, state and stage arrays
    t->V64 = ar.alloc<double>((size_t)32 * n);
    t->Z64 = ar.alloc<double>((size_t)31 * n);
    t->V32 = ar.alloc<float>((size_t)32 * n);
    t->Z32 = ar.alloc<float>((size_t)31 * n);
    t->nblk = (int)std::min<long>(2L * sm_count(), std::max<long>(1, (n + 511) / 512));
    t->partial = ar.alloc<double>((size_t)t->nblk * 40);
    t->st = ar.alloc<double>(4608);
    t->stN = ar.alloc<double>(4608);
    t->gbar = ar.alloc<GridBar>(1);
    t->tickets = ar.alloc<unsigned>(4);
    t->x64 = ar.alloc<double>(n); t->r64 = ar.alloc<double>(n); t->b64 = ar.alloc<double>(n);
    t->b32 = ar.alloc<float>(n); t->e32 = ar.alloc<float>(n);
    t->eta = ar.alloc<double>(nc); t->eta_new = ar.alloc<double>(nc); t->Keta = ar.alloc<double>(nc);
    t->f_eta = ar.alloc<double>(nc); t->eta_x = ar.alloc<double>(nc); t->eta_y = ar.alloc<double>(nc);
    t->zero_s = ar.alloc<double>(nc);
    t->u = ar.alloc<double>(n); t->v = ar.alloc<double>(n); t->w = ar.alloc<double>(n);
    t->Ku = ar.alloc<double>(n); t->Kv = ar.alloc<double>(n); t->Kw = ar.alloc<double>(n);
    t->p = ar.alloc<double>(n);
    for (int i = 0; i < 18; ++i) t->work.push_back(ar.alloc<double>(n));
    if (nu != 0.0)                     // viscous term: three Laplacians and eight temporaries
      for (int i = 0; i < 11; ++i) t->visc.push_back(ar.alloc<double>(n));
    t->io_s1 = ar.alloc<double>(nc); t->io_s2 = ar.alloc<double>(nc);
    t->io_f1 = ar.alloc<double>(n); t->io_f2 = ar.alloc<double>(n);
    t->dflag = ar.alloc<int>(4);
    WT_CK(cudaMallocHost(&t->hflag, sizeof(int) * 4));
    WT_CK(cudaMallocHost(&t->hst, sizeof(double) * 16));
    build_hierarchy(*t);
    // bathymetry
    const double* hd = in_dev(*t, bathymetry, t->io_s1, nc);
    std::vector<double> hh(nc);
    WT_CK(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * nc, cudaMemcpyDefault, t->s));
    WT_CK(cudaStreamSynchronize(t->s));
    for (double v : hh)
      if (!(v > 0) || !std::isfinite(v)) return fail(WT_EINVAL, "bathymetry must be positive and finite");
    t->hmin = *std::min_element(hh.begin(), hh.end());
    t->hmax = *std::max_element(hh.begin(), hh.end());
    WT_CK(cudaMemcpyAsync(t->io_s2, hh.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, t->s));
    setup_bathymetry(*t, t->io_s2);
    WT_CK(cudaStreamSynchronize(t->s));
    WT_CK(cudaGetLastError());
    *out = t.release();
    return WT_OK;
  });
}

int wt_set_options(wt_tank* t, const wt_options* o) {
  if (!t || !o) return fail(WT_EINVAL, "NULL argument");
  int st = check_options(*o);
  if (st != WT_OK) return st;
  return guarded([&]() -> int {
    const bool rebuild = o->coarsest_max != t->opt.coarsest_max || o->bc_transfer != t->opt.bc_transfer;
    WT_CK(cudaStreamSynchronize(t->s));
    destroy_graphs(*t);
    t->opt = *o;
    write_barrier_limit(*t);
    if (rebuild) {
      WT_CK(cudaStreamSynchronize(t->s));
      // keep the fine-level bathymetry across the rebuild
      std::vector<double> hh(t->ncols);
      WT_CK(cudaMemcpy(hh.data(), t->S[0].h, sizeof(double) * t->ncols, cudaMemcpyDeviceToHost));
      build_hierarchy(*t);
      WT_CK(cudaMemcpy(t->io_s2, hh.data(), sizeof(double) * t->ncols, cudaMemcpyHostToDevice));
      setup_bathymetry(*t, t->io_s2);
      WT_CK(cudaStreamSynchronize(t->s));
    }
    ensure_spectral(*t);
    return WT_OK;
  });
}

int wt_get_options(const wt_tank* t, wt_options* o) {
  if (!t || !o) return fail(WT_EINVAL, "NULL argument");
  *o = t->opt;
  return WT_OK;
}

int wt_set_stream(wt_tank* t, void* stream) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  return guarded([&]() -> int {
    WT_CK(cudaStreamSynchronize(t->s));
    t->s = stream ? static_cast<cudaStream_t>(stream) : t->own_stream;
    return WT_OK;
  });
}

int wt_get_grid(const wt_tank* t, double* x, double* y, double* sigma) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (x)
    for (int j = 0; j < t->Nx; ++j) x[j] = j * t->L / t->Nx;
  if (y)
    for (int j = 0; j < t->Ny; ++j) y[j] = t->Ny > 1 ? j * t->L / t->Ny : 0.0;
  if (sigma) {
    auto xi = cgl_xi(t->Nz);
    for (int m = 0; m <= t->Nz; ++m) sigma[m] = 0.5 * (xi[m] + 1.0);
  }
  return WT_OK;
}

int wt_get_levels(const wt_tank* t, int* nlevels, int* dims) {
  if (!t || !nlevels) return fail(WT_EINVAL, "NULL argument");
  *nlevels = (int)t->dims.size();
  if (dims)
    for (size_t l = 0; l < t->dims.size(); ++l)
      for (int k = 0; k < 3; ++k) dims[3 * l + k] = t->dims[l][k];
  return WT_OK;
}

int wt_set_state(wt_tank* t, const double* eta, const double* u, const double* v, const double* w,
                 double time) {
  if (!t || !eta || !u || !w || (t->Ny > 1 && !v)) return fail(WT_EINVAL, "NULL state array");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const int nc = t->ncols;
    const double* e = in_dev(*t, eta, t->io_s1, nc);
    WT_CK(cudaMemcpyAsync(t->eta, e, sizeof(double) * nc, cudaMemcpyDeviceToDevice, t->s));
    const double* uu = in_dev(*t, u, t->io_f1, n);
    WT_CK(cudaMemcpyAsync(t->u, uu, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    const double* ww = in_dev(*t, w, t->io_f2, n);
    WT_CK(cudaMemcpyAsync(t->w, ww, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    if (t->Ny > 1) {
      const double* vv = in_dev(*t, v, t->io_f1, n);
      WT_CK(cudaMemcpyAsync(t->v, vv, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    } else {
      WT_CK(cudaMemsetAsync(t->v, 0, sizeof(double) * n, t->s));
    }
    WT_CK(cudaMemsetAsync(t->Keta, 0, sizeof(double) * nc, t->s));
    WT_CK(cudaMemsetAsync(t->Ku, 0, sizeof(double) * n, t->s));
    WT_CK(cudaMemsetAsync(t->Kv, 0, sizeof(double) * n, t->s));
    WT_CK(cudaMemsetAsync(t->Kw, 0, sizeof(double) * n, t->s));
    WT_CK(cudaMemsetAsync(t->p, 0, sizeof(double) * n, t->s));
    WT_CK(cudaStreamSynchronize(t->s));
    t->time = time;
    t->have_state = true;
    t->solves = 0;
    t->iterations = 0;
    return WT_OK;
  });
}

int wt_get_state(const wt_tank* tc, double* eta, double* u, double* v, double* w, double* time) {
  if (!tc) return fail(WT_EINVAL, "NULL tank");
  wt_tank* t = const_cast<wt_tank*>(tc);
  return guarded([&]() -> int {
    enter(*t);
    if (eta) out_copy(*t, eta, t->eta, t->ncols);
    if (u) out_copy(*t, u, t->u, t->n);
    if (v) out_copy(*t, v, t->v, t->n);
    if (w) out_copy(*t, w, t->w, t->n);
    WT_CK(cudaStreamSynchronize(t->s));
    if (time) *time = t->time;
    return WT_OK;
  });
}

int wt_get_pressure(const wt_tank* tc, double* p) {
  if (!tc || !p) return fail(WT_EINVAL, "NULL argument");
  wt_tank* t = const_cast<wt_tank*>(tc);
  return guarded([&]() -> int {
    enter(*t);
    out_copy(*t, p, t->p, t->n);
    WT_CK(cudaStreamSynchronize(t->s));
    return WT_OK;
  });
}

int wt_apply_operator(wt_tank* t, const double* eta_a, const double* eta_b, const double* p, double* Ap,
                      int precision) {
  if (!t || !eta_a || !eta_b || !p || !Ap) return fail(WT_EINVAL, "NULL argument");
  if (precision != WT_FP64 && precision != WT_FP32) return fail(WT_EINVAL, "precision must be WT_FP64 or WT_FP32");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    setup_geometry(*t, ea, eb, precision, false, false);
    const double* pd = in_dev(*t, p, t->io_f1, n);
    if (precision == WT_FP64) {
      apply_op<double>(*t, 0, pd, t->io_f2, nullptr, false);
    } else {
      auto& L = t->L32[0];
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<double, float>(pd, L.x, n, nullptr, 0, t->s)));
      apply_op<float>(*t, 0, L.x, L.f, nullptr, false);
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<float, double>(L.f, t->io_f2, n, nullptr, 0, t->s)));
    }
    out_copy(*t, Ap, t->io_f2, n);
    const int fl = read_flags(*t);
    if (fl) return fail(WT_EBREAK, "water depth d <= 0 or non-finite surface");
    return WT_OK;
  });
}

int wt_time_kernel(wt_tank* t, const double* eta_a, const double* eta_b, int what, int precision, int reps,
                   double* ms_per_call, long* launches_per_call) {
  if (!t || !eta_a || !eta_b || !ms_per_call) return fail(WT_EINVAL, "NULL argument");
  if (precision != WT_FP64 && precision != WT_FP32) return fail(WT_EINVAL, "precision must be WT_FP64 or WT_FP32");
  if (what != WT_TIME_OPERATOR && what != WT_TIME_VCYCLE) return fail(WT_EINVAL, "unknown unit to time");
  if (reps < 1 || reps > 10000) return fail(WT_EINVAL, "reps must be in [1, 10000]");
  if (t->prof.mask != 0) return fail(WT_EINVAL, "per-launch timing (wt_profile) is on");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    setup_geometry(*t, ea, eb, precision, what == WT_TIME_VCYCLE, what == WT_TIME_VCYCLE);
    // a smooth non-zero input (the timing does not depend on its values)
    std::vector<double> hx(n);
    for (long i = 0; i < n; ++i) hx[i] = std::sin(0.001 * (double)i) + 0.5;
    WT_CK(cudaMemcpyAsync(t->b64, hx.data(), sizeof(double) * n, cudaMemcpyHostToDevice, t->s));
    WT_CK((launch_convert<double, float>(t->b64, t->b32, n, nullptr, 0, t->s)));
    auto unit = [&]() {
      if (what == WT_TIME_OPERATOR) {
        if (precision == WT_FP64) apply_op<double>(*t, 0, t->b64, t->x64, nullptr, false);
        else apply_op<float>(*t, 0, t->b32, t->e32, nullptr, false);
      } else {
        if (precision == WT_FP64) mg_cycle<double>(*t, t->b64, t->x64);
        else mg_cycle<float>(*t, t->b32, t->e32);
      }
    };
    unit();                                   // warm-up (and any one-time set-up)
    WT_CK(cudaStreamSynchronize(t->s));
    const long l0 = t->prof.launches;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    WT_CK(cudaStreamBeginCapture(t->s, cudaStreamCaptureModeThreadLocal));
    try {
      for (int r = 0; r < reps; ++r) unit();
    } catch (...) {
      cudaStreamEndCapture(t->s, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    WT_CK(cudaStreamEndCapture(t->s, &graph));
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    WT_CK(ei);
    const long per = (t->prof.launches - l0) / reps;
    t->prof.launches = l0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, t->s);          // warm replay
    if (e == cudaSuccess) e = cudaEventRecord(e0, t->s);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, t->s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, t->s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    WT_CK(e);
    t->prof.launches += 2 * per * reps;
    *ms_per_call = (double)ms / reps;
    if (launches_per_call) *launches_per_call = per;
    const int fl = read_flags(*t);
    if (fl) return fail(WT_EBREAK, "water depth d <= 0 or non-finite surface");
    return WT_OK;
  });
}

int wt_precondition(wt_tank* t, const double* eta_a, const double* eta_b, const double* r, double* z,
                    int precision) {
  if (!t || !eta_a || !eta_b || !r || !z) return fail(WT_EINVAL, "NULL argument");
  if (precision != WT_FP64 && precision != WT_FP32) return fail(WT_EINVAL, "precision must be WT_FP64 or WT_FP32");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    setup_geometry(*t, ea, eb, precision, true, true);
    const double* rd = in_dev(*t, r, t->io_f1, n);
    if (precision == WT_FP64) {
      WT_CK(cudaMemcpyAsync(t->b64, rd, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
      mg_cycle<double>(*t, t->b64, t->x64);
      out_copy(*t, z, t->x64, n);
    } else {
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<double, float>(rd, t->b32, n, nullptr, 0, t->s)));
      mg_cycle<float>(*t, t->b32, t->e32);
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<float, double>(t->e32, t->io_f2, n, nullptr, 0, t->s)));
      out_copy(*t, z, t->io_f2, n);
    }
    const int fl = read_flags(*t);
    if (fl) return fail(WT_EBREAK, "water depth d <= 0, non-finite surface or singular block");
    return WT_OK;
  });
}

int wt_poisson_solve(wt_tank* t, const double* eta_a, const double* eta_b, const double* rhs, double* p,
                     double tol, wt_solve_info* info) {
  if (!t || !eta_a || !eta_b || !rhs || !p) return fail(WT_EINVAL, "NULL argument");
  if (tol <= 0) tol = t->opt.tol;
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    const int prec = t->opt.mode == WT_FP64 ? WT_FP64 : WT_FP32;
    setup_geometry(*t, ea, eb, prec, true, true);
    const double* bd = in_dev(*t, rhs, t->io_f1, n);
    WT_CK(cudaMemcpyAsync(t->b64, bd, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    const double* p0 = in_dev(*t, p, t->io_f2, n);
    WT_CK(cudaMemcpyAsync(t->x64, p0, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    wt_solve_info inf{};
    int st = poisson_solve_device(*t, t->b64, t->x64, tol, &inf);
    out_copy(*t, p, t->x64, n);
    WT_CK(cudaStreamSynchronize(t->s));
    if (info) *info = inf;
    if (st == WT_ENOCONV) return fail(st, "solve stopped above its tolerance");
    if (st == WT_ETIMEOUT) return fail(st, "a grid barrier of the one-launch V-cycle gave up waiting");
    if (st != WT_OK) return fail(st, "depth <= 0, singular block or non-finite value in the solve");
    return WT_OK;
  });
}

int wt_rk_stage(wt_tank* t, int k, double dt) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (k < 1 || k > 5) return fail(WT_EINVAL, "stage k must be in [1, 5]");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(WT_EINVAL, "dt must be positive");
  if (!t->have_state) return fail(WT_EINVAL, "no state: call wt_set_state first");
  return guarded_t(t, [&]() -> int { return rk_stage(*t, k, dt); });
}

int wt_step(wt_tank* t, double dt, int nsteps) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (nsteps < 0) return fail(WT_EINVAL, "nsteps must be >= 0");
  for (int s = 0; s < nsteps; ++s)
    for (int k = 1; k <= 5; ++k) {
      const int st = wt_rk_stage(t, k, dt);
      if (st != WT_OK) return st;
    }
  return WT_OK;
}

int wt_get_stats(const wt_tank* t, long* solves, long* iterations) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (solves) *solves = t->solves;
  if (iterations) *iterations = t->iterations;
  return WT_OK;
}

int wt_profile(wt_tank* t, unsigned mask) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  return guarded([&]() -> int {
    WT_CK(cudaStreamSynchronize(t->s));
    t->prof.rec.clear();
    t->prof.used = 0;
    t->prof.mask = mask;
    return WT_OK;
  });
}

int wt_profile_read(wt_tank* t, int k, double* ms, long* launches, double* bytes, double* flops) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (k < 0 || k >= K_NCAT) return fail(WT_EINVAL, "kernel class out of range");
  return guarded([&]() -> int {
    WT_CK(cudaStreamSynchronize(t->s));
    double tot = 0.0, b = 0.0, f = 0.0;
    long cnt = 0;
    for (const auto& r : t->prof.rec) {
      if (r.cat != k) continue;
      float e = 0.f;
      WT_CK(cudaEventElapsedTime(&e, t->prof.pool[r.ev0], t->prof.pool[r.ev1]));
      tot += e;
      b += r.bytes;
      f += r.flops;
      ++cnt;
    }
    if (ms) *ms = tot;
    if (launches) *launches = cnt;
    if (bytes) *bytes = b;
    if (flops) *flops = f;
    return WT_OK;
  });
}

int wt_get_launches(const wt_tank* t, long* launches) {
  if (!t || !launches) return fail(WT_EINVAL, "NULL argument");
  *launches = t->prof.launches;
  return WT_OK;
}

// ================================================================ adjoint
int wt_set_bathymetry(wt_tank* t, const double* h) {
  if (!t || !h) return fail(WT_EINVAL, "NULL argument");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const double* hd = in_dev(*t, h, t->io_s1, t->ncols);
    std::vector<double> hh(t->ncols);
    WT_CK(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * t->ncols, cudaMemcpyDefault, t->s));
    WT_CK(cudaStreamSynchronize(t->s));
    for (double v : hh)
      if (!(v > 0) || !std::isfinite(v)) return fail(WT_EINVAL, "bathymetry must be positive and finite");
    setup_bathymetry(*t, hd);
    WT_CK(cudaStreamSynchronize(t->s));
    const double hmin = *std::min_element(hh.begin(), hh.end());
    t->hmax = *std::max_element(hh.begin(), hh.end());
    if (hmin != t->hmin) {                       // the spectral smoother's reference depth moved
      t->hmin = hmin;
      t->spec_ready = false;
      ensure_spectral(*t);
    }
    return WT_OK;
  });
}

int wt_relax(wt_tank* t, double x0, double x1, const double* eta_target, const double* u_target,
             const double* v_target, const double* w_target) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (!std::isfinite(x0) || !std::isfinite(x1) || x0 == x1) return fail(WT_EINVAL, "the zone needs x0 != x1");
  if (!t->have_state) return fail(WT_EINVAL, "no state: call wt_set_state first");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const int Nx = t->Nx, nc = t->ncols;
    const double lo = std::min(x0, x1), hi = std::max(x0, x1);
    std::vector<double> wg(nc, 0.0);
    for (int j = 0; j < Nx; ++j) {
      const double x = j * t->L / Nx;
      if (x < lo || x > hi) continue;
      const double xi = (x - x0) / (x1 - x0);               // 0 at x0, 1 at x1
      const double g = (std::exp(std::pow(xi, 3.5)) - 1.0) / (std::exp(1.0) - 1.0);
      for (int jy = 0; jy < t->Ny; ++jy) wg[(size_t)jy * Nx + j] = g;
    }
    if (!t->relax_w) t->relax_w = t->ar.alloc<double>(nc);
    WT_CK(cudaMemcpyAsync(t->relax_w, wg.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, t->s));
    const long n = t->n;
    // targets: device arrays as they are, host arrays through the staging buffers
    const double* et = eta_target ? in_dev(*t, eta_target, t->io_s1, nc) : nullptr;
    const double* ut = u_target ? in_dev(*t, u_target, t->io_f1, n) : nullptr;
    const double* wt_ = w_target ? in_dev(*t, w_target, t->io_f2, n) : nullptr;
    const double* vt = nullptr;
    if (v_target && t->Ny > 1) {
      vt = in_dev(*t, v_target, t->work[0], n);
    }
    WT_CK(launch_relax(nc, t->M1, t->relax_w, et, ut, vt, wt_, t->eta, t->u, t->Ny > 1 ? t->v : nullptr, t->w,
                       t->s));
    WT_CK(cudaStreamSynchronize(t->s));
    t->prof.launches += 1;
    return WT_OK;
  });
}

int wt_stream_function_wave(wt_tank* t, int nwaves, double H, int nmodes, double time, double* eta,
                            double* u, double* w, double* c) {
  if (!t) return fail(WT_EINVAL, "NULL tank");
  if (t->Ny != 1) return fail(WT_ENOTSUP, "stream-function waves are set on 2D tanks");
  if (nwaves < 1 || nwaves > t->Nx / 4) return fail(WT_EINVAL, "nwaves must be in [1, Nx/4]");
  if (nmodes < 2 || nmodes > 128) return fail(WT_EINVAL, "nmodes must be in [2, 128]");
  if (!(H > 0) || !std::isfinite(H) || !std::isfinite(time)) return fail(WT_EINVAL, "H must be positive");
  if (t->hmax - t->hmin > 1e-12 * t->hmax) return fail(WT_EINVAL, "stream-function waves need a flat bottom");
  const double k = 2.0 * M_PI * nwaves / t->L, d = t->hmax;
  if (H * k / (2.0 * M_PI) > 0.85 * 0.1401 * std::tanh(0.8863 * k * d))
    return fail(WT_EINVAL, "H above 0.85 x the Battjes breaking steepness");
  return guarded_t(t, [&]() -> int {
    SfWave& W = t->sf;
    if (!(W.k == k && W.d == d && W.H == H && W.g == t->g && W.N == nmodes)) {
      SfWave nw;
      if (!sf_solve(k, d, H, t->g, nmodes, nw)) return fail(WT_ENOCONV, "stream-function Newton iteration failed");
      W = nw;
    }
    const int Nx = t->Nx, M1 = t->M1;
    std::vector<double> he(Nx), hu((size_t)M1 * Nx), hw((size_t)M1 * Nx);
    for (int j = 0; j < Nx; ++j) {
      const double x = j * t->L / Nx;
      he[j] = sf_eta(W, x, time);
      for (int m = 0; m < M1; ++m) {
        const double sig = 0.5 * (std::cos(M_PI * m / t->Nz) + 1.0);
        const double z = sig * (d + he[j]) - d;
        sf_velocity(W, x, z, time, hu[(size_t)m * Nx + j], hw[(size_t)m * Nx + j]);
      }
    }
    if (eta) WT_CK(cudaMemcpy(eta, he.data(), sizeof(double) * Nx, cudaMemcpyDefault));
    if (u) WT_CK(cudaMemcpy(u, hu.data(), sizeof(double) * hu.size(), cudaMemcpyDefault));
    if (w) WT_CK(cudaMemcpy(w, hw.data(), sizeof(double) * hw.size(), cudaMemcpyDefault));
    if (c) *c = W.c;
    return WT_OK;
  });
}

int wt_levels_for(int Nx, int Ny, int Nz, int coarsest_max, int* nlevels, int* dims) {
  if (!nlevels) return fail(WT_EINVAL, "nlevels pointer is NULL");
  if (!pow2(Nx) || Nx < 4 || Nx > 4096) return fail(WT_EINVAL, "Nx must be a power of two in [4, 4096]");
  if (!(Ny == 1 || (pow2(Ny) && Ny >= 4 && Ny <= 1024)))
    return fail(WT_EINVAL, "Ny must be 1 or a power of two in [4, 1024]");
  if (Nz < 2 || Nz > 32) return fail(WT_EINVAL, "Nz must be in [2, 32]");
  if (coarsest_max < 1 || coarsest_max > 128) return fail(WT_EINVAL, "coarsest_max must be in [1, 128]");
  const auto lv = hierarchy(Nx, Ny, Nz, coarsest_max);
  if ((int)lv.size() > kMaxLevels) return fail(WT_EINVAL, "too many multigrid levels");
  *nlevels = (int)lv.size();
  if (dims)
    for (size_t l = 0; l < lv.size(); ++l)
      for (int k = 0; k < 3; ++k) dims[3 * l + k] = lv[l][k];
  const auto& c = lv.back();
  const long nc = (long)c[0] * c[1] * (c[2] + 1);
  if (nc > 128)
    return fail(WT_ENOTSUP, "coarsest level has " + std::to_string(nc) +
                                " unknowns; the dense FP64 solve takes at most 128");
  return WT_OK;
}

int wt_sigma_matrices(int Nz, int Nzc, int bc_transfer, double* D, double* F, double* R, double* P) {
  if (Nz < 2 || Nz > 32) return fail(WT_EINVAL, "Nz must be in [2, 32]");
  if (Nzc < 2 || Nzc > Nz) return fail(WT_EINVAL, "Nzc must be in [2, Nz]");
  if (bc_transfer != 0 && bc_transfer != 1) return fail(WT_EINVAL, "bc_transfer is 0 or 1");
  return guarded([&]() -> int {
    if (D) {
      const auto m = cheb_D(Nz);
      std::copy(m.begin(), m.end(), D);
    }
    if (F) {
      const auto m = cheb_filter(Nz);
      std::copy(m.begin(), m.end(), F);
    }
    if (R) {
      const auto m = cheb_restrict(Nz, Nzc, bc_transfer == 0);
      std::copy(m.begin(), m.end(), R);
    }
    if (P) {
      const auto m = cheb_prolong(Nzc, Nz);
      std::copy(m.begin(), m.end(), P);
    }
    return WT_OK;
  });
}

int wt_stream_function_solve(double k, double d, double H, double g, int nmodes, double* params, double* B,
                             double* E) {
  if (!(k > 0) || !std::isfinite(k)) return fail(WT_EINVAL, "k must be positive");
  if (!(d > 0) || !std::isfinite(d)) return fail(WT_EINVAL, "d must be positive");
  if (!(g > 0) || !std::isfinite(g)) return fail(WT_EINVAL, "g must be positive");
  if (nmodes < 2 || nmodes > 128) return fail(WT_EINVAL, "nmodes must be in [2, 128]");
  if (!(H > 0) || !std::isfinite(H)) return fail(WT_EINVAL, "H must be positive");
  if (H * k / (2.0 * M_PI) > 0.85 * 0.1401 * std::tanh(0.8863 * k * d))
    return fail(WT_EINVAL, "H above 0.85 x the Battjes breaking steepness");
  return guarded([&]() -> int {
    SfWave W;
    if (!sf_solve(k, d, H, g, nmodes, W)) return fail(WT_ENOCONV, "stream-function Newton iteration failed");
    if (params) {
      params[0] = W.c;
      params[1] = W.Q;
      params[2] = W.R;
    }
    if (B) std::copy(W.B.begin(), W.B.end(), B);
    if (E) std::copy(W.E.begin(), W.E.end(), E);
    return WT_OK;
  });
}

int wt_apply_operator_transposed(wt_tank* t, const double* eta_a, const double* eta_b, const double* lam,
                                 double* out, int precision) {
  if (!t || !eta_a || !eta_b || !lam || !out) return fail(WT_EINVAL, "NULL argument");
  if (precision != WT_FP64 && precision != WT_FP32) return fail(WT_EINVAL, "precision must be WT_FP64 or WT_FP32");
  if (t->Ny != 1) return fail(WT_ENOTSUP, "the transposed operator is 2D only");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    setup_geometry(*t, ea, eb, precision, false, false);
    const double* ld = in_dev(*t, lam, t->io_f1, n);
    if (precision == WT_FP64) {
      apply_op<double>(*t, 0, ld, t->io_f2, nullptr, false, true);
    } else {
      auto& L = t->L32[0];
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<double, float>(ld, L.x, n, nullptr, 0, t->s)));
      apply_op<float>(*t, 0, L.x, L.f, nullptr, false, true);
      WT_LAUNCH(*t, K_KRYLOV, 12.0 * n, 0.0, (launch_convert<float, double>(L.f, t->io_f2, n, nullptr, 0, t->s)));
    }
    out_copy(*t, out, t->io_f2, n);
    const int fl = read_flags(*t);
    if (fl) return fail(WT_EBREAK, "water depth d <= 0 or non-finite surface");
    return WT_OK;
  });
}

int wt_adjoint_solve(wt_tank* t, const double* eta_a, const double* eta_b, const double* rhs, double* lam,
                     double tol, wt_solve_info* info) {
  if (!t || !eta_a || !eta_b || !rhs || !lam) return fail(WT_EINVAL, "NULL argument");
  if (t->Ny != 1) return fail(WT_ENOTSUP, "the transposed problem is 2D only");
  if (tol <= 0) tol = t->opt.tol;
  return guarded_t(t, [&]() -> int {
    enter(*t);
    const long n = t->n;
    const double* ea = in_dev(*t, eta_a, t->io_s1, t->ncols);
    const double* eb = in_dev(*t, eta_b, t->io_s2, t->ncols);
    const int prec = t->opt.mode == WT_FP64 ? WT_FP64 : WT_FP32;
    setup_geometry(*t, ea, eb, prec, true, true);
    const double* bd = in_dev(*t, rhs, t->io_f1, n);
    WT_CK(cudaMemcpyAsync(t->b64, bd, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    const double* l0 = in_dev(*t, lam, t->io_f2, n);
    WT_CK(cudaMemcpyAsync(t->x64, l0, sizeof(double) * n, cudaMemcpyDeviceToDevice, t->s));
    wt_solve_info inf{};
    int st = poisson_solve_device(*t, t->b64, t->x64, tol, &inf, true);
    out_copy(*t, lam, t->x64, n);
    WT_CK(cudaStreamSynchronize(t->s));
    if (info) *info = inf;
    if (st == WT_ENOCONV) return fail(st, "transposed solve stopped above its tolerance");
    if (st != WT_OK) return fail(st, "depth <= 0, singular block or non-finite value in the solve");
    return WT_OK;
  });
}

int wt_adjoint_step(wt_tank* t, double dt, const double* eta, const double* u, const double* w,
                    double* lam_eta, double* lam_u, double* lam_w, double* dJ_dh) {
  if (t && t->nu != 0.0) return fail(WT_ENOTSUP, "the adjoint step covers the inviscid model (nu = 0)");
  if (!t || !eta || !u || !w || !lam_eta || !lam_u || !lam_w) return fail(WT_EINVAL, "NULL argument");
  if (t->Ny != 1) return fail(WT_ENOTSUP, "the adjoint step is 2D only");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(WT_EINVAL, "dt must be positive");
  NvtxRange range("wt adjoint step");
  return guarded_t(t, [&]() -> int {
    enter(*t);
    alloc_adj(*t);
    AdjBufs& B = *t->adj;
    const long n = t->n, nc = t->ncols;
    cudaStream_t s = t->s;
    auto load = [&](double* dst, const double* user, double* staging, long count) {
      const double* d = in_dev(*t, user, staging, count);
      WT_CK(cudaMemcpyAsync(dst, d, sizeof(double) * count, cudaMemcpyDeviceToDevice, s));
    };
    // recompute the step from its start, keeping every stage's values
    load(t->eta, eta, t->io_s1, nc);
    load(t->u, u, t->io_f1, n);
    load(t->w, w, t->io_f2, n);
    WT_CK(cudaMemsetAsync(t->v, 0, sizeof(double) * n, s));
    WT_CK(cudaMemsetAsync(t->Keta, 0, sizeof(double) * nc, s));
    WT_CK(cudaMemsetAsync(t->Ku, 0, sizeof(double) * n, s));
    WT_CK(cudaMemsetAsync(t->Kw, 0, sizeof(double) * n, s));
    WT_CK(cudaMemsetAsync(t->p, 0, sizeof(double) * n, s));
    t->have_state = true;
    bool noconv = false;
    for (int k = 1; k <= 5; ++k) {
      const int st = rk_stage(*t, k, dt, &B.st[k - 1]);
      if (st == WT_ENOCONV) noconv = true;
      else if (st != WT_OK) return st;
    }
    t->time += dt;
    // reverse the stages
    load(B.Le, lam_eta, t->io_s1, nc);
    load(B.Lu, lam_u, t->io_f1, n);
    load(B.Lw, lam_w, t->io_f2, n);
    WT_CK(cudaMemsetAsync(B.LKe, 0, sizeof(double) * nc, s));
    WT_CK(cudaMemsetAsync(B.LKu, 0, sizeof(double) * n, s));
    WT_CK(cudaMemsetAsync(B.LKw, 0, sizeof(double) * n, s));
    WT_CK(cudaMemsetAsync(B.lh, 0, sizeof(double) * nc, s));
    for (int k = 5; k >= 1; --k) {
      const int st = adjoint_stage(*t, k, dt, kAlpha, kBeta);
      if (st == WT_ENOCONV) noconv = true;
      else if (st != WT_OK) return fail(st, "transposed solve failed (depth <= 0 or non-finite)");
    }
    out_copy(*t, lam_eta, B.Le, nc);
    out_copy(*t, lam_u, B.Lu, n);
    out_copy(*t, lam_w, B.Lw, n);
    if (dJ_dh) {
      const double* hd = in_dev(*t, dJ_dh, t->io_s2, nc);
      WT_CK(launch_add(const_cast<double*>(hd), B.lh, nc, s));
      if (hd != dJ_dh) out_copy(*t, dJ_dh, hd, nc);
    }
    const int fl = read_flags(*t);
    if (fl) return fail(WT_EBREAK, "water depth d <= 0 or non-finite state in the adjoint step");
    if (noconv) return fail(WT_ENOCONV, "a forward or transposed solve stopped above its tolerance");
    return WT_OK;
  });
}

// ================================================================ batches
}  // extern "C"

struct wt_batch {
  std::vector<wt_tank*> tanks;
  wt::Arena ar;
  wt::BatchTankDesc* d_desc = nullptr;
  int* d_order = nullptr;
  double* d_dt = nullptr;
  double* d_stats = nullptr;      // 4 doubles per tank
  cudaStream_t s = nullptr;       // the stream launches go to (own_s unless the caller set one)
  cudaStream_t own_s = nullptr;
  int smem = 96 * 1024;
  std::vector<int> order;
};

namespace {
void fill_desc(wt_batch& b) {
  const int nt = (int)b.tanks.size();
  std::vector<BatchTankDesc> d(nt);
  for (int i = 0; i < nt; ++i) {
    wt_tank& t = *b.tanks[i];
    BatchTankDesc& D = d[i];
    D.nl = (int)t.L64.size();
    D.Nx = t.Nx; D.logNx = ilog2(t.Nx); D.Nz = t.Nz; D.M1 = t.M1; D.ncols = t.ncols; D.n = t.n;
    D.L = t.L; D.g = t.g;
    D.lv32 = t.tl32; D.lv64 = t.tl64; D.S = t.sd;
    D.AinvT = t.cLU; D.cDx = t.cDx; D.cDy = t.cDy;
    D.V64 = t.V64; D.Z64 = t.Z64; D.b32 = t.b32; D.e32 = t.e32;
    D.V32 = t.V32; D.Z32 = t.Z32; D.r64 = t.r64;
    D.eta = t.eta; D.eta_new = t.eta_new; D.Keta = t.Keta; D.f_eta = t.f_eta; D.eta_x = t.eta_x;
    D.u = t.u; D.w = t.w; D.Ku = t.Ku; D.Kw = t.Kw; D.p = t.p; D.zero_s = t.zero_s;
    for (int k = 0; k < 18; ++k) D.work[k] = t.work[k];
    D.filt_x = t.filt_x; D.Fcheb = t.Fcheb;
    D.flag = t.dflag;
    D.stats = b.d_stats + 4 * i;
    D.tol = t.opt.tol; D.omega = t.opt.omega; D.inner_tol = t.opt.inner_tol;
    D.nu1 = t.opt.nu1; D.nu2 = t.opt.nu2; D.restart = t.opt.restart; D.max_it = t.opt.max_it;
    D.max_ir = t.opt.max_ir;
    D.filter = t.opt.filter; D.linear = t.opt.linear;
  }
  WT_CK(cudaMemcpy(b.d_desc, d.data(), sizeof(BatchTankDesc) * nt, cudaMemcpyHostToDevice));
}

// Everything one CTA stages in its dynamic shared memory must fit in smem
// bytes: an FP64 row pair of the finest level without prefetch (two complex
// rows plus half a row of twiddles), the coarsest dense inverse, one block of
// the smoother per warp.
int check_batch_tank(const wt_tank& t, int smem) {
  if (t.Ny != 1) return fail(WT_EINVAL, "batched tanks are 2D (Ny = 1)");
  if (t.opt.smoother != 0 || t.opt.cycle != 0)
    return fail(WT_ENOTSUP, "batched tanks use the block-Jacobi smoother and the V-cycle");
  const size_t row = (2 * (size_t)t.Nx + t.Nx / 2) * 2 * sizeof(double);
  const size_t coarse = (size_t)t.ncoarse * (t.ncoarse + 1) * sizeof(double) + (t.ncoarse + 1) * sizeof(int);
  const size_t blk = (size_t)t.M1 * (2 * t.M1 + 1) * (t.opt.mode == WT_FP64 ? sizeof(double) : sizeof(float));
  if (row > (size_t)smem) return fail(WT_ENOTSUP, "batched tanks need Nx <= 2048");
  if (coarse > (size_t)smem) return fail(WT_ENOTSUP, "batched tank's coarsest level is too large (coarsest_max)");
  if (blk > (size_t)smem) return fail(WT_ENOTSUP, "batched tank's Nz is too large");
  return WT_OK;
}
}  // namespace

extern "C" {

int wt_create_batch(int ntanks, const int* Nx, const int* Nz, const double* L, double g, double nu,
                    const double* const* bathymetry, wt_batch** out) {
  if (!out || !Nx || !Nz || !L || !bathymetry) return fail(WT_EINVAL, "NULL argument");
  *out = nullptr;
  if (ntanks < 1 || ntanks > 65535) return fail(WT_EINVAL, "ntanks must be in [1, 65535]");
  if (nu != 0.0) return fail(WT_ENOTSUP, "batched tanks run the inviscid model (nu = 0)");
  std::unique_ptr<wt_batch> b(new wt_batch());
  for (int i = 0; i < ntanks; ++i) {
    wt_tank* t = nullptr;
    const int st = wt_create(Nx[i], 1, Nz[i], L[i], g, nu, bathymetry[i], &t);
    if (st != WT_OK) {
      for (wt_tank* q : b->tanks) wt_destroy(q);
      return st;
    }
    b->tanks.push_back(t);
    const int c = check_batch_tank(*t, b->smem);
    if (c != WT_OK) {
      for (wt_tank* q : b->tanks) wt_destroy(q);
      return c;
    }
  }
  const int rc = guarded([&]() -> int {
    WT_CK(cudaStreamCreateWithFlags(&b->own_s, cudaStreamNonBlocking));
    b->s = b->own_s;
    b->d_desc = b->ar.alloc<BatchTankDesc>(ntanks);
    b->d_order = b->ar.alloc<int>(ntanks);
    b->d_dt = b->ar.alloc<double>(ntanks);
    b->d_stats = b->ar.alloc<double>(4 * (size_t)ntanks);
    WT_CK(cudaMemset(b->d_stats, 0, sizeof(double) * 4 * ntanks));
    // longest-processing-time first: largest tanks take the first CTAs
    b->order.resize(ntanks);
    for (int i = 0; i < ntanks; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->tanks[x]->n > b->tanks[y]->n; });
    WT_CK(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * ntanks, cudaMemcpyHostToDevice));
    fill_desc(*b);
    return WT_OK;
  });
  if (rc != WT_OK) {
    for (wt_tank* q : b->tanks) wt_destroy(q);
    if (b->own_s) cudaStreamDestroy(b->own_s);
    return rc;
  }
  *out = b.release();
  return WT_OK;
}

int wt_batch_set_options(wt_batch* b, const wt_options* o) {
  if (!b || !o) return fail(WT_EINVAL, "NULL argument");
  for (wt_tank* t : b->tanks) {
    const int st = wt_set_options(t, o);
    if (st != WT_OK) return st;
    const int c = check_batch_tank(*t, b->smem);
    if (c != WT_OK) return c;
  }
  return guarded([&]() -> int {
    fill_desc(*b);
    return WT_OK;
  });
}

int wt_batch_set_state(wt_batch* b, int i, const double* eta, const double* u, const double* w,
                       double time) {
  if (!b || i < 0 || i >= (int)b->tanks.size()) return fail(WT_EINVAL, "tank index out of range");
  return wt_set_state(b->tanks[i], eta, u, nullptr, w, time);
}

int wt_batch_get_state(const wt_batch* b, int i, double* eta, double* u, double* w, double* time) {
  if (!b || i < 0 || i >= (int)b->tanks.size()) return fail(WT_EINVAL, "tank index out of range");
  return wt_get_state(b->tanks[i], eta, u, nullptr, w, time);
}

int wt_batch_step(wt_batch* b, const double* dt, int nsteps) {
  if (!b || !dt) return fail(WT_EINVAL, "NULL argument");
  if (nsteps < 0) return fail(WT_EINVAL, "nsteps must be >= 0");
  NvtxRange range("wt batch step");
  const int nt = (int)b->tanks.size();
  for (int i = 0; i < nt; ++i) {
    if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(WT_EINVAL, "dt must be positive");
    if (!b->tanks[i]->have_state) return fail(WT_EINVAL, "tank without state: call wt_batch_set_state");
  }
  if (nsteps == 0) return WT_OK;
  return guarded([&]() -> int {
    fill_desc(*b);
    for (wt_tank* t : b->tanks) WT_CK(cudaStreamSynchronize(t->s));   // pending state uploads
    WT_CK(cudaMemcpyAsync(b->d_dt, dt, sizeof(double) * nt, cudaMemcpyHostToDevice, b->s));
    const int mode = b->tanks[0]->opt.mode;              // one option set for every tank
    WT_CK(launch_batch_step(b->d_desc, b->d_order, nt, b->d_dt, nsteps, b->smem, mode, b->s));
    WT_CK(cudaStreamSynchronize(b->s));
    int bad = 0;
    for (int i = 0; i < nt; ++i) {
      wt_tank& t = *b->tanks[i];
      t.time += nsteps * dt[i];
      t.prof.launches += 1;
      const int f = read_flags(t);
      if (f & 15) bad |= 1;
      if (f & 16) bad |= 2;
    }
    if (bad & 1) return fail(WT_EBREAK, "a batched tank has depth <= 0 or a non-finite state");
    if (bad & 2) return fail(WT_ENOCONV, "a batched pressure solve stopped above its tolerance");
    return WT_OK;
  });
}

int wt_batch_stats(const wt_batch* b, int i, long* solves, long* iterations, double* last_rel) {
  if (!b || i < 0 || i >= (int)b->tanks.size()) return fail(WT_EINVAL, "tank index out of range");
  return guarded([&]() -> int {
    double s[4];
    WT_CK(cudaMemcpy(s, b->d_stats + 4 * i, sizeof(s), cudaMemcpyDeviceToHost));
    if (solves) *solves = (long)s[0];
    if (iterations) *iterations = (long)s[1];
    if (last_rel) *last_rel = s[2];
    return WT_OK;
  });
}

int wt_batch_destroy(wt_batch* b) {
  if (!b) return WT_OK;
  if (b->s) cudaStreamSynchronize(b->s);
  for (wt_tank* t : b->tanks) wt_destroy(t);
  if (b->own_s) cudaStreamDestroy(b->own_s);
  delete b;
  return WT_OK;
}

int wt_batch_size(const wt_batch* b, int* ntanks) {
  if (!b || !ntanks) return fail(WT_EINVAL, "NULL argument");
  *ntanks = (int)b->tanks.size();
  return WT_OK;
}

int wt_batch_tank_dims(const wt_batch* b, int i, int* Nx, int* Nz) {
  if (!b || i < 0 || i >= (int)b->tanks.size()) return fail(WT_EINVAL, "tank index out of range");
  if (Nx) *Nx = b->tanks[i]->Nx;
  if (Nz) *Nz = b->tanks[i]->Nz;
  return WT_OK;
}

int wt_batch_get_options(const wt_batch* b, wt_options* o) {
  if (!b || !o || b->tanks.empty()) return fail(WT_EINVAL, "NULL argument");
  *o = b->tanks[0]->opt;
  return WT_OK;
}

int wt_batch_set_stream(wt_batch* b, void* stream) {
  if (!b) return fail(WT_EINVAL, "NULL batch");
  return guarded([&]() -> int {
    WT_CK(cudaStreamSynchronize(b->s));
    b->s = stream ? static_cast<cudaStream_t>(stream) : b->own_s;
    return WT_OK;
  });
}

int wt_destroy(wt_tank* t) {
  if (!t) return WT_OK;
  cudaStreamSynchronize(t->s);
  destroy_graphs(*t);
  if (t->side) cudaStreamSynchronize(t->side);
  if (t->side2) cudaStreamSynchronize(t->side2);
  if (t->ev_fork) cudaEventDestroy(t->ev_fork);
  if (t->ev_join) cudaEventDestroy(t->ev_join);
  if (t->ev_join2) cudaEventDestroy(t->ev_join2);
  if (t->side) cudaStreamDestroy(t->side);
  if (t->side2) cudaStreamDestroy(t->side2);
  if (t->order_ev) cudaEventDestroy(t->order_ev);
  if (t->own_stream) cudaStreamDestroy(t->own_stream);
  if (t->hflag) cudaFreeHost(t->hflag);
  if (t->hst) cudaFreeHost(t->hst);
  delete t;
  return WT_OK;
}

int wt_last_error(char* buf, size_t n) {
  if (buf && n) {
    const size_t k = std::min(n - 1, g_err.size());
    std::memcpy(buf, g_err.data(), k);
    buf[k] = '\0';
  }
  return g_code;
}

}  // extern "C"
