// wt_apply_operator_static: the mixed-stage operator of a 2D tank for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all - code running inside another
// framework's memory pool, an embedded solver that only receives buffers, or
// a process that must not change its device-memory footprint after start-up.
// This entry point therefore allocates nothing: every temporary (metric,
// derivative rows, Chebyshev matrices, FFT twiddles, the error flag) lives in
// one file-scope __device__ array of fixed size, and the caller passes device
// pointers for all inputs and outputs.  It computes exactly what
// wt_apply_operator(..., WT_FP64) computes for Ny = 1, with the same kernels.
#include "../../include/wt.h"
#include "wt_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace {

// Maximum problem: Nx <= 2048, Nz <= 32 (67,584 unknowns).  Layout (doubles):
// Px, Gx, part (3 x 67,584), metric (14 x 2048), surface derivatives
// (3 x 2048), D, D^2, D diag(sigma) D (3 x 33 x 33), sigma (33), twiddles
// (1024 complex), error flag.  2.5 MiB covers it with 256-byte alignment of
// every piece.  Every GPU that loads the library holds this array until exit.
constexpr size_t kScratchBytes = 5u << 19;   // 2.5 MiB
constexpr int kMaxNx = 2048, kMaxNz = 32;

__device__ __align__(256) unsigned char wt_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch[kMaxDevices] = {nullptr};
std::mutex g_mu;

int fail(int code, const char* msg) { return wt::set_error(code, msg); }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device memory of the current device (or managed memory): memory of another
// GPU would be read without peer access, so it is refused like host memory.
bool is_device_ptr(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Host-side address of the scratch array on the current device (the array's
// name in host code is only a stand-in, never a device address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, wt_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int wt_apply_operator_static(int Nx, int Nz, double L, const double* h,
                                        const double* eta_a, const double* eta_b,
                                        const double* p, double* Ap, void* stream) {
  using namespace wt;
  if (Nx < 4 || Nx > kMaxNx || (Nx & (Nx - 1)) != 0)
    return fail(WT_EINVAL, "wt_apply_operator_static: Nx must be a power of two in [4, 2048]");
  if (Nz < 2 || Nz > kMaxNz) return fail(WT_EINVAL, "wt_apply_operator_static: Nz must be in [2, 32]");
  if (!(L > 0) || !std::isfinite(L)) return fail(WT_EINVAL, "wt_apply_operator_static: L must be positive");
  if (!h || !eta_a || !eta_b || !p || !Ap) return fail(WT_EINVAL, "wt_apply_operator_static: NULL pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(WT_ECUDA, "wt_apply_operator_static: no current CUDA device");
  }
  if (!is_device_ptr(h, dev) || !is_device_ptr(eta_a, dev) || !is_device_ptr(eta_b, dev) ||
      !is_device_ptr(p, dev) || !is_device_ptr(Ap, dev))
    return fail(WT_EINVAL, "wt_apply_operator_static: all arrays must be device memory of the current device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(WT_ECUDA, cudaGetErrorString(e));

  const int M1 = Nz + 1;
  const long n = (long)M1 * Nx;
  int logNx = 0;
  while ((1 << logNx) < Nx) ++logNx;
  // carve the scratch array
  unsigned char* cur = static_cast<unsigned char*>(base);
  auto take = [&](size_t bytes) {
    unsigned char* q = cur;
    cur += align256(bytes);
    return q;
  };
  double* Px = reinterpret_cast<double*>(take(sizeof(double) * n));
  double* Gx = reinterpret_cast<double*>(take(sizeof(double) * n));
  double* part = reinterpret_cast<double*>(take(sizeof(double) * n));
  double* meta = reinterpret_cast<double*>(take(sizeof(double) * kMeta * Nx));
  double* hx = reinterpret_cast<double*>(take(sizeof(double) * Nx));
  double* eax = reinterpret_cast<double*>(take(sizeof(double) * Nx));
  double* ebx = reinterpret_cast<double*>(take(sizeof(double) * Nx));
  double* dD = reinterpret_cast<double*>(take(sizeof(double) * 3 * M1 * M1));
  double* dsig = reinterpret_cast<double*>(take(sizeof(double) * M1));
  double2* dtw = reinterpret_cast<double2*>(take(sizeof(double2) * (Nx / 2)));
  int* dflag = reinterpret_cast<int*>(take(sizeof(int)));
  if ((size_t)(cur - static_cast<unsigned char*>(base)) > kScratchBytes)
    return fail(WT_EINVAL, "wt_apply_operator_static: problem exceeds the static scratch");

  // host FP64 tables on the stack: CGL nodes, d/dsigma, D^2, D diag(sigma) D, twiddles
  double xi[kMaxNz + 1], sig[kMaxNz + 1];
  double D[(kMaxNz + 1) * (kMaxNz + 1)], D2[(kMaxNz + 1) * (kMaxNz + 1)], DSD[(kMaxNz + 1) * (kMaxNz + 1)];
  double tw[kMaxNx];      // Nx/2 complex values
  for (int m = 0; m < M1; ++m) {
    xi[m] = std::cos(M_PI * m / Nz);
    sig[m] = 0.5 * (xi[m] + 1.0);
  }
  for (int i = 0; i < M1; ++i) {
    double rs = 0.0;
    for (int j = 0; j < M1; ++j) {
      if (i == j) continue;
      const double ci = (i == 0 || i == Nz) ? 2.0 : 1.0, cj = (j == 0 || j == Nz) ? 2.0 : 1.0;
      const double v = ci / cj * (((i + j) & 1) ? -1.0 : 1.0) / (xi[i] - xi[j]);
      D[i * M1 + j] = 2.0 * v;
      rs += v;
    }
    D[i * M1 + i] = -2.0 * rs;
  }
  for (int i = 0; i < M1; ++i)
    for (int j = 0; j < M1; ++j) {
      double a2 = 0.0, a3 = 0.0;
      for (int k = 0; k < M1; ++k) {
        a2 += D[i * M1 + k] * D[k * M1 + j];
        a3 += D[i * M1 + k] * sig[k] * D[k * M1 + j];
      }
      D2[i * M1 + j] = a2;
      DSD[i * M1 + j] = a3;
    }
  for (int j = 0; j < Nx / 2; ++j) {
    tw[2 * j] = std::cos(2.0 * M_PI * j / Nx);
    tw[2 * j + 1] = -std::sin(2.0 * M_PI * j / Nx);
  }
  const size_t MM = sizeof(double) * M1 * M1;
  if ((e = cudaMemcpyAsync(dD, D, MM, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dD + M1 * M1, D2, MM, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dD + 2 * M1 * M1, DSD, MM, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dsig, sig, sizeof(double) * M1, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dtw, tw, sizeof(double2) * (Nx / 2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(dflag, 0, sizeof(int), s)) != cudaSuccess)   // the flag must start at zero
    return fail(WT_ECUDA, cudaGetErrorString(e));

  auto pass = [&](const double* in, double* out, int nrows) {
    RowPass<double> a;
    a.in = in;
    a.out = out;
    a.nrows = nrows;
    a.Nin = a.Nout = Nx;
    a.logNin = a.logNout = logNx;
    a.op = XOP_DERIV;
    a.kscale = 2.0 * M_PI / L;
    a.tw = dtw;
    a.logNtw = logNx;
    return a;
  };
  // surface slopes, metric of both geometries (Eq. 1_Scoef)
  if ((e = launch_rowpass(pass(h, hx, 1), s)) != cudaSuccess ||
      (e = launch_rowpass(pass(eta_a, eax, 1), s)) != cudaSuccess ||
      (e = launch_rowpass(pass(eta_b, ebx, 1), s)) != cudaSuccess ||
      (e = launch_metric_fill(Nx, h, hx, nullptr, eta_a, eax, nullptr, eta_b, ebx, nullptr, meta, dflag, s)) !=
          cudaSuccess)
    return fail(WT_ECUDA, cudaGetErrorString(e));
  // Ap = Div_a(Grad_b p) inside, p on the surface rows, n . Grad_b p at the bottom
  LevelView<double> V;
  V.Nx = Nx; V.Ny = 1; V.Nz = Nz; V.M1 = M1; V.logNx = logNx; V.logNy = 0;
  V.ncols = Nx; V.n = n; V.L = L;
  V.sigma = dsig; V.D = dD; V.D2 = dD + M1 * M1; V.DSD = dD + 2 * M1 * M1; V.meta = meta;
  V.tw = dtw; V.logNtw = logNx;
  RowPass<double> last = pass(Gx, Ap, M1);
  last.skip_bc = 1;
  last.Ny = 1;
  last.M1 = M1;
  last.add = part;
  last.epi = EPI_ADD;
  if ((e = launch_rowpass(pass(p, Px, M1), s)) != cudaSuccess ||
      (e = launch_op_cols<double>(V, p, Px, nullptr, Gx, nullptr, part, s)) != cudaSuccess ||
      (e = launch_rowpass(last, s)) != cudaSuccess)
    return fail(WT_ECUDA, cudaGetErrorString(e));
  int hflag = 0;
  if ((e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(WT_ECUDA, cudaGetErrorString(e));
  if (hflag) return fail(WT_EBREAK, "wt_apply_operator_static: water depth d <= 0 or non-finite surface");
  return WT_OK;
}
