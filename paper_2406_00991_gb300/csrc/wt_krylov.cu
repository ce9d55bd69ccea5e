// Krylov kernels of the outer iteration (Sec. 4.4): flexible GMRES(m) with
// classical Gram-Schmidt applied twice (two block dot products per Arnoldi
// step instead of j sequential ones), warp-shuffle + shared-memory
// reductions accumulated in FP64, and the small Hessenberg / Givens update on
// the device so the host only reads one residual estimate per iteration.
//
// GMRES state vector st (FP64, device), offsets in wt_internal.h users:
//   st[0] beta, st[1] |g_{j+1}|, st[2] 1/h_{j+1,j}, st[3] done flag,
//   st[4] ||b||, st[5] h_{j+1,j}, st[6] tolerance, then h1, h2, cs, sn, g, y
//   and H (column-major).  The tolerance and ||b|| live on the device so a
//   captured Arnoldi step stays valid across solves.
#include "wt_internal.h"

#include <algorithm>

namespace wt {

constexpr int OFF_H1 = 8, OFF_H2 = 72, OFF_CS = 136, OFF_SN = 200, OFF_G = 264, OFF_Y = 328,
              OFF_H = 392;

// Per-CTA partial sums of V_i^T w (i < nvec) and, with with_norm, ||w||^2.
// NV >= nvec bounds the unrolled vector loops at compile time (0, 4, 8, 16,
// 32), so that short bases keep few registers and a high occupancy.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_dots(const T* __restrict__ w, const T* __restrict__ V,
                                             long ldv, int nvec, long n, double* __restrict__ partial,
                                             int with_norm) {
  pdl_enter();
  __shared__ double red[8][NV + 1];
  T acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = T(0);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const T wv = w[e];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) acc[i] += wv * V[i * ldv + e];
    acc[NV] += wv * wv;
  }
  const int nvals = nvec + with_norm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i <= NV; ++i) {
    const bool used = (i < nvec) || (i == NV && with_norm);
    if (!used) continue;
    double v = (double)acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
    const int src = (i < nvec) ? i : NV;
    double s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][src];
    partial[(long)blockIdx.x * nvals + i] = s;
  }
}

// vout = (w - V h) * inv_norm, h = st[OFF_H2..], inv_norm = st[2]; vout may
// be w itself (each element is read and written by one thread), and v32, if
// given, receives the FP32 rounding of vout (the FP32 V-cycle's input).
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_update_normalize(const T* w, const T* __restrict__ V,
                                                         long ldv, int nvec, long n,
                                                         const double* __restrict__ h,
                                                         const double* __restrict__ inv_norm,
                                                         T* vout, float* __restrict__ v32) {
  pdl_enter();
  __shared__ T sh[NV + 1];
  for (int i = threadIdx.x; i < NV; i += blockDim.x) sh[i] = i < nvec ? (T)h[i] : T(0);
  __syncthreads();
  const T s = (T)(*inv_norm);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    T wv = w[e];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) wv -= sh[i] * V[i * ldv + e];
    wv *= s;
    vout[e] = wv;
    if (v32) v32[e] = (float)wv;
  }
}

// x += sum_i y_i Z_i, y = st[OFF_Y..]
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_lincomb(T* __restrict__ x, const T* __restrict__ Z, long ldz,
                                                int nvec, long n, const double* __restrict__ y) {
  pdl_enter();
  __shared__ T sy[NV + 1];
  for (int i = threadIdx.x; i < NV; i += blockDim.x) sy[i] = i < nvec ? (T)y[i] : T(0);
  __syncthreads();
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    T acc = x[e];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) acc += sy[i] * Z[i * ldz + e];
    x[e] = acc;
  }
}

template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, long n,
                          const double* __restrict__ scale, int invert) {
  pdl_enter();
  double s = 1.0;
  if (scale) s = invert ? 1.0 / *scale : *scale;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = (To)((double)in[e] * s);
}

template <typename T>
__global__ void k_axpy_from(double* __restrict__ x, const T* __restrict__ e, long n,
                            const double* __restrict__ scale) {
  pdl_enter();
  const double s = *scale;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] += s * (double)e[i];
}

__global__ void k_nyquist_coef_f(const float* __restrict__ r, int nrows, int N, float* __restrict__ rho) {
  pdl_enter();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  float s = 0;
  for (int j = lane; j < N; j += 32) s += ((j & 1) ? -1.f : 1.f) * r[(long)warp * N + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rho[warp] = s / (float)N;
}
__global__ void k_nyquist_coef_d(const double* __restrict__ r, int nrows, int N, double* __restrict__ rho) {
  pdl_enter();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  double s = 0;
  for (int j = lane; j < N; j += 32) s += ((j & 1) ? -1.0 : 1.0) * r[(long)warp * N + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rho[warp] = s / (double)N;
}

// ---- small dense GMRES part
// Sum over b < nblk of partial[b * nvals + i], by one warp: the lanes stride
// over the blocks with four accumulators in flight, then a shuffle tree; the
// result is returned in every lane.  __ldcg: the partials were written by
// other CTAs of the same (or the previous) launch.
__device__ double warp_sum_partials(const double* partial, int nblk, int nvals, int i, int lane) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int b = lane;
  for (; b + 96 < nblk; b += 128) {
    s0 += __ldcg(partial + (long)b * nvals + i);
    s1 += __ldcg(partial + (long)(b + 32) * nvals + i);
    s2 += __ldcg(partial + (long)(b + 64) * nvals + i);
    s3 += __ldcg(partial + (long)(b + 96) * nvals + i);
  }
  for (; b < nblk; b += 32) s0 += __ldcg(partial + (long)b * nvals + i);
  double s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One warp.
__global__ void k_gmres_init(double* st, const double* __restrict__ partial, int nblk, int m,
                             double bnorm, double tol) {
  pdl_enter();
  const double ww = warp_sum_partials(partial, nblk, 1, 0, threadIdx.x & 31);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(ww);
  st[0] = beta;
  st[1] = beta;
  st[2] = beta > 0 ? 1.0 / beta : 0.0;
  st[3] = (beta <= tol * bnorm) ? 1.0 : 0.0;
  st[4] = bnorm;
  st[6] = tol;
  for (int i = 0; i <= m; ++i) st[OFF_G + i] = 0.0;
  st[OFF_G] = beta;
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes (h1 in
// st, h2 and ||w||^2 given), the Givens rotations, the residual estimate and
// the done flag (one thread).
__device__ void arnoldi_update(double* st, const double* h2, double ww, int j, int m) {
  const double tol = st[6];
  double* H = st + OFF_H + (long)j * (m + 1);
  double hh = ww;
  for (int i = 0; i <= j; ++i) {
    H[i] = st[OFF_H1 + i] + h2[i];
    st[OFF_H2 + i] = h2[i];
    hh -= h2[i] * h2[i];
  }
  const double hn = hh > 0 ? sqrt(hh) : 0.0;
  for (int i = 0; i < j; ++i) {
    const double c = st[OFF_CS + i], s = st[OFF_SN + i];
    const double t = c * H[i] + s * H[i + 1];
    H[i + 1] = -s * H[i] + c * H[i + 1];
    H[i] = t;
  }
  const double den = hypot(H[j], hn);
  const double c = den > 0 ? H[j] / den : 1.0, s = den > 0 ? hn / den : 0.0;
  st[OFF_CS + j] = c;
  st[OFF_SN + j] = s;
  H[j] = den;
  const double gj = st[OFF_G + j];
  st[OFF_G + j + 1] = -s * gj;
  st[OFF_G + j] = c * gj;
  const double res = fabs(st[OFF_G + j + 1]);
  st[1] = res;
  st[5] = hn;
  // a numerically negligible new direction ends the cycle (lucky breakdown)
  const bool breakdown = !(hn > 1e-14 * den);
  st[2] = breakdown ? 0.0 : 1.0 / hn;
  st[3] = (res <= tol * st[4] || breakdown) ? 1.0 : 0.0;
}

__global__ void k_gmres_solve_y(double* st, int k, int m) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = st[OFF_G + i];
    for (int l = i + 1; l < k; ++l) s -= st[OFF_H + (long)l * (m + 1) + i] * st[OFF_Y + l];
    st[OFF_Y + i] = s / st[OFF_H + (long)i * (m + 1) + i];
  }
}

// ---- single-launch reductions: every CTA writes its partial sums, and the
// last CTA to finish (an atomic ticket; no CTA waits for another) adds them
// up.  The ticket counter returns to zero for the next launch.
__device__ inline bool last_block(unsigned* ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0u;
  }
  return s_last != 0;
}

// k_dots followed (in the last CTA) by the sum of the partials into out.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_dots_sum(const T* __restrict__ w, const T* __restrict__ V, long ldv,
                                                 int nvec, long n, double* __restrict__ partial, int with_norm,
                                                 double* __restrict__ out, unsigned* ticket) {
  pdl_enter();
  __shared__ double red[8][NV + 1];
  T acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = T(0);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const T wv = w[e];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) acc[i] += wv * V[i * ldv + e];
    acc[NV] += wv * wv;
  }
  const int nvals = nvec + with_norm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i <= NV; ++i) {
    const bool used = (i < nvec) || (i == NV && with_norm);
    if (!used) continue;
    double v = (double)acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
    const int src = (i < nvec) ? i : NV;
    double s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][src];
    partial[(long)blockIdx.x * nvals + i] = s;
  }
  if (!last_block(ticket)) return;
  for (int i = warp; i < nvals; i += (int)(blockDim.x >> 5)) {
    const double s = warp_sum_partials(partial, (int)gridDim.x, nvals, i, lane);
    if (lane == 0) out[i] = s;
  }
}

// w -= V h1 (h1 = st[OFF_H1..]) and the per-CTA sums of (V^T w, ||w||^2);
// the last CTA adds them up and performs the Arnoldi / Givens update of
// column j (arnoldi_update).  NV >= nvec >= 1.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_update_dots_arnoldi(T* __restrict__ w, const T* __restrict__ V,
                                                            long ldv, int nvec, long n, double* st,
                                                            double* __restrict__ partial, int j, int m,
                                                            unsigned* ticket) {
  pdl_enter();
  __shared__ double red[8][NV + 1];
  __shared__ T sh[NV];
  const double* h = st + OFF_H1;
  for (int i = threadIdx.x; i < NV; i += blockDim.x) sh[i] = i < nvec ? (T)h[i] : T(0);
  __syncthreads();
  T acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = T(0);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    T v[NV];
    T wv = w[e];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) { v[i] = V[i * ldv + e]; wv -= sh[i] * v[i]; }
    w[e] = wv;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nvec) acc[i] += wv * v[i];
    acc[NV] += wv * wv;
  }
  const int nvals = nvec + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i <= NV; ++i) {
    if (!(i < nvec || i == NV)) continue;
    double v = (double)acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
    const int src = (i < nvec) ? i : NV;
    double s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][src];
    partial[(long)blockIdx.x * nvals + i] = s;
  }
  if (!last_block(ticket)) return;
  __shared__ double h2[64];
  __shared__ double ww;
  for (int i = warp; i < nvals; i += (int)(blockDim.x >> 5)) {
    const double s = warp_sum_partials(partial, (int)gridDim.x, nvals, i, lane);
    if (lane == 0) {
      if (i < j + 1) h2[i] = s; else ww = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) arnoldi_update(st, h2, ww, j, m);
}

// ------------------------------------------------------------------ launchers
static inline int blocks_for(long n) {
  return (int)std::min<long>(std::max<long>(1, (n + 255) / 256), (long)sm_count() * 4);
}

// The compile-time bound NV of the basis loops: the smallest of 0 (no
// vectors), 4, 8, 16, 32 that holds nvec.
#define WT_NV_DISPATCH(nvec, CALL) \
  ((nvec) <= 0 ? CALL(0) : (nvec) <= 4 ? CALL(4) : (nvec) <= 8 ? CALL(8) : (nvec) <= 16 ? CALL(16) : CALL(32))
#define WT_NV1_DISPATCH(nvec, CALL) \
  ((nvec) <= 4 ? CALL(4) : (nvec) <= 8 ? CALL(8) : (nvec) <= 16 ? CALL(16) : CALL(32))

template <typename T>
cudaError_t launch_dots(const T* w, const T* V, long ldv, int nvec, long n, double* partial, int nblk,
                        int with_norm, cudaStream_t s) {
#define WT_C(NV) launch_k(k_dots<T, NV>, dim3(nblk), dim3(256), 0, s, w, V, ldv, nvec, n, partial, with_norm)
  return WT_NV_DISPATCH(nvec, WT_C);
#undef WT_C
}
template <typename T>
cudaError_t launch_update_normalize(const T* w, const T* V, long ldv, int nvec, long n, const double* h,
                                    const double* inv_norm, T* vout, float* v32, cudaStream_t s) {
#define WT_C(NV) launch_k(k_update_normalize<T, NV>, dim3(blocks_for(n)), dim3(256), 0, s, w, V, ldv, nvec, n, h, \
                          inv_norm, vout, v32)
  return WT_NV_DISPATCH(nvec, WT_C);
#undef WT_C
}
template <typename T>
cudaError_t launch_lincomb(T* x, const T* Z, long ldz, int nvec, long n, const double* y,
                           cudaStream_t s) {
#define WT_C(NV) launch_k(k_lincomb<T, NV>, dim3(blocks_for(n)), dim3(256), 0, s, x, Z, ldz, nvec, n, y)
  return WT_NV_DISPATCH(nvec, WT_C);
#undef WT_C
}
template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* in, To* out, long n, const double* scale, int invert,
                           cudaStream_t s) {
  return launch_k(k_convert<Ti, To>, dim3(blocks_for(n)), dim3(256), 0, s, in, out, n, scale, invert);
}
template <typename T>
cudaError_t launch_axpy_from(double* x, const T* e, long n, const double* scale, cudaStream_t s) {
  return launch_k(k_axpy_from<T>, dim3(blocks_for(n)), dim3(256), 0, s, x, e, n, scale);
}
cudaError_t launch_nyquist_coef(const void* r, int is_double, int nrows, int Nx, int logNx, void* rho,
                                cudaStream_t s) {
  (void)logNx;
  const int threads = 256;
  const int blocks = (nrows * 32 + threads - 1) / threads;
  if (is_double)
    return launch_k(k_nyquist_coef_d, dim3(blocks), dim3(threads), 0, s, (const double*)r, nrows, Nx, (double*)rho);
  return launch_k(k_nyquist_coef_f, dim3(blocks), dim3(threads), 0, s, (const float*)r, nrows, Nx, (float*)rho);
}
cudaError_t launch_gmres_init(double* st, const double* partial, int nblk, int m, double bnorm,
                              double tol, cudaStream_t s) {
  return launch_k(k_gmres_init, dim3(1), dim3(32), 0, s, st, partial, nblk, m, bnorm, tol);
}
cudaError_t launch_gmres_solve_y(double* st, int k, int m, cudaStream_t s) {
  return launch_k(k_gmres_solve_y, dim3(1), dim3(32), 0, s, st, k, m);
}

template <typename T>
cudaError_t launch_dots_sum(const T* w, const T* V, long ldv, int nvec, long n, double* partial, int nblk,
                            int with_norm, double* out, unsigned* ticket, cudaStream_t s) {
#define WT_C(NV) launch_k(k_dots_sum<T, NV>, dim3(nblk), dim3(256), 0, s, w, V, ldv, nvec, n, partial, with_norm, \
                          out, ticket)
  return WT_NV_DISPATCH(nvec, WT_C);
#undef WT_C
}
template <typename T>
cudaError_t launch_update_dots_arnoldi(T* w, const T* V, long ldv, int nvec, long n, double* st,
                                       double* partial, int nblk, int j, int m, unsigned* ticket,
                                       cudaStream_t s) {
#define WT_C(NV) launch_k(k_update_dots_arnoldi<T, NV>, dim3(nblk), dim3(256), 0, s, w, V, ldv, nvec, n, st, \
                          partial, j, m, ticket)
  return WT_NV1_DISPATCH(nvec, WT_C);
#undef WT_C
}

#define WT_KINST(T)                                                                                  \
  template cudaError_t launch_dots<T>(const T*, const T*, long, int, long, double*, int, int,         \
                                      cudaStream_t);                                                 \
  template cudaError_t launch_update_normalize<T>(const T*, const T*, long, int, long, const double*, \
                                                  const double*, T*, float*, cudaStream_t);          \
  template cudaError_t launch_lincomb<T>(T*, const T*, long, int, long, const double*, cudaStream_t); \
  template cudaError_t launch_axpy_from<T>(double*, const T*, long, const double*, cudaStream_t);     \
  template cudaError_t launch_dots_sum<T>(const T*, const T*, long, int, long, double*, int, int,      \
                                          double*, unsigned*, cudaStream_t);                          \
  template cudaError_t launch_update_dots_arnoldi<T>(T*, const T*, long, int, long, double*, double*, \
                                                     int, int, int, unsigned*, cudaStream_t);
WT_KINST(float)
WT_KINST(double)
template cudaError_t launch_convert<double, float>(const double*, float*, long, const double*, int,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long, const double*, int,
                                                   cudaStream_t);

}  // namespace wt
