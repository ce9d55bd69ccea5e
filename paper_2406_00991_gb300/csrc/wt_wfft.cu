// Spectral x- and y-derivative and filter passes with one warp per pair of
// real lines, the transform held in registers (paper Sec. 3.5: D f =
// F^{-1}(i kappa F f), the Nyquist coefficient multiplied by 0; Sec. 3.6: the
// exponential cut-off filter F^{-1}(F_S F f)).  For passes over many lines (the
// 3D levels) the CTA-per-line Stockham passes of wt_fft.cu spend most of
// their instructions on idle threads, barriers and shared-memory index
// arithmetic; here a warp transforms two real lines packed as one complex
// sequence z = r0 + i r1 of length N = 32 R, lane l holding z[l + 32 q] in
// slot q, by the four-step factorisation N = R x 32:
//   1. an R-point DFT over the slots in registers (radix-2, decimation in
//      frequency: slot q then holds frequency brev_R(q)),
//   2. the twiddle W_N^(l k2),
//   3. a 32-point DFT across the lanes per slot by __shfl_xor_sync butterflies
//      (decimation in frequency: lane l then holds k1 = brev_32(l)),
// so lane l, slot q holds Z[k2 + R k1]; the derivative multiplies it by
// i kappa(k) (the filter by its real response at |k|); the inverse runs the
// three steps backwards (decimation in time from the bit-reversed orders,
// conjugate twiddles), leaving N z' in natural order.  Both operators are
// real, so the real and imaginary parts of z' are the two lines' results.
// x-rows are loaded and stored coalesced (lane-consecutive); y-lines go
// through a shared-memory tile of 16 x-columns per CTA (one column pair per
// warp).  FP32 data are transformed in FP32; FP64 data (option df64) in
// double-float arithmetic (wt_ff.cuh).
#include "wt_dev.cuh"
#include "wt_ff.cuh"

#include <algorithm>

namespace wt {

namespace {

template <int R>
struct Log2 {
  static constexpr int value = 1 + Log2<R / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

template <int R>
__host__ __device__ constexpr int brev_const(int q) {
  int r = 0;
  for (int b = 0; b < Log2<R>::value; ++b) r |= ((q >> b) & 1) << (Log2<R>::value - 1 - b);
  return r;
}

// W_N^e = exp(-2 pi i e / N) for any e, from the staged half table tws (t < N/2)
template <typename T>
__device__ __forceinline__ c2_t<T> wN(const c2_t<T>* tws, int e, int N) {
  e &= N - 1;
  const int H = N >> 1;
  if (e < H) return tws[e];
  const c2_t<T> w = tws[e - H];
  return mk<T>(-w.x, -w.y);
}

template <typename T>
__device__ __forceinline__ c2_t<T> cconj(c2_t<T> a) { return mk<T>(a.x, -a.y); }

template <typename T>
__device__ __forceinline__ c2_t<T> shfl_xor_c(c2_t<T> v, int m) {
  return mk<T>(shfl_xor_a(v.x, m), shfl_xor_a(v.y, m));
}

// Forward transform of the warp's sequence (see the file comment).
template <typename T, int R>
__device__ __forceinline__ void warp_fft_forward(c2_t<T> (&x)[R], const c2_t<T>* tws, int N, int lane) {
  using c2 = c2_t<T>;
  // 1. R-point DIF over the slots
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * s) {
#pragma unroll
      for (int j = 0; j < s; ++j) {
        const c2 a = x[blk + j], b = x[blk + j + s];
        x[blk + j] = mk<T>(a.x + b.x, a.y + b.y);
        const c2 d = mk<T>(a.x - b.x, a.y - b.y);
        x[blk + j + s] = j == 0 ? d : cmul<T>(d, wN<T>(tws, j * (N / (2 * s)), N));
      }
    }
  }
  // 2. twiddle W_N^(lane k2), k2 = brev_R(q)
#pragma unroll
  for (int q = 1; q < R; ++q) x[q] = cmul<T>(x[q], wN<T>(tws, lane * brev_const<R>(q), N));
  // 3. 32-point DIF across the lanes
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const int j = lane & (2 * h - 1);
    const bool lo = j < h;
    const c2 w = wN<T>(tws, (lo ? 0 : j - h) * (N / (2 * h)), N);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const c2 v = x[q];
      const c2 p = shfl_xor_c<T>(v, h);
      x[q] = lo ? mk<T>(v.x + p.x, v.y + p.y) : cmul<T>(mk<T>(p.x - v.x, p.y - v.y), w);
    }
  }
}

// Inverse of warp_fft_forward (unnormalised: N times the sequence).
template <typename T, int R>
__device__ __forceinline__ void warp_fft_inverse(c2_t<T> (&x)[R], const c2_t<T>* tws, int N, int lane) {
  using c2 = c2_t<T>;
  // 3'. 32-point DIT across the lanes, bit-reversed lanes to natural
#pragma unroll
  for (int h = 1; h <= 16; h <<= 1) {
    const int j = lane & (2 * h - 1);
    const bool lo = j < h;
    const c2 w = cconj<T>(wN<T>(tws, (lo ? 0 : j - h) * (N / (2 * h)), N));
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const c2 t = lo ? x[q] : cmul<T>(x[q], w);
      const c2 p = shfl_xor_c<T>(t, h);
      x[q] = lo ? mk<T>(t.x + p.x, t.y + p.y) : mk<T>(p.x - t.x, p.y - t.y);
    }
  }
  // 2'. conjugate twiddle
#pragma unroll
  for (int q = 1; q < R; ++q) x[q] = cmul<T>(x[q], cconj<T>(wN<T>(tws, lane * brev_const<R>(q), N)));
  // 1'. R-point DIT over the slots, bit-reversed slots to natural
#pragma unroll
  for (int s = 1; s < R; s <<= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * s) {
#pragma unroll
      for (int j = 0; j < s; ++j) {
        const c2 a = x[blk + j];
        const c2 b = j == 0 ? x[blk + j + s] : cmul<T>(x[blk + j + s], cconj<T>(wN<T>(tws, j * (N / (2 * s)), N)));
        x[blk + j] = mk<T>(a.x + b.x, a.y + b.y);
        x[blk + j + s] = mk<T>(a.x - b.x, a.y - b.y);
      }
    }
  }
}

// D in the spectrum: Z[k] *= i kappa_k * s, kappa_k = kscale * signed k, 0 at N/2.
template <typename T, int R>
__device__ __forceinline__ void warp_deriv(c2_t<T> (&x)[R], int N, int lane, T kscale, T s) {
  const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int k = brev_const<R>(q) + R * k1;
    const int sk = k < N / 2 ? k : k - N;
    const T kap = (k == N / 2) ? a_zero<T>() : kscale * a_int<T>(sk) * s;
    x[q] = mk<T>(-kap * x[q].y, kap * x[q].x);
  }
}

// The exponential filter in the spectrum: Z[k] *= s filt[|signed k|] (the
// table in the storage type T, read through the read-only path).
template <typename T, typename A, int R>
__device__ __forceinline__ void warp_filter(c2_t<A> (&x)[R], int N, int lane, const T* __restrict__ filt, A s) {
  const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int k = brev_const<R>(q) + R * k1;
    const int an = k <= N / 2 ? k : N - k;
    const A f = to_arith<A, T>(__ldg(filt + an)) * s;
    x[q] = mk<A>(f * x[q].x, f * x[q].y);
  }
}

template <typename T>
__device__ __forceinline__ T epilogue(const RowPass<T>& a, long o, T v) {
  if (a.epi == EPI_ADD) return a.add[o] + v;
  if (a.epi == EPI_RESID) return a.rhs[o] - (a.add[o] + v);
  return v;
}

// The half twiddle table of an N-point transform in the arithmetic type A.
template <typename T, typename A>
__device__ __forceinline__ void stage_tw(c2_t<A>* tws, const RowPass<T>& a, int N, int logN) {
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
    const c2_t<T> w = a.tw[t << (a.logNtw - logN)];
    tws[t] = mk<A>(to_arith<A, T>(w.x), to_arith<A, T>(w.y));
  }
}

}  // namespace

// x-rows: rows r (of a [rows][N] array), row m = r / Ny for the boundary
// rows.  T: the storage type; A: the arithmetic type of the transform (T
// itself for FP32, double-float for FP64 data).
template <typename T, typename A, int R>
__global__ void __launch_bounds__(256) k_xderiv_warp(RowPass<T> a) {
  pdl_enter();
  using c2 = c2_t<A>;
  extern __shared__ __align__(16) unsigned char smraw[];
  c2* tws = reinterpret_cast<c2*>(smraw);
  const int N = 32 * R;
  stage_tw<T, A>(tws, a, N, a.logNin);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long pair = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long r0 = 2 * pair, r1 = r0 + 1;
  if (r0 >= a.nrows) return;                 // whole warp (no block-level barrier follows)
  const bool has1 = r1 < a.nrows;
  c2 x[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = lane + 32 * q;
    x[q] = mk<A>(to_arith<A, T>(a.in[r0 * N + j]), has1 ? to_arith<A, T>(a.in[r1 * N + j]) : a_zero<A>());
  }
  warp_fft_forward<A, R>(x, tws, N, lane);
  if (a.op == XOP_FILTER)
    warp_filter<T, A, R>(x, N, lane, a.filt, to_arith<A, T>(a.scale / T(N)));
  else
    warp_deriv<A, R>(x, N, lane, to_arith<A, T>(a.kscale), to_arith<A, T>(a.scale / T(N)));
  warp_fft_inverse<A, R>(x, tws, N, lane);
  const bool z0 = a.skip_bc && ((r0 / a.Ny) == 0 || (r0 / a.Ny) == a.M1 - 1);
  const bool z1 = a.skip_bc && ((r1 / a.Ny) == 0 || (r1 / a.Ny) == a.M1 - 1);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = lane + 32 * q;
    const long o0 = r0 * N + j;
    a.out[o0] = epilogue<T>(a, o0, z0 ? T(0) : from_arith<T, A>(x[q].x));
    if (has1) {
      const long o1 = r1 * N + j;
      a.out[o1] = epilogue<T>(a, o1, z1 ? T(0) : from_arith<T, A>(x[q].y));
    }
  }
}

// y-lines of a [planes][N][Nxl] array: CTA (blockIdx.x, blockIdx.y) takes
// columns 16 blockIdx.x .. + 15 of plane blockIdx.y through a shared tile
// [N][17]; warp w transforms columns 2w and 2w + 1.
template <typename T, typename A, int R>
__global__ void __launch_bounds__(256) k_yderiv_warp(RowPass<T> a) {
  pdl_enter();
  using c2 = c2_t<A>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = 32 * R;
  c2* tws = reinterpret_cast<c2*>(smraw);
  T* tile = reinterpret_cast<T*>(tws + N / 2);          // [N][17]
  stage_tw<T, A>(tws, a, N, a.logNin);
  const int plane = blockIdx.y, jx0 = blockIdx.x * 16, Nxl = a.Nxl;
  const long base = (long)plane * N * Nxl;
  for (int i = threadIdx.x; i < N * 16; i += blockDim.x) {
    const int j = i >> 4, c = i & 15;
    tile[j * 17 + c] = (jx0 + c < Nxl) ? a.in[base + (long)j * Nxl + jx0 + c] : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < 8) {
    c2 x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int j = lane + 32 * q;
      x[q] = mk<A>(to_arith<A, T>(tile[j * 17 + 2 * w]), to_arith<A, T>(tile[j * 17 + 2 * w + 1]));
    }
    warp_fft_forward<A, R>(x, tws, N, lane);
    if (a.op == XOP_FILTER)
      warp_filter<T, A, R>(x, N, lane, a.filt, to_arith<A, T>(a.scale / T(N)));
    else
      warp_deriv<A, R>(x, N, lane, to_arith<A, T>(a.kscale), to_arith<A, T>(a.scale / T(N)));
    warp_fft_inverse<A, R>(x, tws, N, lane);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int j = lane + 32 * q;
      tile[j * 17 + 2 * w] = from_arith<T, A>(x[q].x);
      tile[j * 17 + 2 * w + 1] = from_arith<T, A>(x[q].y);
    }
  }
  __syncthreads();
  const bool zero = a.skip_bc && (plane == 0 || plane == a.M1 - 1);
  for (int i = threadIdx.x; i < N * 16; i += blockDim.x) {
    const int j = i >> 4, c = i & 15;
    if (jx0 + c >= Nxl) continue;
    const long o = base + (long)j * Nxl + jx0 + c;
    a.out[o] = epilogue<T>(a, o, zero ? T(0) : tile[j * 17 + c]);
  }
}

// Whether the warp passes take this row pass: a derivative or the filter with equal in/out
// lengths of 32..1024 points (FP32) or 32..256 points (FP64 data, option
// df64: double-float arithmetic), a plain epilogue (store, add or residual),
// no Nyquist coefficient and no second transform, and enough lines to fill
// the GPU (x-rows: >= 512; y-lines: >= 16 x-columns).
template <typename T>
bool warp_deriv_fits(const RowPass<T>& a) {
  // FP64 in FP64 arithmetic is bound by the FP64 rate: the register-resident
  // form (up to 186 registers a thread) measured slower than the CTA-per-line
  // passes (FP64 operator apply on 256 x 256 x 16: 692 against 599 us), so
  // FP64 data take the warp passes only in double-float
  const int maxN = sizeof(T) == 4 ? 1024 : 256;
  if (sizeof(T) != 4 && !a.df) return false;
  if (!(a.op == XOP_DERIV || (a.op == XOP_FILTER && a.filt))) return false;
  if (a.Nin != a.Nout || a.Nin < 32 || a.Nin > maxN) return false;
  if (a.nyq || a.out2 || !a.write_out) return false;
  if (a.epi != EPI_STORE && a.epi != EPI_ADD && a.epi != EPI_RESID) return false;
  if (a.ylines) return a.Nxl >= 16 && a.nrows >= 32 * 16;
  return a.nrows >= 512;
}

template <typename T, typename A, int R>
static cudaError_t launch_r(const RowPass<T>& a, cudaStream_t s) {
  const int N = 32 * R;
  cudaError_t e;
  if (a.ylines) {
    const size_t smem = (size_t)(N / 2) * sizeof(c2_t<A>) + (size_t)N * 17 * sizeof(T);
    if ((e = ensure_dyn_smem((const void*)k_yderiv_warp<T, A, R>, smem)) != cudaSuccess) return e;
    const int planes = a.nrows / a.Nxl;
    const dim3 grid((a.Nxl + 15) / 16, planes);
    return launch_k(k_yderiv_warp<T, A, R>, grid, dim3(256), smem, s, a);
  } else {
    const size_t smem = (size_t)(N / 2) * sizeof(c2_t<A>);
    const long pairs = ((long)a.nrows + 1) / 2;
    return launch_k(k_xderiv_warp<T, A, R>, dim3((unsigned)((pairs + 7) / 8)), dim3(256), smem, s, a);
  }
}

template <typename T>
cudaError_t launch_deriv_warp(const RowPass<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    switch (a.Nin) {
      case 32: return launch_r<T, ff, 1>(a, s);
      case 64: return launch_r<T, ff, 2>(a, s);
      case 128: return launch_r<T, ff, 4>(a, s);
      case 256: return launch_r<T, ff, 8>(a, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (a.Nin) {
      case 32: return launch_r<T, T, 1>(a, s);
      case 64: return launch_r<T, T, 2>(a, s);
      case 128: return launch_r<T, T, 4>(a, s);
      case 256: return launch_r<T, T, 8>(a, s);
      case 512: return launch_r<T, T, 16>(a, s);
      case 1024: return launch_r<T, T, 32>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

template bool warp_deriv_fits<float>(const RowPass<float>&);
template bool warp_deriv_fits<double>(const RowPass<double>&);
template cudaError_t launch_deriv_warp<float>(const RowPass<float>&, cudaStream_t);
template cudaError_t launch_deriv_warp<double>(const RowPass<double>&, cudaStream_t);

}  // namespace wt
