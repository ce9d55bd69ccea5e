// Spectral passes along x-rows and y-lines (paper Sec. 3.5 and 4.2):
//   derivative   D f = F^{-1}( i kappa F f ), Nyquist coefficient multiplied by 0
//   resampling   Fourier truncation (restriction) / zero padding (prolongation)
//   filter       exponential cut-off on |n| (Sec. 3.6)
// followed by a fused epilogue (store / add / residual / accumulate) and an
// optional per-row Nyquist coefficient (used by the Nyquist-split smoother).
//
// Design: one CTA transforms `nb` pairs of real rows in shared memory; the
// two real rows of a pair are packed as real and imaginary part of one
// complex sequence.  Every operation above is a real linear map (its
// multiplier is Hermitian), so the real and imaginary parts of the result are
// the results for the two rows.  The transform is a radix-4 (plus one
// radix-2 stage for odd log2 N) Stockham self-sorting FFT with host-computed
// FP64 twiddles staged in shared memory.
#include "wt_dev.cuh"
#include "wt_ff.cuh"

#include <algorithm>

namespace wt {

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass(RowPass<T> a, int ppc) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  rowpass_body<T>(a, ppc, blockIdx.x, gridDim.x, smraw);
}

// Single real rows through a half-length complex FFT, one row per CTA: half
// the transform length and twice the CTAs of the row-pair pass (measured
// faster in FP32 and FP64; FP64 gains most, its per-SM rate makes the
// row-pair transform the long pole).  For a real row x of length N, H = N/2:
//   z_k = x_2k + i x_2k+1,  Z = DFT_H(z),
//   X_m = E_m + W^m O_m, E_m = (Z_m + conj Z_{H-m}) / 2, O_m = (Z_m - conj Z_{H-m}) / 2i,
//   X_H = E_0 - O_0,  W = exp(-2 pi i / N)      (m = 0..H: the Hermitian half);
// the spectral operation maps X (length Nin) to Y (length Nout, m = 0..Hout);
// then with H = Hout, W = exp(-2 pi i / Nout)
//   C_m = (Y_m + conj Y_{H-m}) + i W^-m (Y_m - conj Y_{H-m})   (Y_{H-0} = Y_H),
//   IDFT_H(C)_k = y_2k + i y_2k+1  (times Nin, removed by the epilogue scale).
// T: the arithmetic type (the storage type S only for the filter table).
template <typename T, typename S>
__device__ c2_t<T>* real_spectral(c2_t<T>* A, c2_t<T>* B, int logNin, int logNout, int op, T kscale,
                                  const S* filt, const c2_t<T>* tws, int logNt) {
  using c2 = c2_t<T>;
  const int Hin = 1 << (logNin - 1), Hout = 1 << (logNout - 1);
  const int keep = (Hin < Hout ? Hin : Hout) * 2;          // resample: keep |m| < keep / 2
  const int sin = logNt - logNin, sout = logNt - logNout;
  c2* Z = fft_smem<T>(A, B, logNin - 1, 1, 0, tws, logNt, false);
  c2* Y = (Z == A) ? B : A;
  for (int m = threadIdx.x; m <= Hout; m += blockDim.x) {
    c2 X = mk<T>(a_zero<T>(), a_zero<T>());
    if (m < Hin) {
      const c2 zm = Z[m], zc0 = Z[(Hin - m) & (Hin - 1)];
      const c2 E = mk<T>(a_half<T>() * (zm.x + zc0.x), a_half<T>() * (zm.y - zc0.y));
      const c2 Om = mk<T>(a_half<T>() * (zm.y + zc0.y), -(a_half<T>() * (zm.x - zc0.x)));   // (zm - conj zc) / 2i
      const c2 WO = cmul<T>(tws[m << sin], Om);
      X = mk<T>(E.x + WO.x, E.y + WO.y);
    } else if (m == Hin) {
      const c2 z0 = Z[0];
      X = mk<T>(z0.x - z0.y, a_zero<T>());                   // E_0 - O_0 (real)
    }
    c2 v = mk<T>(a_zero<T>(), a_zero<T>());
    if (op == XOP_DERIV || op == XOP_RESAMPLE_DERIV) {
      if (m < Hout && 2 * m < keep) {
        const T kap = kscale * a_int<T>(m);
        v = mk<T>(-kap * X.y, kap * X.x);
      }
    } else if (op == XOP_RESAMPLE) {
      if (2 * m < keep) v = X;
    } else if (op == XOP_FILTER) {
      const T f = to_arith<T, S>(filt[m]);
      v = mk<T>(f * X.x, f * X.y);
    } else {
      v = X;                                                // XOP_NONE
    }
    Y[m] = v;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < Hout; m += blockDim.x) {
    const c2 ym = Y[m];
    const c2 yh = Y[Hout - m];                              // m = 0: the Nyquist term
    const c2 yc = mk<T>(yh.x, -yh.y);
    const c2 sum = mk<T>(ym.x + yc.x, ym.y + yc.y);
    const c2 dif = mk<T>(ym.x - yc.x, ym.y - yc.y);
    const c2 w = tws[m << sout];
    const c2 t = cmul<T>(mk<T>(w.x, -w.y), dif);              // W^-m (Y_m - conj Y_{H-m})
    Z[m] = mk<T>(sum.x - t.y, sum.y + t.x);
  }
  __syncthreads();
  return fft_smem<T>(Z, Y, logNout - 1, 1, 0, tws, logNt, true);
}

// One real x-row per CTA: the spectral operation of the pass, its epilogue
// (store / add / residual / accumulate, boundary rows, Nyquist coefficient)
// and the optional second transform of the result into out2.  T: the
// storage type; A: the arithmetic type of the transforms (T itself, or
// double-float for FP64 data); epilogue in T.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_rowpass_real(RowPass<T> a) {
  pdl_enter();
  using c2 = c2_t<A>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Nin = a.Nin, Nout = a.Nout;
  const int logNt = a.Nin > a.Nout ? a.logNin : a.logNout;
  const int Nt = 1 << logNt;
  const int Hb = Nt / 2 + 1;
  c2* P = reinterpret_cast<c2*>(smraw);
  c2* Q = P + Hb;
  c2* tws = Q + Hb;                                         // exp(-2 pi i t / Nt), t < Nt/2
  for (int t = threadIdx.x; t < Nt / 2; t += blockDim.x) {
    const c2_t<T> w = a.tw[t << (a.logNtw - logNt)];
    tws[t] = mk<A>(to_arith<A, T>(w.x), to_arith<A, T>(w.y));
  }
  const int r = blockIdx.x;
  const int Hin = Nin >> 1, Hout = Nout >> 1;
  const T* in = a.in + (long)r * Nin;
  for (int k = threadIdx.x; k < Hin; k += blockDim.x) P[k] = mk<A>(to_arith<A, T>(in[2 * k]), to_arith<A, T>(in[2 * k + 1]));
  __syncthreads();
  c2* R = real_spectral<A, T>(P, Q, a.logNin, a.logNout, a.op, to_arith<A, T>(a.kscale), a.filt, tws, logNt);
  const T sc = a.scale / T(Nin);
  const bool bc = bc_row(a, r);
  T alt = T(0);                                  // sum of (-1)^n out_n for the Nyquist coefficient
  for (int k = threadIdx.x; k < Hout; k += blockDim.x) {
    const c2 y = R[k];
    T vv[2];
    for (int h = 0; h < 2; ++h) {
      const long o = (long)r * Nout + 2 * k + h;
      T v = from_arith<T, A>(h ? y.y : y.x) * sc;
      if (bc) v = T(0);
      if (a.epi == EPI_ADD) v += a.add[o];
      else if (a.epi == EPI_RESID) v = a.rhs[o] - (a.add[o] + v);
      else if (a.epi == EPI_ACC) v += a.out[o];
      if (a.write_out) a.out[o] = v;
      alt += h ? -v : v;
      vv[h] = v;
    }
    if (a.out2) R[k] = mk<A>(to_arith<A, T>(vv[0]), to_arith<A, T>(vv[1]));   // input of the second transform
  }
  if (a.nyq) {
    __shared__ T red[32];
    for (int o = 16; o > 0; o >>= 1) alt += __shfl_xor_sync(0xffffffffu, alt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = alt;
    __syncthreads();
    if (threadIdx.x == 0) {
      T s = T(0);
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
      a.nyq[r] = s / T(Nout);
    }
  }
  if (a.out2) {
    __syncthreads();
    c2* O = (R == P) ? Q : P;
    c2* R2 = real_spectral<A, T>(R, O, a.logNout, a.logNout2, a.op2, to_arith<A, T>(a.kscale), (const T*)nullptr, tws, logNt);
    const T s2 = T(1) / T(Nout);
    for (int k = threadIdx.x; k < (a.Nout2 >> 1); k += blockDim.x) {
      const c2 y = R2[k];
      a.out2[(long)r * a.Nout2 + 2 * k] = from_arith<T, A>(y.x) * s2;
      a.out2[(long)r * a.Nout2 + 2 * k + 1] = from_arith<T, A>(y.y) * s2;
    }
  }
}

template <typename T>
cudaError_t launch_rowpass(const RowPass<T>& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  if (a.warp && warp_deriv_fits(a)) return launch_deriv_warp(a, s);
  if (!a.ylines && a.Nin >= 8 && a.Nout >= 8 && (!a.out2 || (a.Nout2 >= 8 && a.Nout2 <= a.Nout))) {
    const int Nt = std::max(a.Nin, a.Nout);
    const size_t smem = (size_t)(2 * (Nt / 2 + 1) + Nt / 2) * sizeof(c2_t<T>);
    // (the kernel's 32-word static reduction buffer counts against the
    // default 48 KB as well)
    if constexpr (sizeof(T) == 8) {
      if (a.df >= 2) {
        // FP64 rows in double-float (the same shared-memory footprint)
        if (smem > 32 * 1024) {
          cudaError_t e = ensure_dyn_smem((const void*)k_rowpass_real<T, ff>, smem);
          if (e != cudaSuccess) return e;
        }
        return launch_k(k_rowpass_real<T, ff>, dim3(a.nrows), dim3(256), smem, s, a);
      }
    }
    if (smem > 32 * 1024) {
      cudaError_t e = ensure_dyn_smem((const void*)k_rowpass_real<T, T>, smem);
      if (e != cudaSuccess) return e;
    }
    return launch_k(k_rowpass_real<T, T>, dim3(a.nrows), dim3(256), smem, s, a);
  }
  const int Nmax = std::max(a.Nin, a.Nout);
  const int npairs = (a.nrows + 1) / 2;
  int ppc = std::max(1, 1024 / Nmax);
  const int want = (npairs + 303) / 304;     // spread small passes over the SMs
  ppc = std::max(1, std::min(ppc, want));
  const size_t smem = rowpass_smem(a, ppc);
  if (smem > 32 * 1024) {
    cudaError_t e = ensure_dyn_smem((const void*)k_rowpass<T>, smem);
    if (e != cudaSuccess) return e;
  }
  int grid = (npairs + ppc - 1) / ppc;
  grid = std::min(grid, sm_count() * 16);
  return launch_k(k_rowpass<T>, dim3(grid), dim3(256), smem, s, a, ppc);
}

template cudaError_t launch_rowpass<float>(const RowPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass<double>(const RowPass<double>&, cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass_multi(const __grid_constant__ MultiPass<T> m) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  int i = 0;
  while (i + 1 < m.n && (int)blockIdx.x >= m.start[i + 1]) ++i;
  const int u = blockIdx.x - m.start[i];
  rowpass_body<T>(m.d[i], 1, u, m.start[i + 1] - m.start[i], smraw);
}

template <typename T>
cudaError_t launch_rowpass_multi(const MultiPass<T>& m0, cudaStream_t s) {
  if (m0.n <= 0) return cudaSuccess;
  if (m0.n > kMaxPasses) return cudaErrorInvalidValue;
  MultiPass<T> m = m0;
  size_t smem = 0;
  m.start[0] = 0;
  for (int i = 0; i < m.n; ++i) {
    const int npairs = (m.d[i].nrows + 1) / 2;
    m.start[i + 1] = m.start[i] + npairs;
    smem = std::max(smem, rowpass_smem(m.d[i], 1));
  }
  if (smem > 32 * 1024) {
    cudaError_t e = ensure_dyn_smem((const void*)k_rowpass_multi<T>, smem);
    if (e != cudaSuccess) return e;
  }
  if (m.start[m.n] <= 0) return cudaSuccess;
  return launch_k(k_rowpass_multi<T>, dim3(m.start[m.n]), dim3(256), smem, s, m);
}

template cudaError_t launch_rowpass_multi<float>(const MultiPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass_multi<double>(const MultiPass<double>&, cudaStream_t);

}  // namespace wt
