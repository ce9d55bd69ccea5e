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
// the results for the two rows.  The transform is an iterative radix-2
// Stockham (self-sorting) FFT with host-computed FP64 twiddles.
#include "wt_internal.h"

#include <algorithm>

namespace wt {

template <typename T> __device__ __forceinline__ c2_t<T> mk(T re, T im);
template <> __device__ __forceinline__ float2 mk<float>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ double2 mk<double>(double re, double im) { return make_double2(re, im); }

// Radix-2 Stockham FFT of nb sequences of length N = 2^logN stored with stride
// S in `a`; `b` is workspace.  Returns the buffer holding the result.
template <typename T>
__device__ c2_t<T>* fft_smem(c2_t<T>* a, c2_t<T>* b, int logN, int nb, int S,
                             const c2_t<T>* __restrict__ tw, int logNtw, bool inverse) {
  using c2 = c2_t<T>;
  const int N = 1 << logN;
  const int half = N >> 1;
  const int total = nb << (logN - 1);
  const int tshift = logNtw - logN;
  for (int s = 0; s < logN; ++s) {
    const int m = 1 << s;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int q = idx >> (logN - 1);
      const int bf = idx & (half - 1);
      const int j = bf >> s;
      const int k = bf & (m - 1);
      const c2 c0 = a[q * S + k + j * m];
      const c2 c1 = a[q * S + k + j * m + half];
      c2 w = tw[(j * m) << tshift];
      if (inverse) w.y = -w.y;
      const T dre = c0.x - c1.x, dim = c0.y - c1.y;
      b[q * S + k + 2 * j * m] = mk<T>(c0.x + c1.x, c0.y + c1.y);
      b[q * S + k + 2 * j * m + m] = mk<T>(w.x * dre - w.y * dim, w.x * dim + w.y * dre);
    }
    __syncthreads();
    c2* t = a;
    a = b;
    b = t;
  }
  return a;
}

template <typename T>
__device__ __forceinline__ long row_offset(const RowPass<T>& a, int r, int j, int Nlen) {
  if (!a.ylines) return (long)r * Nlen + j;
  const int plane = r / a.Nxl, jx = r - plane * a.Nxl;
  return ((long)plane * Nlen + j) * a.Nxl + jx;
}

template <typename T>
__device__ __forceinline__ bool bc_row(const RowPass<T>& a, int r) {
  if (!a.skip_bc) return false;
  const int m = a.ylines ? r / a.Nxl : r / a.Ny;
  return m == 0 || m == a.M1 - 1;
}

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass(RowPass<T> a, int ppc) {
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Nmax = a.Nin > a.Nout ? a.Nin : a.Nout;
  const int S = Nmax + (a.ylines ? 1 : 0);
  c2* buf0 = reinterpret_cast<c2*>(smraw);
  c2* buf1 = buf0 + ppc * S;
  const int npairs = (a.nrows + 1) >> 1;
  const T inv_n = T(1) / T(a.Nin);

  for (int p0 = blockIdx.x * ppc; p0 < npairs; p0 += gridDim.x * ppc) {
    const int nb = min(ppc, npairs - p0);
    // ---- load two real rows per complex sequence
    for (int idx = threadIdx.x; idx < nb * a.Nin; idx += blockDim.x) {
      int q, j;
      if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNin; j = idx & (a.Nin - 1); }
      const int r0 = 2 * (p0 + q), r1 = r0 + 1;
      const T re = a.in[row_offset(a, r0, j, a.Nin)];
      const T im = r1 < a.nrows ? a.in[row_offset(a, r1, j, a.Nin)] : T(0);
      buf0[q * S + j] = mk<T>(re, im);
    }
    __syncthreads();
    c2* X = fft_smem<T>(buf0, buf1, a.logNin, nb, S, a.tw, a.logNtw, false);
    c2* Yb = (X == buf0) ? buf1 : buf0;
    // ---- spectral operation into Yb (length Nout)
    const int nkeep2 = (a.Nin < a.Nout ? a.Nin : a.Nout);   // keep |n| < nkeep2 / 2
    for (int idx = threadIdx.x; idx < nb * a.Nout; idx += blockDim.x) {
      const int q = idx >> a.logNout, n = idx & (a.Nout - 1);
      const int ns = n < a.Nout / 2 ? n : n - a.Nout;          // signed wavenumber index
      c2 v = mk<T>(T(0), T(0));
      if (a.op == XOP_DERIV) {
        const c2 x = X[q * S + n];
        const T kap = (n == a.Nout / 2) ? T(0) : a.kscale * T(ns);
        v = mk<T>(-kap * x.y, kap * x.x);
      } else if (a.op == XOP_RESAMPLE) {
        const int an = ns < 0 ? -ns : ns;
        if (2 * an < nkeep2) {
          const int nin = ns < 0 ? ns + a.Nin : ns;
          v = X[q * S + nin];
        }
      } else if (a.op == XOP_FILTER) {
        const c2 x = X[q * S + n];
        const int an = ns < 0 ? -ns : ns;
        const T f = a.filt[an];
        v = mk<T>(f * x.x, f * x.y);
      } else {
        v = X[q * S + n];
      }
      Yb[q * S + n] = v;
    }
    __syncthreads();
    c2* Y = fft_smem<T>(Yb, X, a.logNout, nb, S, a.tw, a.logNtw, true);
    // ---- epilogue
    const T sc = a.scale * inv_n;
    for (int idx = threadIdx.x; idx < nb * a.Nout; idx += blockDim.x) {
      int q, j;
      if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNout; j = idx & (a.Nout - 1); }
      const int r0 = 2 * (p0 + q), r1 = r0 + 1;
      c2 y = Y[q * S + j];
      T v0 = y.x * sc, v1 = y.y * sc;
      if (bc_row(a, r0)) v0 = T(0);
      if (r1 < a.nrows && bc_row(a, r1)) v1 = T(0);
      const long o0 = row_offset(a, r0, j, a.Nout);
      const long o1 = row_offset(a, r1, j, a.Nout);
      const bool has1 = r1 < a.nrows;
      if (a.epi == EPI_ADD) {
        v0 += a.add[o0];
        if (has1) v1 += a.add[o1];
      } else if (a.epi == EPI_RESID) {
        v0 = a.rhs[o0] - (a.add[o0] + v0);
        if (has1) v1 = a.rhs[o1] - (a.add[o1] + v1);
      } else if (a.epi == EPI_ACC) {
        v0 += a.out[o0];
        if (has1) v1 += a.out[o1];
      }
      a.out[o0] = v0;
      if (has1) a.out[o1] = v1;
      if (a.nyq) Y[q * S + j] = mk<T>(v0, has1 ? v1 : T(0));
    }
    if (a.nyq) {
      __syncthreads();
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int q = warp; q < nb; q += nw) {
        T s0 = 0, s1 = 0;
        for (int j = lane; j < a.Nout; j += 32) {
          const c2 y = Y[q * S + j];
          const T sg = (j & 1) ? T(-1) : T(1);
          s0 += sg * y.x;
          s1 += sg * y.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {
          const int r0 = 2 * (p0 + q), r1 = r0 + 1;
          a.nyq[r0] = s0 / T(a.Nout);
          if (r1 < a.nrows) a.nyq[r1] = s1 / T(a.Nout);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_rowpass(const RowPass<T>& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  const int Nmax = std::max(a.Nin, a.Nout);
  const int npairs = (a.nrows + 1) / 2;
  int ppc = std::max(1, 1024 / Nmax);
  const int want = (npairs + 303) / 304;     // spread small passes over the SMs
  ppc = std::max(1, std::min(ppc, want));
  const int S = Nmax + (a.ylines ? 1 : 0);
  const size_t smem = 2 * (size_t)ppc * S * sizeof(c2_t<T>);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_rowpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int grid = (npairs + ppc - 1) / ppc;
  grid = std::min(grid, 152 * 16);
  k_rowpass<T><<<grid, 256, smem, s>>>(a, ppc);
  return cudaGetLastError();
}

template cudaError_t launch_rowpass<float>(const RowPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass<double>(const RowPass<double>&, cudaStream_t);

}  // namespace wt
