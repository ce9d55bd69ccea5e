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

#include <algorithm>

namespace wt {

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass(RowPass<T> a, int ppc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  rowpass_body<T>(a, ppc, blockIdx.x, gridDim.x, smraw);
}

// x-derivative of single real rows through a half-length complex FFT, one
// row per CTA: half the transform length and twice the CTAs of the row-pair
// pass (measured faster in FP32 and FP64; FP64 gains most, its per-SM rate
// makes the row-pair transform the long pole): with H = N/2,
//   z_k = x_2k + i x_2k+1,  Z = DFT_H(z),
//   X_m = E_m + W^m O_m, E_m = (Z_m + conj Z_{H-m}) / 2, O_m = (Z_m - conj Z_{H-m}) / 2i,
//   Y_m = i kappa_m X_m (m < H; the Nyquist coefficient Y_H = 0),
//   C_m = (Y_m + conj Y_{H-m}) + i W^-m (Y_m - conj Y_{H-m}),  W = exp(-2 pi i / N),
//   IDFT_H(C)_k / N = y_2k + i y_2k+1,
// then the store / add / residual / accumulate epilogue of the general pass
// and, when asked, the output row's Nyquist coefficient.
template <typename T>
__global__ void __launch_bounds__(256) k_rowpass_real(RowPass<T> a) {
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.Nin, logN = a.logNin, H = N >> 1;
  c2* z = reinterpret_cast<c2*>(smraw);
  c2* w = z + H;
  c2* tws = w + H;                                  // exp(-2 pi i t / N), t < N/2
  for (int t = threadIdx.x; t < H; t += blockDim.x) tws[t] = a.tw[t << (a.logNtw - logN)];
  const int r = blockIdx.x;
  const T* in = a.in + (long)r * N;
  for (int k = threadIdx.x; k < H; k += blockDim.x) z[k] = mk<T>(in[2 * k], in[2 * k + 1]);
  __syncthreads();
  c2* Z = fft_smem<T>(z, w, logN - 1, 1, H, tws, logN, false);
  c2* Yb = (Z == z) ? w : z;
  for (int m = threadIdx.x; m < H; m += blockDim.x) {
    const c2 zm = Z[m], zc0 = Z[(H - m) & (H - 1)];
    const c2 zc = mk<T>(zc0.x, -zc0.y);
    const c2 E = mk<T>(T(0.5) * (zm.x + zc.x), T(0.5) * (zm.y + zc.y));
    const c2 Om = mk<T>(T(0.5) * (zm.y - zc.y), -T(0.5) * (zm.x - zc.x));   // (zm - zc) / 2i
    const c2 X = mk<T>(E.x, E.y);
    const c2 WO = cmul<T>(tws[m], Om);
    const T kap = a.kscale * T(m);
    // Y_m = i kappa (E + W^m O)
    Yb[m] = mk<T>(-kap * (X.y + WO.y), kap * (X.x + WO.x));
  }
  __syncthreads();
  for (int m = threadIdx.x; m < H; m += blockDim.x) {
    const c2 ym = Yb[m];
    const c2 yh = m == 0 ? mk<T>(T(0), T(0)) : Yb[H - m];          // Y_H = 0
    const c2 yc = mk<T>(yh.x, -yh.y);
    const c2 sum = mk<T>(ym.x + yc.x, ym.y + yc.y);
    const c2 dif = mk<T>(ym.x - yc.x, ym.y - yc.y);
    const c2 wm = mk<T>(tws[m].x, -tws[m].y);                        // W^-m
    const c2 t = cmul<T>(wm, dif);
    Z[m] = mk<T>(sum.x - t.y, sum.y + t.x);                          // sum + i t
  }
  __syncthreads();
  c2* R = fft_smem<T>(Z, Yb, logN - 1, 1, H, tws, logN, true);
  const T sc = a.scale / T(N);
  T alt = T(0);                                  // sum of (-1)^n out_n for the Nyquist coefficient
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    const c2 y = R[k];
    for (int h = 0; h < 2; ++h) {
      const long o = (long)r * N + 2 * k + h;
      T v = (h ? y.y : y.x) * sc;
      if (bc_row(a, r)) v = T(0);
      if (a.epi == EPI_ADD) v += a.add[o];
      else if (a.epi == EPI_RESID) v = a.rhs[o] - (a.add[o] + v);
      else if (a.epi == EPI_ACC) v += a.out[o];
      a.out[o] = v;
      alt += h ? -v : v;
    }
  }
  if (a.nyq) {
    __shared__ T red[32];
    for (int o = 16; o > 0; o >>= 1) alt += __shfl_xor_sync(0xffffffffu, alt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = alt;
    __syncthreads();
    if (threadIdx.x == 0) {
      T s = T(0);
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
      a.nyq[r] = s / T(N);
    }
  }
}

template <typename T>
cudaError_t launch_rowpass(const RowPass<T>& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  if (a.op == XOP_DERIV && a.Nin == a.Nout && a.Nin >= 8 && !a.ylines && !a.out2) {
    const size_t smem = (size_t)(3 * (a.Nin / 2)) * sizeof(c2_t<T>);
    // (the kernel's 32-word static reduction buffer counts against the
    // default 48 KB as well)
    if (smem > 32 * 1024) {
      cudaError_t e = ensure_dyn_smem((const void*)k_rowpass_real<T>, smem);
      if (e != cudaSuccess) return e;
    }
    return launch_k(k_rowpass_real<T>, dim3(a.nrows), dim3(256), smem, s, a);
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
  grid = std::min(grid, 152 * 16);
  return launch_k(k_rowpass<T>, dim3(grid), dim3(256), smem, s, a, ppc);
}

template cudaError_t launch_rowpass<float>(const RowPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass<double>(const RowPass<double>&, cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256) k_rowpass_multi(const __grid_constant__ MultiPass<T> m) {
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
  k_rowpass_multi<T><<<m.start[m.n], 256, smem, s>>>(m);
  return cudaGetLastError();
}

template cudaError_t launch_rowpass_multi<float>(const MultiPass<float>&, cudaStream_t);
template cudaError_t launch_rowpass_multi<double>(const MultiPass<double>&, cudaStream_t);

}  // namespace wt
