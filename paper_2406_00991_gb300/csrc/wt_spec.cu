// Mean-depth spectral smoother: x <- x + omega_s S (f - A x), where S solves
// the flat reference problem (eta = 0, depth dref = min h) exactly, one
// horizontal Fourier mode at a time.  On the flat reference tank the operator
// A_{a,b} of Eq. poissonp separates: for the mode exp(i kappa . x) the column
// p(sigma) obeys
//   interior rows  D D p / dref^2 - kappa^2 p,
//   surface row    p_0                          (Eq. bcpd),
//   bottom row     (D p)_Nz / dref              (Eq. bcpdneu, n = (0, 0, 1)),
// with kappa^2 the discrete second-derivative symbol (0 along an axis at its
// Nyquist wavenumber, which D_x(D_x .) annihilates).  The host inverts that
// (Nz+1)^2 matrix once per distinct kappa^2 (wt_capi.cu); here:
//   k_spec_fwd_x  one real x-row per CTA -> its Hermitian half spectrum
//                 X_0..X_{N/2} (half-length complex FFT, then the split of the
//                 packed even / odd samples),
//   k_spec_y      (3D) complex FFT along y of the half spectrum, forward or
//                 inverse, several kx per CTA,
//   k_spec_cols   one warp per Fourier mode: the column times the mode's
//                 inverse (or its transpose, for the smoother of A^T),
//   k_spec_inv_x  the inverse of k_spec_fwd_x, with the epilogue
//                 x = s y (first sweep from x = 0) or x += s y.
// Every transform is unnormalised; s = omega_s / (Nx Ny).
#include "wt_dev.cuh"

#include <algorithm>

namespace wt {

// twiddles exp(-2 pi i t / N), t < N/2, of a length-N transform from the
// tank's table of length 2^logNtw >= N
template <typename T>
__device__ __forceinline__ void stage_twiddles(c2_t<T>* tws, const c2_t<T>* tw, int logN, int logNtw) {
  const int N = 1 << logN;
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) tws[t] = tw[t << (logNtw - logN)];
}

template <typename T>
__global__ void __launch_bounds__(256) k_spec_fwd_x(const T* __restrict__ in, c2_t<T>* __restrict__ out,
                                                    int logN, const c2_t<T>* __restrict__ tw, int logNtw) {
  pdl_enter();
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = 1 << logN, H = N >> 1;
  c2* P = reinterpret_cast<c2*>(smraw);
  c2* Q = P + H;
  c2* tws = Q + H;
  stage_twiddles<T>(tws, tw, logN, logNtw);
  const long r = blockIdx.x;
  const T* row = in + r * N;
  for (int k = threadIdx.x; k < H; k += blockDim.x) P[k] = mk<T>(row[2 * k], row[2 * k + 1]);
  __syncthreads();
  const c2* Z = fft_smem<T>(P, Q, logN - 1, 1, 0, tws, logN, false);
  c2* o = out + r * (H + 1);
  for (int m = threadIdx.x; m <= H; m += blockDim.x) {
    c2 X;
    if (m < H) {
      // even samples E_m = (Z_m + conj Z_{H-m}) / 2, odd O_m = (Z_m - conj Z_{H-m}) / 2i,
      // X_m = E_m + W^m O_m with W = exp(-2 pi i / N)
      const c2 zm = Z[m], zc = Z[(H - m) & (H - 1)];
      const c2 E = mk<T>(T(0.5) * (zm.x + zc.x), T(0.5) * (zm.y - zc.y));
      const c2 O = mk<T>(T(0.5) * (zm.y + zc.y), -T(0.5) * (zm.x - zc.x));
      const c2 WO = cmul<T>(tws[m], O);
      X = mk<T>(E.x + WO.x, E.y + WO.y);
    } else {
      const c2 z0 = Z[0];
      X = mk<T>(z0.x - z0.y, T(0));                       // X_{N/2} = E_0 - O_0, real
    }
    o[m] = X;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_spec_inv_x(const c2_t<T>* __restrict__ in, T* __restrict__ x,
                                                    int logN, T scale, int first,
                                                    const c2_t<T>* __restrict__ tw, int logNtw) {
  pdl_enter();
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = 1 << logN, H = N >> 1;
  c2* Y = reinterpret_cast<c2*>(smraw);          // H + 1 values
  c2* C = Y + (H + 1);                           // H values
  c2* Q = C + H;                                 // H values
  c2* tws = Q + H;
  stage_twiddles<T>(tws, tw, logN, logNtw);
  const long r = blockIdx.x;
  const c2* iy = in + r * (H + 1);
  for (int m = threadIdx.x; m <= H; m += blockDim.x) Y[m] = iy[m];
  __syncthreads();
  // C_m = (Y_m + conj Y_{H-m}) + i W^-m (Y_m - conj Y_{H-m}); its inverse
  // half-length transform is N (y_2k + i y_2k+1)
  for (int m = threadIdx.x; m < H; m += blockDim.x) {
    const c2 ym = Y[m], yh = Y[H - m];
    const c2 sum = mk<T>(ym.x + yh.x, ym.y - yh.y);
    const c2 dif = mk<T>(ym.x - yh.x, ym.y + yh.y);
    const c2 w = tws[m];
    const c2 t = cmul<T>(mk<T>(w.x, -w.y), dif);
    C[m] = mk<T>(sum.x - t.y, sum.y + t.x);
  }
  __syncthreads();
  const c2* R = fft_smem<T>(C, Q, logN - 1, 1, 0, tws, logN, true);
  T* row = x + r * N;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    const c2 v = R[k];
    if (first) {
      row[2 * k] = scale * v.x;
      row[2 * k + 1] = scale * v.y;
    } else {
      row[2 * k] += scale * v.x;
      row[2 * k + 1] += scale * v.y;
    }
  }
}

// Complex transforms along y of S[plane][jy][kx] (kx < Nh), tx consecutive
// kx per CTA (coalesced rows of tx complex values), in place.
template <typename T>
__global__ void __launch_bounds__(256) k_spec_y(c2_t<T>* __restrict__ S, int Ny, int logNy, int Nh, int tx,
                                                int inverse, const c2_t<T>* __restrict__ tw, int logNtw) {
  pdl_enter();
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  c2* A = reinterpret_cast<c2*>(smraw);          // tx sequences of Ny
  c2* B = A + tx * Ny;
  c2* tws = B + tx * Ny;
  stage_twiddles<T>(tws, tw, logNy, logNtw);
  const int kx0 = blockIdx.x * tx;
  c2* plane = S + (long)blockIdx.y * Ny * Nh;
  for (int i = threadIdx.x; i < tx * Ny; i += blockDim.x) {
    const int q = i % tx, jy = i / tx;
    A[q * Ny + jy] = (kx0 + q < Nh) ? plane[(long)jy * Nh + kx0 + q] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  const c2* R = fft_smem<T>(A, B, logNy, tx, Ny, tws, logNy, inverse != 0);
  for (int i = threadIdx.x; i < tx * Ny; i += blockDim.x) {
    const int q = i % tx, jy = i / tx;
    if (kx0 + q < Nh) plane[(long)jy * Nh + kx0 + q] = R[q * Ny + jy];
  }
}

// One warp per Fourier mode c = ky * Nh + kx: the column S[0..M1-1][c] times
// the mode's inverse Tab[idx] (row i, column j at i * M1 + j), transposed when
// tr != 0.  idx: 2D - kx, the Nyquist column kx = Nx/2 using the kappa = 0
// table; 3D - sidx[c].
template <typename T>
__global__ void __launch_bounds__(256) k_spec_cols(c2_t<T>* __restrict__ S, const T* __restrict__ Tab,
                                                   const int* __restrict__ sidx, int M1, int Ny, int Nh,
                                                   int tr) {
  pdl_enter();
  using c2 = c2_t<T>;
  const int lane = threadIdx.x & 31;
  const long nmodes = (long)Ny * Nh;
  const long stride = nmodes;
  for (long c = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nmodes;
       c += (long)gridDim.x * (blockDim.x >> 5)) {
    int ti;
    if (sidx) ti = sidx[c];
    else ti = (c == Nh - 1) ? 0 : (int)c;          // 2D: the Nyquist column has kappa = 0
    const T* M = Tab + (long)ti * M1 * M1;
    // lane l holds entries l and l + 32 of the column
    c2 v0 = mk<T>(T(0), T(0)), v1 = mk<T>(T(0), T(0));
    if (lane < M1) v0 = S[(long)lane * stride + c];
    if (lane + 32 < M1) v1 = S[(long)(lane + 32) * stride + c];
    c2 acc0 = mk<T>(T(0), T(0)), acc1 = mk<T>(T(0), T(0));
    for (int j = 0; j < M1; ++j) {
      const T re = __shfl_sync(0xffffffffu, j < 32 ? v0.x : v1.x, j & 31);
      const T im = __shfl_sync(0xffffffffu, j < 32 ? v0.y : v1.y, j & 31);
      if (lane < M1) {
        const T a = tr ? M[(long)j * M1 + lane] : M[(long)lane * M1 + j];
        acc0.x += a * re;
        acc0.y += a * im;
      }
      if (lane + 32 < M1) {
        const T a = tr ? M[(long)j * M1 + lane + 32] : M[(long)(lane + 32) * M1 + j];
        acc1.x += a * re;
        acc1.y += a * im;
      }
    }
    if (lane < M1) S[(long)lane * stride + c] = acc0;
    if (lane + 32 < M1) S[(long)(lane + 32) * stride + c] = acc1;
  }
}

template <typename T>
cudaError_t launch_spectral_smooth(const SpecArgs<T>& a, cudaStream_t s) {
  using c2 = c2_t<T>;
  const int nrows = a.M1 * a.Ny;
  const int H = a.Nx / 2, Nh = H + 1;
  cudaError_t e;
  {
    const size_t smem = (size_t)(2 * H + H) * sizeof(c2);
    if ((e = ensure_dyn_smem((const void*)k_spec_fwd_x<T>, smem)) != cudaSuccess) return e;
    if ((e = launch_k(k_spec_fwd_x<T>, dim3(nrows), dim3(256), smem, s, a.r, a.spec, a.logNx, a.tw, a.logNtw)) != cudaSuccess) return e;
  }
  // kx per CTA: 8 (a 64-byte FP32 / 128-byte FP64 segment per y row) as long
  // as both ping-pong buffers stay within 192 KB of shared memory
  int tx = 8;
  while (tx > 1 && (size_t)(2 * tx * a.Ny + a.Ny / 2) * sizeof(c2) > (size_t)192 * 1024) tx >>= 1;
  const size_t ysmem = (size_t)(2 * tx * a.Ny + a.Ny / 2) * sizeof(c2);
  const dim3 ygrid((Nh + tx - 1) / tx, a.M1);
  if (a.Ny > 1) {
    if ((e = ensure_dyn_smem((const void*)k_spec_y<T>, ysmem)) != cudaSuccess) return e;
    if ((e = launch_k(k_spec_y<T>, dim3(ygrid), dim3(256), ysmem, s, a.spec, a.Ny, a.logNy, Nh, tx, 0, a.tw, a.logNtw)) != cudaSuccess) return e;
  }
  {
    const long nmodes = (long)a.Ny * Nh;
    const int wpb = 8;
    const long blocks = std::min<long>((nmodes + wpb - 1) / wpb, 65535L);
    if ((e = launch_k(k_spec_cols<T>, dim3((unsigned)blocks), dim3(32 * wpb), 0, s, a.spec, a.tab, a.sidx, a.M1, a.Ny, Nh, a.tr)) != cudaSuccess) return e;
  }
  if (a.Ny > 1) {
    if ((e = launch_k(k_spec_y<T>, dim3(ygrid), dim3(256), ysmem, s, a.spec, a.Ny, a.logNy, Nh, tx, 1, a.tw, a.logNtw)) != cudaSuccess) return e;
  }
  {
    const size_t smem = (size_t)((H + 1) + H + H + H) * sizeof(c2);
    if ((e = ensure_dyn_smem((const void*)k_spec_inv_x<T>, smem)) != cudaSuccess) return e;
    if ((e = launch_k(k_spec_inv_x<T>, dim3(nrows), dim3(256), smem, s, a.spec, a.x, a.logNx, a.scale, a.first, a.tw, a.logNtw)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_spectral_smooth<float>(const SpecArgs<float>&, cudaStream_t);
template cudaError_t launch_spectral_smooth<double>(const SpecArgs<double>&, cudaStream_t);

}  // namespace wt
