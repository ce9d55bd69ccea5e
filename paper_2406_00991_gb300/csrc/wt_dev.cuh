// Device-side bodies of the spectral row passes and the column kernels.
//
// Each body works for any CTA size and walks its work units with a
// (first unit, stride) pair, so the same code runs as a multi-CTA kernel
// (first = blockIdx.x, stride = gridDim.x) and inside the single-CTA
// V-cycle kernel of wt_tail.cu (first = 0, stride = 1).  Every body keeps its
// __syncthreads() calls uniform across the CTA (no early return).
#pragma once

#include "wt_internal.h"

// Pointer qualifier of the body parameters: the single-CTA V-cycle kernel
// reads buffers it wrote earlier in the same launch and therefore compiles
// the bodies without WT_DEV_RESTRICT (no read-only-cache loads).
#ifndef WT_DEV_RESTRICT
#define WT_DEV_RESTRICT __restrict__
#endif

namespace wt {

template <typename T> __device__ __forceinline__ c2_t<T> mk(T re, T im);
template <> __device__ __forceinline__ float2 mk<float>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ double2 mk<double>(double re, double im) { return make_double2(re, im); }

// exp(-+2 pi i u / Nt) for 0 <= u < Nt from the half table tws (t < Nt/2).
template <typename T>
__device__ __forceinline__ c2_t<T> twiddle(const c2_t<T>* tws, int u, int halfNt, bool inverse) {
  c2_t<T> w = u < halfNt ? tws[u] : tws[u - halfNt];
  if (u >= halfNt) { w.x = -w.x; w.y = -w.y; }
  if (inverse) w.y = -w.y;
  return w;
}

template <typename T>
__device__ __forceinline__ c2_t<T> cmul(c2_t<T> a, c2_t<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Self-sorting (Stockham) FFT of nb sequences of length N = 2^logN stored with
// stride S in `a` (workspace `b`): one radix-2 stage when log2 N is odd, then
// radix-4 stages; each stage reads a[k + j m + s N/4], takes the 4-point DFT
// and writes W^{t j m} y_t to b[k + 4 j m + t m].  tws holds
// exp(-2 pi i t / Nt), t < Nt/2, Nt = 2^logNt >= N.  Returns the result buffer.
template <typename T>
__device__ c2_t<T>* fft_smem(c2_t<T>* a, c2_t<T>* b, int logN, int nb, int S, const c2_t<T>* tws,
                             int logNt, bool inverse) {
  using c2 = c2_t<T>;
  const int N = 1 << logN;
  const int tshift = logNt - logN;
  const int halfNt = 1 << (logNt - 1);
  int lm = 0;                                  // log2 m
  if (logN & 1) {
    const int half = N >> 1;
    for (int idx = threadIdx.x; idx < nb * half; idx += blockDim.x) {
      const int q = idx >> (logN - 1);
      const int k = idx & (half - 1);          // m = 1: j = k, k' = 0
      const c2 c0 = a[q * S + k], c1 = a[q * S + k + half];
      const c2 w = twiddle<T>(tws, k << tshift, halfNt, inverse);
      b[q * S + 2 * k] = mk<T>(c0.x + c1.x, c0.y + c1.y);
      b[q * S + 2 * k + 1] = cmul<T>(w, mk<T>(c0.x - c1.x, c0.y - c1.y));
    }
    __syncthreads();
    c2* t = a; a = b; b = t;
    lm = 1;
  }
  const int quarter = N >> 2;
  const int lq = logN - 2;
  for (; lm < logN; lm += 2) {
    const int m = 1 << lm;
    for (int idx = threadIdx.x; idx < (nb << lq); idx += blockDim.x) {
      const int q = idx >> lq;
      const int bf = idx & (quarter - 1);
      const int j = bf >> lm, k = bf & (m - 1);
      const c2* src = a + q * S + k + j * m;
      const c2 c0 = src[0], c1 = src[quarter], c2v = src[2 * quarter], c3 = src[3 * quarter];
      const T s02x = c0.x + c2v.x, s02y = c0.y + c2v.y, d02x = c0.x - c2v.x, d02y = c0.y - c2v.y;
      const T s13x = c1.x + c3.x, s13y = c1.y + c3.y, d13x = c1.x - c3.x, d13y = c1.y - c3.y;
      // forward: y1 = d02 - i d13, y3 = d02 + i d13 (inverse swaps them)
      const T sg = inverse ? T(-1) : T(1);
      const c2 y0 = mk<T>(s02x + s13x, s02y + s13y);
      const c2 y2 = mk<T>(s02x - s13x, s02y - s13y);
      const c2 y1 = mk<T>(d02x + sg * d13y, d02y - sg * d13x);
      const c2 y3 = mk<T>(d02x - sg * d13y, d02y + sg * d13x);
      const int u = (j * m) << tshift;
      c2* dst = b + q * S + k + 4 * j * m;
      dst[0] = y0;
      dst[m] = cmul<T>(twiddle<T>(tws, u, halfNt, inverse), y1);
      dst[2 * m] = cmul<T>(twiddle<T>(tws, 2 * u, halfNt, inverse), y2);
      dst[3 * m] = cmul<T>(twiddle<T>(tws, 3 * u, halfNt, inverse), y3);
    }
    __syncthreads();
    c2* t = a; a = b; b = t;
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

// Shared memory of one row-pass batch of ppc row pairs: two ping-pong
// buffers, the twiddles of the larger transform and the epilogue operands.
template <typename T>
__host__ __device__ inline size_t rowpass_smem(const RowPass<T>& a, int ppc) {
  const int Nmax = a.Nin > a.Nout ? a.Nin : a.Nout;
  const int S = Nmax + (a.ylines ? 1 : 0);
  const int nepi = (a.epi == EPI_ADD || a.epi == EPI_ACC) ? 1 : (a.epi == EPI_RESID ? 2 : 0);
  return ((2 + nepi) * (size_t)ppc * S + (size_t)(Nmax / 2)) * sizeof(c2_t<T>);
}

// One spectral pass over all row pairs: units of ppc pairs, unit u0, u0 +
// ustep, ...  The twiddles of the larger size are staged in shared memory and
// the epilogue operands (add / rhs / out) are fetched in the same loop as the
// input rows, so each batch costs one global round trip before the FFT.
template <typename T>
__device__ void rowpass_body(const RowPass<T>& a, int ppc, int u0, int ustep, unsigned char* smraw) {
  using c2 = c2_t<T>;
  const int Nmax = a.Nin > a.Nout ? a.Nin : a.Nout;
  const int logNmax = a.Nin > a.Nout ? a.logNin : a.logNout;
  const int S = Nmax + (a.ylines ? 1 : 0);
  const bool use_add = a.epi == EPI_ADD || a.epi == EPI_RESID;
  const bool use_rhs = a.epi == EPI_RESID || a.epi == EPI_ACC;
  c2* buf0 = reinterpret_cast<c2*>(smraw);
  c2* buf1 = buf0 + ppc * S;
  c2* tws = buf1 + ppc * S;
  c2* eA = tws + Nmax / 2;                     // add operand rows (pair packed)
  c2* eB = eA + (use_add ? ppc * S : 0);       // rhs (RESID) or old out (ACC)
  for (int t = threadIdx.x; t < Nmax / 2; t += blockDim.x) tws[t] = a.tw[t << (a.logNtw - logNmax)];
  const int npairs = (a.nrows + 1) >> 1;
  const T inv_n = T(1) / T(a.Nin);

  for (int p0 = u0 * ppc; p0 < npairs; p0 += ustep * ppc) {
    const int nb = min(ppc, npairs - p0);
    // ---- load two real rows per complex sequence (+ epilogue operands)
    for (int idx = threadIdx.x; idx < nb * a.Nin; idx += blockDim.x) {
      int q, j;
      if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNin; j = idx & (a.Nin - 1); }
      const int r0 = 2 * (p0 + q), r1 = r0 + 1;
      const T re = a.in[row_offset(a, r0, j, a.Nin)];
      const T im = r1 < a.nrows ? a.in[row_offset(a, r1, j, a.Nin)] : T(0);
      buf0[q * S + j] = mk<T>(re, im);
    }
    if (use_add || use_rhs) {
      const T* B = a.epi == EPI_ACC ? a.out : a.rhs;
      for (int idx = threadIdx.x; idx < nb * a.Nout; idx += blockDim.x) {
        int q, j;
        if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNout; j = idx & (a.Nout - 1); }
        const int r0 = 2 * (p0 + q), r1 = r0 + 1;
        const long o0 = row_offset(a, r0, j, a.Nout), o1 = row_offset(a, r1, j, a.Nout);
        const bool has1 = r1 < a.nrows;
        if (use_add) eA[q * S + j] = mk<T>(a.add[o0], has1 ? a.add[o1] : T(0));
        if (use_rhs) eB[q * S + j] = mk<T>(B[o0], has1 ? B[o1] : T(0));
      }
    }
    __syncthreads();
    c2* X = fft_smem<T>(buf0, buf1, a.logNin, nb, S, tws, logNmax, false);
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
    c2* Y = fft_smem<T>(Yb, X, a.logNout, nb, S, tws, logNmax, true);
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
        const c2 ad = eA[q * S + j];
        v0 += ad.x;
        v1 += ad.y;
      } else if (a.epi == EPI_RESID) {
        const c2 ad = eA[q * S + j], rh = eB[q * S + j];
        v0 = rh.x - (ad.x + v0);
        v1 = rh.y - (ad.y + v1);
      } else if (a.epi == EPI_ACC) {
        const c2 ol = eB[q * S + j];
        v0 += ol.x;
        v1 += ol.y;
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

// Column kernels: one warp owns one vertical column.  Lane l holds the
// sigma rows m = l and m = l + 32 (M1 <= 33), so a sigma contraction
// out[m] = sum_k M[m][k] in[k] takes in[k] by warp shuffle from its owner and
// M[m][k] from shared memory; columns are spread over all warps of the grid
// (unit u0, stride ustep counts CTAs).
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T bcast(T v0, T v1, int k) {
  return k < 32 ? __shfl_sync(kFull, v0, k) : __shfl_sync(kFull, v1, k - 32);
}

// sum_k M[m][k] v[k] for the lane's two rows (row-major M, leading dimension ld)
template <typename T>
__device__ __forceinline__ void contract(const T* sM, int ld, int Mi, int m0, int m1, bool r0, bool r1,
                                         T v0, T v1, T& o0, T& o1) {
  T a0 = 0, a1 = 0;
  for (int k = 0; k < Mi; ++k) {
    const T vk = bcast(v0, v1, k);
    if (r0) a0 += sM[m0 * ld + k] * vk;
    if (r1) a1 += sM[m1 * ld + k] * vk;
  }
  o0 = a0;
  o1 = a1;
}

template <typename T>
__host__ __device__ inline size_t opcols_smem(int M1) {
  return sizeof(T) * ((size_t)M1 * M1 + 64);
}

template <typename T, int DIM>
__device__ void opcols_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT p,
                            const T* WT_DEV_RESTRICT Px, const T* WT_DEV_RESTRICT Py,
                            T* WT_DEV_RESTRICT Gx, T* WT_DEV_RESTRICT Gy, T* WT_DEV_RESTRICT part,
                            int u0, int ustep, unsigned char* smraw) {
  const int M1 = L.M1;
  T* sD = reinterpret_cast<T*>(smraw);            // M1*M1
  T* sS = sD + M1 * M1;                           // sigma
  for (int i = threadIdx.x; i < M1 * M1; i += blockDim.x) sD[i] = L.D[i];
  for (int i = threadIdx.x; i < M1; i += blockDim.x) sS[i] = L.sigma[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long nc = L.ncols;
  const int m0 = lane, m1 = lane + 32;
  const bool r0 = m0 < M1, r1 = m1 < M1;
  const T* meta = L.meta;
  for (long c = (long)u0 * nw + wib; c < nc; c += (long)ustep * nw) {
    const T p0 = r0 ? p[m0 * nc + c] : T(0), p1 = r1 ? p[m1 * nc + c] : T(0);
    T ps0, ps1;
    contract(sD, M1, M1, m0, m1, r0, r1, p0, p1, ps0, ps1);            // P_s = D p
    const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
    const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
    const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
    const T HX = meta[M_HX * nc + c];
    const T s0 = r0 ? sS[m0] : T(0), s1 = r1 ? sS[m1] : T(0);
    T gx0 = r0 ? Px[m0 * nc + c] + (AXb - s0 * BXb) * ps0 : T(0);      // G_x
    T gx1 = r1 ? Px[m1 * nc + c] + (AXb - s1 * BXb) * ps1 : T(0);
    if (r0) Gx[m0 * nc + c] = gx0;
    if (r1) Gx[m1 * nc + c] = gx1;
    T gy0 = 0, gy1 = 0, AYa = 0, BYa = 0, HY = 0;
    if constexpr (DIM == 3) {
      const T AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
      AYa = meta[M_AYa * nc + c];
      BYa = meta[M_BYa * nc + c];
      HY = meta[M_HY * nc + c];
      gy0 = r0 ? Py[m0 * nc + c] + (AYb - s0 * BYb) * ps0 : T(0);      // G_y
      gy1 = r1 ? Py[m1 * nc + c] + (AYb - s1 * BYb) * ps1 : T(0);
      if (r0) Gy[m0 * nc + c] = gy0;
      if (r1) Gy[m1 * nc + c] = gy1;
    }
    T q0, q1, z0, z1, y0 = 0, y1 = 0;
    contract(sD, M1, M1, m0, m1, r0, r1, gx0, gx1, q0, q1);            // D G_x
    contract(sD, M1, M1, m0, m1, r0, r1, ps0, ps1, z0, z1);            // D P_s
    if constexpr (DIM == 3) contract(sD, M1, M1, m0, m1, r0, r1, gy0, gy1, y0, y1);
    const T ZZ = Za * Zb;
    auto row = [&](int m, T pv, T ps, T gx, T gy, T q, T z, T y, T s) -> T {
      if (m == 0) return pv;                                        // surface row: p
      if (m == M1 - 1) {                                            // bottom row: n . Grad_b p
        T b = HX * gx + Zb * ps;
        if constexpr (DIM == 3) b += HY * gy;
        return b;
      }
      T o = (AXa - s * BXa) * q + ZZ * z;
      if constexpr (DIM == 3) o += (AYa - s * BYa) * y;
      return o;
    };
    if (r0) part[m0 * nc + c] = row(m0, p0, ps0, gx0, gy0, q0, z0, y0, s0);
    if (r1) part[m1 * nc + c] = row(m1, p1, ps1, gx1, gy1, q1, z1, y1, s1);
  }
  __syncthreads();
}

// Block inverses are stored per column, contiguous and transposed:
// Binv[((c * nclass + cls) * M1 + k) * M1 + m] = (A_rr^{-1})[m][k], so lane m
// of a warp reads consecutive words for every k.
template <typename T, int DIM, int MAXM>
__device__ void smooth_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT r,
                            const T* WT_DEV_RESTRICT rhoX, const T* WT_DEV_RESTRICT rhoY,
                            const T* WT_DEV_RESTRICT rhoXY, const T* WT_DEV_RESTRICT Binv,
                            T* WT_DEV_RESTRICT x, T omega, int first, int u0, int ustep,
                            unsigned char* smraw) {
  constexpr int NC = DIM == 2 ? 2 : 4;
  const int M1 = L.M1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long nc = L.ncols;
  const int m0 = lane, m1 = lane + 32;
  const bool r0 = m0 < M1, r1 = m1 < M1;
  const long blk = (long)M1 * M1;
  for (long c = (long)u0 * nw + wib; c < nc; c += (long)ustep * nw) {
    const int jx = (int)(c % L.Nx), jy = (int)(c / L.Nx);
    const T sx = (jx & 1) ? T(-1) : T(1), sy = (jy & 1) ? T(-1) : T(1);
    T rp0[NC], rp1[NC];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = h ? m1 : m0;
      const bool ok = h ? r1 : r0;
      T rr = 0, rNx = 0, rNy = 0, rNN = 0;
      if (ok) {
        rr = r[m * nc + c];
        if constexpr (DIM == 2) {
          if (rhoX) rNx = rhoX[m] * sx;
        } else {
          const T cxy = rhoXY ? rhoXY[m] : T(0);
          rNN = cxy * sx * sy;
          if (rhoX) rNx = (rhoX[m * L.Ny + jy] - cxy * sy) * sx;
          if (rhoY) rNy = (rhoY[m * L.Nx + jx] - cxy * sx) * sy;
        }
      }
      T* rp = h ? rp1 : rp0;
      rp[0] = rr - rNx - rNy - rNN;
      rp[1] = rNx;
      if constexpr (DIM == 3) {
        rp[2] = rNy;
        rp[3] = rNN;
      }
    }
    const T xo0 = (!first && r0) ? x[m0 * nc + c] : T(0);
    const T xo1 = (!first && r1) ? x[m1 * nc + c] : T(0);
    T e0 = 0, e1 = 0;
#pragma unroll
    for (int cls = 0; cls < NC; ++cls) {
      const T* B = Binv + (c * NC + cls) * blk;
      // the lane's whole block row first (independent loads, one round trip);
      // shuffles stay outside lane-dependent branches
      T b0[MAXM];
      T b1[MAXM > 32 ? MAXM : 1];
#pragma unroll
      for (int k = 0; k < MAXM; ++k) b0[k] = (k < M1 && r0) ? B[k * M1 + m0] : T(0);
      if constexpr (MAXM > 32) {
#pragma unroll
        for (int k = 0; k < MAXM; ++k) b1[k] = (k < M1 && r1) ? B[k * M1 + m1] : T(0);
      }
#pragma unroll
      for (int k = 0; k < MAXM; ++k) {
        if (k < M1) {
          const T vk = bcast(rp0[cls], rp1[cls], k);
          e0 += b0[k] * vk;
          if constexpr (MAXM > 32) e1 += b1[k] * vk;
        }
      }
    }
    if (r0) x[m0 * nc + c] = xo0 + omega * e0;
    if (r1) x[m1 * nc + c] = xo1 + omega * e1;
  }
  __syncthreads();
}

// M1 bucket dispatch of smooth_body (MAXM >= M1).
template <typename T, int DIM>
__device__ void smooth_any(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                           const T* rhoXY, const T* Binv, T* x, T omega, int first, int u0,
                           int ustep, unsigned char* sm) {
  if (L.M1 <= 9)
    smooth_body<T, DIM, 9>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else if (L.M1 <= 17)
    smooth_body<T, DIM, 17>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else if (L.M1 <= 25)
    smooth_body<T, DIM, 25>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else
    smooth_body<T, DIM, 33>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
}

template <typename T>
__device__ void colmat_body(const T* WT_DEV_RESTRICT M, int Mo, int Mi, const T* WT_DEV_RESTRICT in,
                            T* WT_DEV_RESTRICT out, int ncols, int accumulate, int u0, int ustep,
                            unsigned char* smraw) {
  T* sM = reinterpret_cast<T*>(smraw);            // Mo*Mi
  for (int i = threadIdx.x; i < Mo * Mi; i += blockDim.x) sM[i] = M[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long nc = ncols;
  const int m0 = lane, m1 = lane + 32;
  const bool i0 = m0 < Mi, i1 = m1 < Mi, o0 = m0 < Mo, o1 = m1 < Mo;
  for (long c = (long)u0 * nw + wib; c < nc; c += (long)ustep * nw) {
    const T v0 = i0 ? in[m0 * nc + c] : T(0), v1 = i1 ? in[m1 * nc + c] : T(0);
    T a0, a1;
    contract(sM, Mi, Mi, m0, m1, o0, o1, v0, v1, a0, a1);
    if (o0) out[m0 * nc + c] = a0 + (accumulate ? out[m0 * nc + c] : T(0));
    if (o1) out[m1 * nc + c] = a1 + (accumulate ? out[m1 * nc + c] : T(0));
  }
  __syncthreads();
}

// Nyquist coefficient rho_r = (1/N) sum_j (-1)^j f[r*N + j] of rows w0, w0 +
// wstep, ... (one warp per row; w0 / wstep count warps).
template <typename T>
__device__ void nyquist_body(const T* WT_DEV_RESTRICT r, int nrows, int N, T* WT_DEV_RESTRICT rho,
                             int w0, int wstep) {
  const int lane = threadIdx.x & 31;
  for (int row = w0; row < nrows; row += wstep) {
    T s = 0;
    for (int j = lane; j < N; j += 32) s += ((j & 1) ? T(-1) : T(1)) * r[(long)row * N + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[row] = s / T(N);
  }
}

}  // namespace wt
