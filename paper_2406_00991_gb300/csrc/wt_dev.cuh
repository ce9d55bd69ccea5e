// Device-side bodies of the spectral row passes and the column kernels.
//
// Each body works for any CTA size and walks its work units with a
// (first unit, stride) pair, so the same code runs as a multi-CTA kernel
// (first = blockIdx.x, stride = gridDim.x) and inside the single-CTA
// V-cycle kernel of wt_tail.cu (first = 0, stride = 1).  Every body keeps its
// __syncthreads() calls uniform across the CTA (no early return).
#pragma once

#include "wt_internal.h"

// Pointer qualifier of the body parameters: the one-launch V-cycle kernels
// (one CTA, one cluster, the cooperative grid) and the batched tank kernel
// read buffers they wrote earlier in the same launch and therefore compile
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
// The thread group that runs a row pass (the whole CTA; the FFT and the row
// pass core are written against this interface).
struct BlockG {
  static constexpr bool block = true;
  static __device__ __forceinline__ int rank() { return threadIdx.x; }
  static __device__ __forceinline__ int size() { return blockDim.x; }
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};

template <typename T, typename G = BlockG>
__device__ c2_t<T>* fft_smem(c2_t<T>* a, c2_t<T>* b, int logN, int nb, int S, const c2_t<T>* tws,
                             int logNt, bool inverse) {
  using c2 = c2_t<T>;
  const int N = 1 << logN;
  const int tshift = logNt - logN;
  const int halfNt = 1 << (logNt - 1);
  int lm = 0;                                  // log2 m
  if (logN & 1) {
    const int half = N >> 1;
    for (int idx = G::rank(); idx < nb * half; idx += G::size()) {
      const int q = idx >> (logN - 1);
      const int k = idx & (half - 1);          // m = 1: j = k, k' = 0
      const c2 c0 = a[q * S + k], c1 = a[q * S + k + half];
      const c2 w = twiddle<T>(tws, k << tshift, halfNt, inverse);
      b[q * S + 2 * k] = mk<T>(c0.x + c1.x, c0.y + c1.y);
      b[q * S + 2 * k + 1] = cmul<T>(w, mk<T>(c0.x - c1.x, c0.y - c1.y));
    }
    G::sync();
    c2* t = a; a = b; b = t;
    lm = 1;
  }
  const int quarter = N >> 2;
  const int lq = logN - 2;
  for (; lm < logN; lm += 2) {
    const int m = 1 << lm;
    for (int idx = G::rank(); idx < (nb << lq); idx += G::size()) {
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
    G::sync();
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
  const int nepi = !a.prefetch ? 0 : (a.epi == EPI_ADD || a.epi == EPI_ACC) ? 1 : (a.epi == EPI_RESID ? 2 : 0);
  return ((2 + nepi) * (size_t)ppc * S + (size_t)(Nmax / 2)) * sizeof(c2_t<T>);
}

// One spectral pass over all row pairs: units of ppc pairs, unit u0, u0 +
// ustep, ...  The twiddles of the larger size are staged in shared memory and
// the epilogue operands (add / rhs / out) are fetched in the same loop as the
// input rows, so each batch costs one global round trip before the FFT.
template <typename T, typename G>
__device__ void rowpass_core(const RowPass<T>& a, int ppc, int u0, int ustep, c2_t<T>* buf0, c2_t<T>* buf1,
                             const c2_t<T>* tws, c2_t<T>* eA, c2_t<T>* eB) {
  using c2 = c2_t<T>;
  const int Nmax = a.Nin > a.Nout ? a.Nin : a.Nout;
  const int logNmax = a.Nin > a.Nout ? a.logNin : a.logNout;
  const int S = Nmax + (a.ylines ? 1 : 0);
  const bool use_add = a.prefetch && (a.epi == EPI_ADD || a.epi == EPI_RESID);
  const bool use_rhs = a.prefetch && (a.epi == EPI_RESID || a.epi == EPI_ACC);
  const int npairs = (a.nrows + 1) >> 1;
  const T inv_n = T(1) / T(a.Nin);

  for (int p0 = u0 * ppc; p0 < npairs; p0 += ustep * ppc) {
    const int nb = min(ppc, npairs - p0);
    // ---- load two real rows per complex sequence (+ epilogue operands)
    for (int idx = G::rank(); idx < nb * a.Nin; idx += G::size()) {
      int q, j;
      if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNin; j = idx & (a.Nin - 1); }
      const int r0 = 2 * (p0 + q), r1 = r0 + 1;
      const T re = a.in[row_offset(a, r0, j, a.Nin)];
      const T im = r1 < a.nrows ? a.in[row_offset(a, r1, j, a.Nin)] : T(0);
      buf0[q * S + j] = mk<T>(re, im);
    }
    if (use_add || use_rhs) {
      const T* B = a.epi == EPI_ACC ? a.out : a.rhs;
      for (int idx = G::rank(); idx < nb * a.Nout; idx += G::size()) {
        int q, j;
        if (a.ylines) { q = idx % nb; j = idx / nb; } else { q = idx >> a.logNout; j = idx & (a.Nout - 1); }
        const int r0 = 2 * (p0 + q), r1 = r0 + 1;
        const long o0 = row_offset(a, r0, j, a.Nout), o1 = row_offset(a, r1, j, a.Nout);
        const bool has1 = r1 < a.nrows;
        if (use_add) eA[q * S + j] = mk<T>(a.add[o0], has1 ? a.add[o1] : T(0));
        if (use_rhs) eB[q * S + j] = mk<T>(B[o0], has1 ? B[o1] : T(0));
      }
    }
    G::sync();
    c2* X = fft_smem<T, G>(buf0, buf1, a.logNin, nb, S, tws, logNmax, false);
    c2* Yb = (X == buf0) ? buf1 : buf0;
    // ---- spectral operation into Yb (length Nout)
    const int nkeep2 = (a.Nin < a.Nout ? a.Nin : a.Nout);   // keep |n| < nkeep2 / 2
    for (int idx = G::rank(); idx < nb * a.Nout; idx += G::size()) {
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
      } else if (a.op == XOP_RESAMPLE_DERIV) {
        const int an = ns < 0 ? -ns : ns;
        if (2 * an < nkeep2) {
          const int nin = ns < 0 ? ns + a.Nin : ns;
          const c2 x = X[q * S + nin];
          const T kap = a.kscale * T(ns);
          v = mk<T>(-kap * x.y, kap * x.x);
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
    G::sync();
    c2* Y = fft_smem<T, G>(Yb, X, a.logNout, nb, S, tws, logNmax, true);
    // ---- epilogue
    const T sc = a.scale * inv_n;
    for (int idx = G::rank(); idx < nb * a.Nout; idx += G::size()) {
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
      if (a.prefetch) {
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
      } else if (a.epi == EPI_ADD) {
        v0 += a.add[o0];
        if (has1) v1 += a.add[o1];
      } else if (a.epi == EPI_RESID) {
        v0 = a.rhs[o0] - (a.add[o0] + v0);
        if (has1) v1 = a.rhs[o1] - (a.add[o1] + v1);
      } else if (a.epi == EPI_ACC) {
        v0 += a.out[o0];
        if (has1) v1 += a.out[o1];
      }
      if (a.write_out) {
        a.out[o0] = v0;
        if (has1) a.out[o1] = v1;
      }
      if (a.nyq || a.out2) Y[q * S + j] = mk<T>(v0, has1 ? v1 : T(0));
    }
    if (a.nyq) {
      G::sync();
      const int lane = threadIdx.x & 31;
      const int warp = G::block ? (threadIdx.x >> 5) : 0, nw = G::block ? (blockDim.x >> 5) : 1;
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
    if (a.out2) {
      // second transform of the result rows held in Y: forward FFT, spectral
      // op2, inverse FFT of length Nout2, store with 1 / Nout
      G::sync();
      c2* Z = (Y == X) ? Yb : X;
      c2* Fq = fft_smem<T, G>(Y, Z, a.logNout, nb, S, tws, logNmax, false);
      c2* Gq = (Fq == Y) ? Z : Y;
      const int keep = a.Nout < a.Nout2 ? a.Nout : a.Nout2;
      for (int idx = G::rank(); idx < nb * a.Nout2; idx += G::size()) {
        const int q = idx >> a.logNout2, n = idx & (a.Nout2 - 1);
        const int ns = n < a.Nout2 / 2 ? n : n - a.Nout2;
        const int an = ns < 0 ? -ns : ns;
        c2 v = mk<T>(T(0), T(0));
        if (a.op2 == XOP_DERIV) {
          const c2 x = Fq[q * S + n];
          const T kap = (n == a.Nout2 / 2) ? T(0) : a.kscale * T(ns);
          v = mk<T>(-kap * x.y, kap * x.x);
        } else if (2 * an < keep) {
          v = Fq[q * S + (ns < 0 ? ns + a.Nout : ns)];
        }
        Gq[q * S + n] = v;
      }
      G::sync();
      c2* R = fft_smem<T, G>(Gq, Fq, a.logNout2, nb, S, tws, logNmax, true);
      const T s2 = T(1) / T(a.Nout);
      for (int idx = G::rank(); idx < nb * a.Nout2; idx += G::size()) {
        const int q = idx >> a.logNout2, j = idx & (a.Nout2 - 1);
        const int r0 = 2 * (p0 + q), r1 = r0 + 1;
        const c2 y = R[q * S + j];
        a.out2[(long)r0 * a.Nout2 + j] = y.x * s2;
        if (r1 < a.nrows) a.out2[(long)r1 * a.Nout2 + j] = y.y * s2;
      }
    }
    G::sync();
  }
}


// Row pass by the whole CTA: units of ppc pairs, unit u0, u0 + ustep, ...
template <typename T>
__device__ void rowpass_body(const RowPass<T>& a, int ppc, int u0, int ustep, unsigned char* smraw) {
  using c2 = c2_t<T>;
  const int Nmax = a.Nin > a.Nout ? a.Nin : a.Nout;
  const int logNmax = a.Nin > a.Nout ? a.logNin : a.logNout;
  const int S = Nmax + (a.ylines ? 1 : 0);
  const bool use_add = a.prefetch && (a.epi == EPI_ADD || a.epi == EPI_RESID);
  c2* buf0 = reinterpret_cast<c2*>(smraw);
  c2* buf1 = buf0 + ppc * S;
  c2* tws = buf1 + ppc * S;
  c2* eA = tws + Nmax / 2;                     // add operand rows (pair packed)
  c2* eB = eA + (use_add ? ppc * S : 0);       // rhs (RESID) or old out (ACC)
  const int npairs = (a.nrows + 1) >> 1;
  if (u0 * ppc >= npairs) return;              // no unit for this CTA
  for (int t = threadIdx.x; t < Nmax / 2; t += blockDim.x) tws[t] = a.tw[t << (a.logNtw - logNmax)];
  rowpass_core<T, BlockG>(a, ppc, u0, ustep, buf0, buf1, tws, eA, eB);
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

// sum_k M[m][k] v[k] for the lane's two rows (row-major M, leading dimension
// ld).  KM > 0: Mi == ld == KM at compile time, so the loop unrolls and the
// broadcasts issue back to back.
template <typename T, int KM = 0>
__device__ __forceinline__ void contract(const T* sM, int ld, int Mi, int m0, int m1, bool r0, bool r1,
                                         T v0, T v1, T& o0, T& o1) {
  T a0 = 0, a1 = 0;
  if constexpr (KM > 0) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const T vk = bcast(v0, v1, k);
      if (r0) a0 += sM[m0 * KM + k] * vk;
      if (KM > 32 && r1) a1 += sM[m1 * KM + k] * vk;
    }
  } else {
    for (int k = 0; k < Mi; ++k) {
      const T vk = bcast(v0, v1, k);
      if (r0) a0 += sM[m0 * ld + k] * vk;
      if (r1) a1 += sM[m1 * ld + k] * vk;
    }
  }
  o0 = a0;
  o1 = a1;
}

template <typename T>
__host__ __device__ inline size_t opcols_smem(int M1) {
  return sizeof(T) * ((size_t)M1 * M1 + 64);
}

// KM > 0: the level's M1 equals KM (compile-time column length).
template <typename T, int DIM, int KM = 0>
__device__ void opcols_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT p,
                            const T* WT_DEV_RESTRICT Px, const T* WT_DEV_RESTRICT Py,
                            T* WT_DEV_RESTRICT Gx, T* WT_DEV_RESTRICT Gy, T* WT_DEV_RESTRICT part,
                            int u0, int ustep, unsigned char* smraw) {
  const int M1 = KM > 0 ? KM : L.M1;
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
    contract<T, KM>(sD, M1, M1, m0, m1, r0, r1, p0, p1, ps0, ps1);            // P_s = D p
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
    contract<T, KM>(sD, M1, M1, m0, m1, r0, r1, gx0, gx1, q0, q1);            // D G_x
    contract<T, KM>(sD, M1, M1, m0, m1, r0, r1, ps0, ps1, z0, z1);            // D P_s
    if constexpr (DIM == 3) contract<T, KM>(sD, M1, M1, m0, m1, r0, r1, gy0, gy1, y0, y1);
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

// Column part of the transposed operator A_{a,b}^T (2D).  With lam_int =
// lam without its surface and bottom rows and Dlam = D_x lam (all rows):
//   mu_x = -Dlam_int + D^T (sx_a lam_int) + h_x lam_bottom e_bottom
//   mu_z = D^T (Z_a lam_int) + lam_bottom e_bottom
//   part = D^T (sx_b mu_x + Z_b mu_z) + lam_surface e_surface,
// so that A^T lam = part + D_x^T mu_x = part - D_x mu_x (the x-derivative
// matrix is antisymmetric).  mu_x goes to Mx, part to part.
template <typename T>
__device__ void opcolsT_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT lam,
                             const T* WT_DEV_RESTRICT Dlam, T* WT_DEV_RESTRICT Mx,
                             T* WT_DEV_RESTRICT part, int u0, int ustep, unsigned char* smraw) {
  const int M1 = L.M1;
  T* sDt = reinterpret_cast<T*>(smraw);           // D^T, M1*M1
  T* sS = sDt + M1 * M1;                          // sigma
  for (int i = threadIdx.x; i < M1 * M1; i += blockDim.x) {
    const int m = i / M1, k = i - m * M1;
    sDt[i] = L.D[k * M1 + m];
  }
  for (int i = threadIdx.x; i < M1; i += blockDim.x) sS[i] = L.sigma[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long nc = L.ncols;
  const int m0 = lane, m1 = lane + 32;
  const bool r0 = m0 < M1, r1 = m1 < M1;
  const bool i0 = r0 && m0 > 0 && m0 < M1 - 1, i1 = r1 && m1 < M1 - 1;
  const T* meta = L.meta;
  for (long c = (long)u0 * nw + wib; c < nc; c += (long)ustep * nw) {
    const T l0 = r0 ? lam[m0 * nc + c] : T(0), l1 = r1 ? lam[m1 * nc + c] : T(0);
    const T lsurf = bcast(l0, l1, 0), lbot = bcast(l0, l1, M1 - 1);
    const T li0 = i0 ? l0 : T(0), li1 = i1 ? l1 : T(0);
    const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
    const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
    const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
    const T HX = meta[M_HX * nc + c];
    const T s0 = r0 ? sS[m0] : T(0), s1 = r1 ? sS[m1] : T(0);
    T da0, da1, dz0, dz1;
    contract(sDt, M1, M1, m0, m1, r0, r1, (AXa - s0 * BXa) * li0, (AXa - s1 * BXa) * li1, da0, da1);
    contract(sDt, M1, M1, m0, m1, r0, r1, Za * li0, Za * li1, dz0, dz1);
    const T dl0 = i0 ? Dlam[m0 * nc + c] : T(0), dl1 = i1 ? Dlam[m1 * nc + c] : T(0);
    const bool b0 = m0 == M1 - 1, b1 = m1 == M1 - 1;
    const T mx0 = -dl0 + da0 + (b0 ? HX * lbot : T(0));
    const T mx1 = -dl1 + da1 + (b1 ? HX * lbot : T(0));
    const T mz0 = dz0 + (b0 ? lbot : T(0)), mz1 = dz1 + (b1 ? lbot : T(0));
    const T q0 = r0 ? (AXb - s0 * BXb) * mx0 + Zb * mz0 : T(0);
    const T q1 = r1 ? (AXb - s1 * BXb) * mx1 + Zb * mz1 : T(0);
    T o0, o1;
    contract(sDt, M1, M1, m0, m1, r0, r1, q0, q1, o0, o1);
    if (r0) {
      Mx[m0 * nc + c] = mx0;
      part[m0 * nc + c] = o0 + (m0 == 0 ? lsurf : T(0));
    }
    if (r1) {
      Mx[m1 * nc + c] = mx1;
      part[m1 * nc + c] = o1;
    }
  }
  __syncthreads();
}

// The same sigma part with one thread per column, for levels with many
// columns (3D): adjacent threads take adjacent columns, so every load and
// store of a sigma row is coalesced across the warp (the warp-per-column
// layout reads one sector per element there).  MAXM >= M1.
template <typename T, int DIM, int MAXM>
__device__ void opcols_tpc_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT p,
                                const T* WT_DEV_RESTRICT Px, const T* WT_DEV_RESTRICT Py,
                                T* WT_DEV_RESTRICT Gx, T* WT_DEV_RESTRICT Gy, T* WT_DEV_RESTRICT part,
                                unsigned char* smraw) {
  const int M1 = L.M1;
  T* sD = reinterpret_cast<T*>(smraw);
  T* sS = sD + M1 * M1;
  for (int i = threadIdx.x; i < M1 * M1; i += blockDim.x) sD[i] = L.D[i];
  for (int i = threadIdx.x; i < M1; i += blockDim.x) sS[i] = L.sigma[i];
  __syncthreads();
  const long nc = L.ncols;
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const T* meta = L.meta;
  T pv[MAXM], ps[MAXM], gx[MAXM], gy[DIM == 3 ? MAXM : 1];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) pv[m] = m < M1 ? p[m * nc + c] : T(0);
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < MAXM; ++k)
      if (m < M1 && k < M1) a += sD[m * M1 + k] * pv[k];
    ps[m] = a;
  }
  const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
  const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
  const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
  const T HX = meta[M_HX * nc + c];
  T AYa = 0, BYa = 0, HY = 0;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (m < M1) {
      gx[m] = Px[m * nc + c] + (AXb - sS[m] * BXb) * ps[m];
      Gx[m * nc + c] = gx[m];
    } else {
      gx[m] = T(0);
    }
  }
  if constexpr (DIM == 3) {
    const T AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
    AYa = meta[M_AYa * nc + c];
    BYa = meta[M_BYa * nc + c];
    HY = meta[M_HY * nc + c];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m < M1) {
        gy[m] = Py[m * nc + c] + (AYb - sS[m] * BYb) * ps[m];
        Gy[m * nc + c] = gy[m];
      } else {
        gy[m] = T(0);
      }
    }
  }
  const T ZZ = Za * Zb;
  part[c] = pv[0];                                                   // surface row: p
#pragma unroll
  for (int m = 1; m < MAXM; ++m) {
    if (m >= M1 - 1) continue;
    T q = 0, z = 0, y = 0;
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      if (k < M1) {
        const T d = sD[m * M1 + k];
        q += d * gx[k];
        z += d * ps[k];
        if constexpr (DIM == 3) y += d * gy[k];
      }
    }
    const T s = sS[m];
    T o = (AXa - s * BXa) * q + ZZ * z;
    if constexpr (DIM == 3) o += (AYa - s * BYa) * y;
    part[m * nc + c] = o;
  }
  const int N = M1 - 1;                                              // bottom row: n . Grad_b p
  T bsum = 0, gxN = 0, gyN = 0, psN = 0;
#pragma unroll
  for (int m = 0; m < MAXM; ++m)
    if (m == N) {
      gxN = gx[m];
      psN = ps[m];
      if constexpr (DIM == 3) gyN = gy[m];
    }
  bsum = HX * gxN + Zb * psN;
  if constexpr (DIM == 3) bsum += HY * gyN;
  part[N * nc + c] = bsum;
}

// Block inverses are stored per column, contiguous and transposed:
// Binv[((c * nclass + cls) * M1 + k) * M1 + m] = (A_rr^{-1})[m][k], so lane m
// of a warp reads consecutive words for every k.  EXACT: M1 == MAXM, so the
// block stride is a compile-time constant (immediate load offsets from one
// base instead of one address register pair per hoisted load).
template <typename T, int DIM, int MAXM, bool TR = false, bool EXACT = false>
__device__ void smooth_body(const LevelView<T>& L, const T* WT_DEV_RESTRICT r,
                            const T* WT_DEV_RESTRICT rhoX, const T* WT_DEV_RESTRICT rhoY,
                            const T* WT_DEV_RESTRICT rhoXY, const T* WT_DEV_RESTRICT Binv,
                            T* WT_DEV_RESTRICT x, T omega, int first, int u0, int ustep,
                            unsigned char* smraw) {
  constexpr int NC = DIM == 2 ? 2 : 4;
  const int M1 = EXACT ? MAXM : L.M1;
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
      for (int k = 0; k < MAXM; ++k) b0[k] = (k < M1 && r0) ? B[TR ? m0 * M1 + k : k * M1 + m0] : T(0);
      if constexpr (MAXM > 32) {
#pragma unroll
        for (int k = 0; k < MAXM; ++k) b1[k] = (k < M1 && r1) ? B[TR ? m1 * M1 + k : k * M1 + m1] : T(0);
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

// M1 bucket dispatch of smooth_body (MAXM >= M1).  TR: the transposed
// blocks (A_rr^{-1})^T = (A^T)_rr^{-1}, the smoother of A^T.
template <typename T, int DIM, bool TR = false>
__device__ void smooth_any(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                           const T* rhoXY, const T* Binv, T* x, T omega, int first, int u0,
                           int ustep, unsigned char* sm) {
  if (L.M1 <= 9)
    smooth_body<T, DIM, 9, TR>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else if (L.M1 <= 17)
    smooth_body<T, DIM, 17, TR>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else if (L.M1 <= 25)
    smooth_body<T, DIM, 25, TR>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
  else
    smooth_body<T, DIM, 33, TR>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, u0, ustep, sm);
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

// Diagonal column block of A_{a,b} (the same expression the oracle pins
// against its dense assembly): interior rows
//   cdiag I + (sx_a AX_b + sy_a AY_b + Z_a Z_b) D^2 - (sx_a BX_b + sy_a BY_b) D diag(sigma) D,
// surface row e_0, bottom row (h_x sx_b + h_y sy_b + Z_b) D[Nz, :].
// One (column, class) task of the calling warp, in A (M1 x (2 M1 + 1)
// values of shared memory).
template <typename T>
__device__ void blockinv_task(const LevelView<T>& L, T* WT_DEV_RESTRICT Binv, int nclass, T cxx, T cyy,
                              int* flag, long task, T* A) {
  const int M1 = L.M1;
  const int W = 2 * M1 + 1;                 // padded row of the augmented matrix
  const int lane = threadIdx.x & 31;
  const long nc = L.ncols;
  const long blk = (long)M1 * M1;
  {
    const int c = (int)(task % nc), cls = (int)(task / nc);
    const int ix = cls & 1, iy = (cls >> 1) & 1;
    const T cdiag = (ix ? T(0) : cxx) + (iy ? T(0) : cyy);
    const T* meta = L.meta;
    const T AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
    const T AYa = meta[M_AYa * nc + c], BYa = meta[M_BYa * nc + c];
    const T AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
    const T AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
    const T Za = meta[M_Za * nc + c], Zb = meta[M_Zb * nc + c];
    const T HX = meta[M_HX * nc + c], HY = meta[M_HY * nc + c];
    const T sbot = L.sigma[M1 - 1];
    const T cbot = HX * (AXb - sbot * BXb) + HY * (AYb - sbot * BYb) + Zb;
    for (int i = lane; i < M1 * M1; i += 32) {
      const int m = i / M1, k = i - m * M1;
      T v;
      if (m == 0) {
        v = (k == 0) ? T(1) : T(0);
      } else if (m == M1 - 1) {
        v = cbot * L.D[m * M1 + k];
      } else {
        const T s = L.sigma[m];
        const T sxa = AXa - s * BXa, sya = AYa - s * BYa;
        v = (sxa * AXb + sya * AYb + Za * Zb) * L.D2[m * M1 + k] -
            (sxa * BXb + sya * BYb) * L.DSD[m * M1 + k];
        if (m == k) v += cdiag;
      }
      A[m * W + k] = v;
      A[m * W + M1 + k] = (m == k) ? T(1) : T(0);
    }
    __syncwarp();
    bool bad = false;
    for (int piv = 0; piv < M1; ++piv) {
      // pivot search over rows piv..M1-1
      T best = T(-1);
      int bi = piv;
      for (int i = piv + lane; i < M1; i += 32) {
        const T a = fabs(A[i * W + piv]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (!(best > T(0)) || !isfinite(best)) { bad = true; break; }
      if (bi != piv) {
        for (int j = lane; j < 2 * M1; j += 32) {
          const T t0 = A[piv * W + j];
          A[piv * W + j] = A[bi * W + j];
          A[bi * W + j] = t0;
        }
      }
      __syncwarp();
      const T inv = T(1) / A[piv * W + piv];
      __syncwarp();
      for (int j = lane; j < 2 * M1; j += 32) A[piv * W + j] *= inv;
      __syncwarp();
      for (int i = lane; i < M1; i += 32) {
        if (i == piv) continue;
        const T f = A[i * W + piv];
        if (f != T(0)) {
          for (int j = 0; j < 2 * M1; ++j) A[i * W + j] -= f * A[piv * W + j];
        }
      }
      __syncwarp();
    }
    if (bad) {
      if (lane == 0) atomicOr(flag, 1);
    }
    for (int i = lane; i < M1 * M1; i += 32) {   // i = k * M1 + m: coalesced stores
      const int k = i / M1, m = i - k * M1;
      Binv[((long)c * nclass + cls) * blk + i] = bad ? T(0) : A[m * W + M1 + k];
    }
    __syncwarp();
  }
}

// One warp per (column, class) task; `wmax` warps of the CTA take part (each
// needs M1 x (2 M1 + 1) values of shared memory), CTA u0 of ustep.
template <typename T>
__device__ void blockinv_body(const LevelView<T>& L, T* WT_DEV_RESTRICT Binv, int nclass, T cxx,
                              T cyy, int* flag, int u0, int ustep, int wmax, unsigned char* smraw) {
  const int M1 = L.M1;
  const int wib = threadIdx.x >> 5;
  const int nw = min((int)(blockDim.x >> 5), wmax);
  T* A = reinterpret_cast<T*>(smraw) + wib * (M1 * (2 * M1 + 1));
  if (wib >= nw) return;
  for (long task = (long)u0 * nw + wib; task < (long)L.ncols * nclass; task += (long)ustep * nw)
    blockinv_task<T>(L, Binv, nclass, cxx, cyy, flag, task, A);
}

// Assemble the dense A_{a,b} of the coarsest level and invert it in shared
// memory (one CTA; n (n + 1) doubles + n + 1 ints of shared memory).
__device__ inline void coarse_factor_body(const LevelView<double>& L, const double* WT_DEV_RESTRICT Dx,
                                          const double* WT_DEV_RESTRICT Dy, double* WT_DEV_RESTRICT LUout,
                                          int* flag, unsigned char* smraw) {
  const int Nx = L.Nx, Ny = L.Ny, M1 = L.M1;
  const int n = M1 * Ny * Nx;
  const int ld = n + 1;
  double* A = reinterpret_cast<double*>(smraw);
  int* perm = reinterpret_cast<int*>(A + (size_t)n * ld);
  int& spiv = perm[n];
  const double* Dxx = Dx + Nx * Nx;
  const double* Dyy = Dy + Ny * Ny;
  const long nc = L.ncols;
  const double* meta = L.meta;
  const double* D = L.D;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    const int m = i / (Ny * Nx), y = (i / Nx) % Ny, x = i % Nx;
    const int mp = j / (Ny * Nx), yp = (j / Nx) % Ny, xp = j % Nx;
    const int c = y * Nx + x;
    const bool sy_ = (y == yp), sx_ = (x == xp), sm_ = (m == mp);
    double v = 0.0;
    if (m == 0) {
      v = (i == j) ? 1.0 : 0.0;
    } else if (m == M1 - 1) {
      const double s = L.sigma[m];
      const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double HX = meta[M_HX * nc + c], HY = meta[M_HY * nc + c];
      const double Zb = meta[M_Zb * nc + c];
      const double Dm = D[m * M1 + mp];
      if (sy_) v += HX * ((mp == m ? Dx[x * Nx + xp] : 0.0) + (sx_ ? sxb * Dm : 0.0));
      if (sx_) v += HY * ((mp == m ? Dy[y * Ny + yp] : 0.0) + (sy_ ? syb * Dm : 0.0));
      if (sx_ && sy_) v += Zb * Dm;
    } else {
      const double s = L.sigma[m];
      const double Dm = D[m * M1 + mp];
      const double AXa = meta[M_AXa * nc + c], BXa = meta[M_BXa * nc + c];
      const double AYa = meta[M_AYa * nc + c], BYa = meta[M_BYa * nc + c];
      const double sxa = AXa - s * BXa, sya = AYa - s * BYa;
      const double D2m = L.D2[m * M1 + mp], DSDm = L.DSD[m * M1 + mp];
      if (sy_) {
        const int cp = y * Nx + xp;   // column (y, x')
        const double sxb_p = meta[M_AXb * nc + cp] - s * meta[M_BXb * nc + cp];
        v += (sm_ ? Dxx[x * Nx + xp] : 0.0) + Dx[x * Nx + xp] * sxb_p * Dm;
        v += sxa * Dm * Dx[x * Nx + xp];
      }
      if (sx_) {
        const int cp = yp * Nx + x;   // column (y', x)
        const double syb_p = meta[M_AYb * nc + cp] - s * meta[M_BYb * nc + cp];
        v += (sm_ ? Dyy[y * Ny + yp] : 0.0) + Dy[y * Ny + yp] * syb_p * Dm;
        v += sya * Dm * Dy[y * Ny + yp];
      }
      if (sx_ && sy_) {
        const double AXb = meta[M_AXb * nc + c], BXb = meta[M_BXb * nc + c];
        const double AYb = meta[M_AYb * nc + c], BYb = meta[M_BYb * nc + c];
        v += sxa * (AXb * D2m - BXb * DSDm) + sya * (AYb * D2m - BYb * DSDm);
        v += meta[M_Za * nc + c] * meta[M_Zb * nc + c] * D2m;
      }
    }
    A[i * ld + j] = v;
  }
  __syncthreads();
  // in-place Gauss-Jordan inversion with row pivoting (the pivot column is
  // overwritten by the inverse's column; row swaps become column swaps at the end)
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        const double a = fabs(A[i * ld + k]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        spiv = bi;
        perm[k] = bi;
        if (!(best > 0.0) || !isfinite(best)) atomicOr(flag, 2);
      }
    }
    __syncthreads();
    const int p = spiv;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t0 = A[k * ld + j];
        A[k * ld + j] = A[p * ld + j];
        A[p * ld + j] = t0;
      }
      __syncthreads();
    }
    const double inv = 1.0 / A[k * ld + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[k * ld + j] = (j == k ? 1.0 : A[k * ld + j]) * inv;
    __syncthreads();
    // eliminate column k from every other row; column k of those rows becomes -f * inv
    for (int idx = threadIdx.x; idx < (n - 1) * n; idx += blockDim.x) {
      int i = idx / n;
      const int j = idx - i * n;
      if (i >= k) ++i;
      const double f = A[i * ld + k];
      if (j != k) A[i * ld + j] -= f * A[k * ld + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) A[i * ld + k] = -A[i * ld + k] * A[k * ld + k];
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t0 = A[i * ld + k];
        A[i * ld + k] = A[i * ld + p];
        A[i * ld + p] = t0;
      }
    }
    __syncthreads();
  }
  // store the inverse transposed: LUout[j * n + i] = Ainv[i][j] (coalesced solve)
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    LUout[j * n + i] = A[i * ld + j];
  }
}

// Metric of Eq. 1_Scoef per column for the geometries a (eta_a) and b (eta_b):
// d = h + eta, d_x = h_x + eta_x;  sigma_x = (h_x - sigma d_x)/d = AX - sigma BX.
__device__ inline void metric_body(long t0, long ts, int ncols, const double* WT_DEV_RESTRICT h, const double* WT_DEV_RESTRICT hx,
                              const double* WT_DEV_RESTRICT hy, const double* WT_DEV_RESTRICT ea,
                              const double* WT_DEV_RESTRICT eax, const double* WT_DEV_RESTRICT eay,
                              const double* WT_DEV_RESTRICT eb, const double* WT_DEV_RESTRICT ebx,
                              const double* WT_DEV_RESTRICT eby, double* WT_DEV_RESTRICT meta, int* flag) {
  for (long c = t0; c < ncols; c += ts) {
    const double HX = hx[c], HY = hy ? hy[c] : 0.0;
    const double da = h[c] + ea[c], db = h[c] + eb[c];
    const double dxa = HX + eax[c], dxb = HX + ebx[c];
    const double dya = HY + (eay ? eay[c] : 0.0), dyb = HY + (eby ? eby[c] : 0.0);
    if (!(da > 0.0) || !(db > 0.0) || !isfinite(da) || !isfinite(db) || !isfinite(dxa) ||
        !isfinite(dxb) || !isfinite(dya) || !isfinite(dyb))
      atomicOr(flag, 4);
    const double ia = 1.0 / da, ib = 1.0 / db;
    meta[M_AXa * (long)ncols + c] = HX * ia;
    meta[M_BXa * (long)ncols + c] = dxa * ia;
    meta[M_AYa * (long)ncols + c] = HY * ia;
    meta[M_BYa * (long)ncols + c] = dya * ia;
    meta[M_Za * (long)ncols + c] = ia;
    meta[M_AXb * (long)ncols + c] = HX * ib;
    meta[M_BXb * (long)ncols + c] = dxb * ib;
    meta[M_AYb * (long)ncols + c] = HY * ib;
    meta[M_BYb * (long)ncols + c] = dyb * ib;
    meta[M_Zb * (long)ncols + c] = ib;
    meta[M_HX * (long)ncols + c] = HX;
    meta[M_HY * (long)ncols + c] = HY;
    meta[M_D_A * (long)ncols + c] = da;
    meta[M_D_B * (long)ncols + c] = db;
  }
}


// Kinematic free-surface condition (Eq. kinematicFS) and its 2N register:
// f_eta = -u~ eta_x - v~ eta_y + w~ (linear model: w~); K = alpha K + dt f;
// eta^(k) = eta^(k-1) + beta K.  u~ = surface node (sigma index 0).
__device__ inline void stage_eta_body(long t0, long ts, int ncols, int linear, double alpha, double beta, double dt,
                            const double* WT_DEV_RESTRICT u, const double* WT_DEV_RESTRICT v,
                            const double* WT_DEV_RESTRICT w, const double* WT_DEV_RESTRICT ex,
                            const double* WT_DEV_RESTRICT ey, double* WT_DEV_RESTRICT Keta,
                            const double* WT_DEV_RESTRICT eta, double* WT_DEV_RESTRICT eta_new,
                            double* WT_DEV_RESTRICT f_eta, int* flag) {
  for (long c = t0; c < ncols; c += ts) {
    const double ut = u[c], vt = v ? v[c] : 0.0, wt = w[c];
    const double fe = linear ? wt : (-ut * ex[c] - (v ? vt * ey[c] : 0.0) + wt);
    const double K = alpha * Keta[c] + dt * fe;
    Keta[c] = K;
    const double en = eta[c] + beta * K;
    eta_new[c] = en;
    f_eta[c] = fe;
    if (!isfinite(en)) atomicOr(flag, 8);
  }
}

// Momentum forcing without p_D (Eq. forc1 with the pressure split of Sec. 2):
//   F_q = -(u q_x + v q_y + w_sigma q_sigma) - g (eta_x, eta_y, 0)_q,
//   w_sigma = sigma_t + u sigma_x + v sigma_y + w sigma_z, sigma_t = -sigma f_eta / d,
// then K_q <- alpha K_q + dt F_q and q* = q + beta K_q (q* overwrites the
// sigma-derivative inputs Dq).
__device__ inline void stage_forcing_body(long t0, long ts, StageArgs a, const double* WT_DEV_RESTRICT u, const double* WT_DEV_RESTRICT v,
                                const double* WT_DEV_RESTRICT w, const double* WT_DEV_RESTRICT ux,
                                const double* WT_DEV_RESTRICT uy, const double* WT_DEV_RESTRICT vx,
                                const double* WT_DEV_RESTRICT vy, const double* WT_DEV_RESTRICT wx,
                                const double* WT_DEV_RESTRICT wy, const double* WT_DEV_RESTRICT ex,
                                const double* WT_DEV_RESTRICT ey, const double* WT_DEV_RESTRICT f_eta,
                                double* WT_DEV_RESTRICT Ku, double* WT_DEV_RESTRICT Kv,
                                double* WT_DEV_RESTRICT Kw, double* WT_DEV_RESTRICT us,
                                double* WT_DEV_RESTRICT vs, double* WT_DEV_RESTRICT ws) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  for (long e = t0; e < n; e += ts) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double uu = u[e], ww = w[e], vv = v ? v[e] : 0.0;
    double Fu = -a.g * ex[c], Fv = v ? -a.g * ey[c] : 0.0, Fw = 0.0;
    if (!a.linear) {
      const double* meta = a.meta;
      const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double Zb = meta[M_Zb * nc + c], db = meta[M_D_B * nc + c];
      const double wsig = -s * f_eta[c] / db + uu * sxb + vv * syb + ww * Zb;
      Fu -= uu * ux[e] + wsig * us[e];
      Fw -= uu * wx[e] + wsig * ws[e];
      if (v) {
        Fu -= vv * uy[e];
        Fw -= vv * wy[e];
        Fv -= uu * vx[e] + vv * vy[e] + wsig * vs[e];
      }
    }
    if (a.nu != 0.0) {                   // nu Div_b Grad_b q (Eq. sigmom1, forc1)
      Fu += a.nu * a.lap_u[e];
      Fw += a.nu * a.lap_w[e];
      if (v) Fv += a.nu * a.lap_v[e];
    }
    const double ku = a.alpha * Ku[e] + a.dt * Fu;
    const double kw = a.alpha * Kw[e] + a.dt * Fw;
    Ku[e] = ku;
    Kw[e] = kw;
    us[e] = uu + a.beta * ku;
    ws[e] = ww + a.beta * kw;
    if (v) {
      const double kv = a.alpha * Kv[e] + a.dt * Fv;
      Kv[e] = kv;
      vs[e] = vv + a.beta * kv;
    }
  }
}

// Poisson right-hand side in projection form (Eq. poissonp, bcpd, bcpdneu):
// interior Div_a u* / (beta dt), surface 0, bottom (h_x u* + h_y v* + w*)/(beta dt).
// Inputs: u*_x, v*_y and the sigma-derivatives D u*, D v*, D w* (in Dus, Dvs, Dws).
__device__ inline void stage_rhs_body(long t0, long ts, StageArgs a, const double* WT_DEV_RESTRICT us, const double* WT_DEV_RESTRICT vs,
                            const double* WT_DEV_RESTRICT ws, const double* WT_DEV_RESTRICT usx,
                            const double* WT_DEV_RESTRICT vsy, const double* WT_DEV_RESTRICT Dus,
                            const double* WT_DEV_RESTRICT Dvs, const double* WT_DEV_RESTRICT Dws,
                            double* WT_DEV_RESTRICT rhs) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  const double ib = 1.0 / (a.beta * a.dt);
  for (long e = t0; e < n; e += ts) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double* meta = a.meta;
    double b;
    if (m == 0) {
      b = 0.0;
    } else if (m == a.M1 - 1) {
      b = (meta[M_HX * nc + c] * us[e] + (vs ? meta[M_HY * nc + c] * vs[e] : 0.0) + ws[e]) * ib;
    } else {
      const double s = a.sigma[m];
      const double sxa = meta[M_AXa * nc + c] - s * meta[M_BXa * nc + c];
      double d = usx[e] + sxa * Dus[e] + meta[M_Za * nc + c] * Dws[e];
      if (vs) {
        const double sya = meta[M_AYa * nc + c] - s * meta[M_BYa * nc + c];
        d += vsy[e] + sya * Dvs[e];
      }
      b = d * ib;
    }
    rhs[e] = b;
  }
}

// Projection (Eq. rkforc1): K_q <- K_q - dt (Grad_b p)_q, q^(k) = q^(k-1) + beta K_q.
__device__ inline void stage_project_body(long t0, long ts, StageArgs a, const double* WT_DEV_RESTRICT px, const double* WT_DEV_RESTRICT py,
                                const double* WT_DEV_RESTRICT Dp, double* WT_DEV_RESTRICT Ku,
                                double* WT_DEV_RESTRICT Kv, double* WT_DEV_RESTRICT Kw,
                                double* WT_DEV_RESTRICT u, double* WT_DEV_RESTRICT v, double* WT_DEV_RESTRICT w,
                                int* flag) {
  const long n = (long)a.M1 * a.ncols;
  const long nc = a.ncols;
  for (long e = t0; e < n; e += ts) {
    const int m = (int)(e / nc);
    const long c = e - m * nc;
    const double s = a.sigma[m];
    const double* meta = a.meta;
    const double sxb = meta[M_AXb * nc + c] - s * meta[M_BXb * nc + c];
    const double Zb = meta[M_Zb * nc + c];
    const double Gx = px[e] + sxb * Dp[e];
    const double Gz = Zb * Dp[e];
    const double ku = Ku[e] - a.dt * Gx, kw = Kw[e] - a.dt * Gz;
    Ku[e] = ku;
    Kw[e] = kw;
    const double un = u[e] + a.beta * ku, wn = w[e] + a.beta * kw;
    u[e] = un;
    w[e] = wn;
    bool bad = !isfinite(un) || !isfinite(wn);
    if (v) {
      const double syb = meta[M_AYb * nc + c] - s * meta[M_BYb * nc + c];
      const double Gy = py[e] + syb * Dp[e];
      const double kv = Kv[e] - a.dt * Gy;
      Kv[e] = kv;
      const double vn = v[e] + a.beta * kv;
      v[e] = vn;
      bad = bad || !isfinite(vn);
    }
    if (bad) atomicOr(flag, 8);
  }
}

}  // namespace wt
