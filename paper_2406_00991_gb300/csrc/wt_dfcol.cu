// FP64 sigma-column kernels for levels with many columns (3D) in
// double-float arithmetic (wt_ff.cuh): the sigma part of A_{a,b} (Eq. 1_chain
// with the Chebyshev derivative D of Sec. 3.5) and the plain column-matrix
// product (the sigma derivative and the Chebyshev filter of a stage).  Data
// stay FP64 in memory; each FP64 value is split into a float pair on load
// and recombined on store, and every product-sum runs on the FP32 units,
// which GB300 runs at 64 times its FP64 rate.  The expressions are those of
// the FP64 kernels (opcols_tpc_body, k_col_matrix_tpc), one thread per column.
#include "wt_dev.cuh"
#include "wt_ff.cuh"

namespace wt {

namespace {

// acc + a b: the two-product of the leading parts with both cross terms in
// its error, then a normalised double-float sum.
__device__ __forceinline__ ff ff_mac(ff acc, ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const ff s = ff_two_sum(acc.hi, p);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}

__device__ __forceinline__ ff ld(const double* p, long i) { return to_arith<ff, double>(p[i]); }
__device__ __forceinline__ double st(ff v) { return from_arith<double, ff>(v); }

}  // namespace

// out = M in (accumulate: out += M in), M (Mo x MI) row-major; out may be in.
template <int MI>
__global__ void __launch_bounds__(128) k_col_matrix_df(const double* __restrict__ M, int Mo, const double* in,
                                                       double* out, int ncols, int accumulate) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  ff* sM = reinterpret_cast<ff*>(smraw);
  for (int i = threadIdx.x; i < Mo * MI; i += blockDim.x) sM[i] = to_arith<ff, double>(M[i]);
  __syncthreads();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long nc = ncols;
  ff v[MI];
#pragma unroll
  for (int j = 0; j < MI; ++j) v[j] = ld(in, j * nc + c);
  for (int i = 0; i < Mo; ++i) {
    ff acc = a_zero<ff>();
#pragma unroll
    for (int j = 0; j < MI; ++j) acc = ff_mac(acc, sM[i * MI + j], v[j]);
    const long o = i * nc + c;
    out[o] = accumulate ? out[o] + st(acc) : st(acc);
  }
}

// The sigma part of A_{a,b} p with one thread per column (the same rows as
// opcols_tpc_body): G_x = P_x + sx_b D p (and G_y), interior rows
// sx_a D G_x + sy_a D G_y + Z_a Z_b D D p, surface row p, bottom row
// n . Grad_b p.  MAXM == M1.
template <int DIM, int MAXM>
__global__ void __launch_bounds__(128) k_op_cols_df(LevelView<double> L, const double* __restrict__ p,
                                                    const double* __restrict__ Px,
                                                    const double* __restrict__ Py, double* __restrict__ Gx,
                                                    double* __restrict__ Gy, double* __restrict__ part) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  ff* sD = reinterpret_cast<ff*>(smraw);
  ff* sS = sD + MAXM * MAXM;
  for (int i = threadIdx.x; i < MAXM * MAXM; i += blockDim.x) sD[i] = to_arith<ff, double>(L.D[i]);
  for (int i = threadIdx.x; i < MAXM; i += blockDim.x) sS[i] = to_arith<ff, double>(L.sigma[i]);
  __syncthreads();
  const long nc = L.ncols;
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double* meta = L.meta;
  ff ps[MAXM], gx[MAXM], gy[DIM == 3 ? MAXM : 1];
  {
    ff pv[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) pv[m] = ld(p, m * nc + c);
    part[c] = p[c];                                                  // surface row: p
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      ff a = a_zero<ff>();
#pragma unroll
      for (int k = 0; k < MAXM; ++k) a = ff_mac(a, sD[m * MAXM + k], pv[k]);
      ps[m] = a;
    }
  }
  const ff AXb = ld(meta, M_AXb * nc + c), BXb = ld(meta, M_BXb * nc + c);
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    gx[m] = ld(Px, m * nc + c) + (AXb - sS[m] * BXb) * ps[m];
    Gx[m * nc + c] = st(gx[m]);
  }
  if constexpr (DIM == 3) {
    const ff AYb = ld(meta, M_AYb * nc + c), BYb = ld(meta, M_BYb * nc + c);
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      gy[m] = ld(Py, m * nc + c) + (AYb - sS[m] * BYb) * ps[m];
      Gy[m * nc + c] = st(gy[m]);
    }
  }
  const ff AXa = ld(meta, M_AXa * nc + c), BXa = ld(meta, M_BXa * nc + c);
  const ff ZZ = ld(meta, M_Za * nc + c) * ld(meta, M_Zb * nc + c);
  // interior rows one at a time (m not unrolled: the row of D and sigma_m
  // come from shared memory, while ps, gx and gy stay in registers)
#pragma unroll 1
  for (int m = 1; m < MAXM - 1; ++m) {
    ff q = a_zero<ff>(), z = a_zero<ff>(), y = a_zero<ff>();
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      const ff d = sD[m * MAXM + k];
      q = ff_mac(q, d, gx[k]);
      z = ff_mac(z, d, ps[k]);
      if constexpr (DIM == 3) y = ff_mac(y, d, gy[k]);
    }
    ff o = (AXa - sS[m] * BXa) * q + ZZ * z;
    if constexpr (DIM == 3) {
      const ff AYa = ld(meta, M_AYa * nc + c), BYa = ld(meta, M_BYa * nc + c);
      o = o + (AYa - sS[m] * BYa) * y;
    }
    part[m * nc + c] = st(o);
  }
  const int N = MAXM - 1;                                            // bottom row: n . Grad_b p
  ff b = ld(meta, M_HX * nc + c) * gx[N] + ld(meta, M_Zb * nc + c) * ps[N];
  if constexpr (DIM == 3) b = b + ld(meta, M_HY * nc + c) * gy[N];
  part[N * nc + c] = st(b);
}

bool col_df_fits(int M1) { return M1 == 5 || M1 == 9 || M1 == 13 || M1 == 17; }

cudaError_t launch_col_matrix_df(const double* M, int Mo, int Mi, const double* in, double* out, int ncols,
                                 int accumulate, cudaStream_t s) {
  const dim3 G((unsigned)((ncols + 127) / 128)), B(128);
  const size_t sm = sizeof(ff) * (size_t)Mo * Mi;
  switch (Mi) {
    case 5: return launch_k(k_col_matrix_df<5>, G, B, sm, s, M, Mo, in, out, ncols, accumulate);
    case 9: return launch_k(k_col_matrix_df<9>, G, B, sm, s, M, Mo, in, out, ncols, accumulate);
    case 13: return launch_k(k_col_matrix_df<13>, G, B, sm, s, M, Mo, in, out, ncols, accumulate);
    case 17: return launch_k(k_col_matrix_df<17>, G, B, sm, s, M, Mo, in, out, ncols, accumulate);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_op_cols_df(const LevelView<double>& L, const double* p, const double* Px, const double* Py,
                              double* Gx, double* Gy, double* part, cudaStream_t s) {
  const dim3 G((unsigned)((L.ncols + 127) / 128)), B(128);
  const size_t sm = sizeof(ff) * ((size_t)L.M1 * L.M1 + L.M1);
#define WT_OPDF(DIM, M) launch_k(k_op_cols_df<DIM, M>, G, B, sm, s, L, p, Px, Py, Gx, Gy, part)
  if (L.Ny == 1) {
    switch (L.M1) {
      case 5: return WT_OPDF(2, 5);
      case 9: return WT_OPDF(2, 9);
      case 13: return WT_OPDF(2, 13);
      case 17: return WT_OPDF(2, 17);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.M1) {
    case 5: return WT_OPDF(3, 5);
    case 9: return WT_OPDF(3, 9);
    case 13: return WT_OPDF(3, 13);
    case 17: return WT_OPDF(3, 17);
    default: return cudaErrorInvalidValue;
  }
#undef WT_OPDF
}

}  // namespace wt
