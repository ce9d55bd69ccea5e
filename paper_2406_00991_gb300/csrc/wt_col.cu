// Column (sigma-direction) kernels, one warp per vertical column (bodies in
// wt_dev.cuh).
//
//  k_op_cols      the sigma part of A_{a,b} (Eq. 1_chain, poissonp, bcpdneu):
//                 P_s = D p, G = (P_x + sx_b P_s, P_y + sy_b P_s, Z_b P_s),
//                 part = sx_a D G_x + sy_a D G_y + Z_a Z_b D P_s (interior),
//                 p (surface row), h_x G_x + h_y G_y + Z_b P_s (bottom row).
//  k_smooth_cols  damped block-Jacobi update x += omega sum_class B_class^{-1} r_class
//                 (Sec. 4.3, Nyquist-split column blocks).
//  k_col_matrix   out = M in along sigma (Chebyshev transfers of Sec. 4.2, filter).
//  k_block_inverse_multi  builds and inverts the (Nz+1)^2 diagonal block of
//                 every column of every level by Gauss-Jordan with partial
//                 pivoting, one warp per (column, class), all levels in one launch.
#include "wt_dev.cuh"

#include <algorithm>

namespace wt {

template <typename T, int DIM, int KM>
__global__ void __launch_bounds__(256) k_op_cols(LevelView<T> L, const T* __restrict__ p,
                                                 const T* __restrict__ Px, const T* __restrict__ Py,
                                                 T* __restrict__ Gx, T* __restrict__ Gy,
                                                 T* __restrict__ part) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  opcols_body<T, DIM, KM>(L, p, Px, Py, Gx, Gy, part, blockIdx.x, gridDim.x, smraw);
}

template <typename T, int DIM, int MAXM>
__global__ void __launch_bounds__(128) k_op_cols_tpc(LevelView<T> L, const T* __restrict__ p,
                                                     const T* __restrict__ Px, const T* __restrict__ Py,
                                                     T* __restrict__ Gx, T* __restrict__ Gy,
                                                     T* __restrict__ part) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  opcols_tpc_body<T, DIM, MAXM>(L, p, Px, Py, Gx, Gy, part, smraw);
}

template <typename T>
__global__ void __launch_bounds__(256) k_op_cols_T(LevelView<T> L, const T* __restrict__ lam,
                                                   const T* __restrict__ Dlam, T* __restrict__ Mx,
                                                   T* __restrict__ part) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  opcolsT_body<T>(L, lam, Dlam, Mx, part, blockIdx.x, gridDim.x, smraw);
}

// One instantiation per column-length bucket (MAXM >= M1, chosen on the
// host): a kernel holding every bucket would be register-allocated for the
// largest one.
template <typename T, int DIM, bool TR, int MAXM, bool EXACT>
__global__ void __launch_bounds__(256) k_smooth_cols(LevelView<T> L, const T* __restrict__ r,
                                                     const T* __restrict__ rhoX,
                                                     const T* __restrict__ rhoY,
                                                     const T* __restrict__ rhoXY,
                                                     const T* __restrict__ Binv,
                                                     T* __restrict__ x, T omega, int first) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  smooth_body<T, DIM, MAXM, TR, EXACT>(L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first, blockIdx.x, gridDim.x, smraw);
}

// out = M in (accumulate: out += M in) column by column with one thread per
// column: the column's Mi values in registers, M (Mo x Mi, row-major) in
// shared memory read as warp-wide broadcasts, loads and stores coalesced
// across the threads' consecutive columns.  Every input of a column is read
// before its first output is written, so out may be in (the filter).
template <typename T, int MI>
__global__ void __launch_bounds__(128) k_col_matrix_tpc(const T* __restrict__ M, int Mo, const T* in,
                                                        T* out, int ncols, int accumulate) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sM = reinterpret_cast<T*>(smraw);
  for (int i = threadIdx.x; i < Mo * MI; i += blockDim.x) sM[i] = M[i];
  __syncthreads();
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long nc = ncols;
  T v[MI];
#pragma unroll
  for (int j = 0; j < MI; ++j) v[j] = in[j * nc + c];
  for (int i = 0; i < Mo; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < MI; ++j) acc = fma(sM[i * MI + j], v[j], acc);
    const long o = i * nc + c;
    out[o] = accumulate ? out[o] + acc : acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_col_matrix(const T* __restrict__ M, int Mo, int Mi,
                                                    const T* __restrict__ in, T* __restrict__ out,
                                                    int ncols, int accumulate) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  colmat_body<T>(M, Mo, Mi, in, out, ncols, accumulate, blockIdx.x, gridDim.x, smraw);
}

// Every level's (column, class) tasks in one launch: the levels' inverses
// cost one level's latency (a warp's Gauss-Jordan) instead of the sum.
template <typename T>
__global__ void __launch_bounds__(128) k_block_inverse_multi(const __grid_constant__ BlockInvMulti<T> m, int* flag) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* A = reinterpret_cast<T*>(smraw) + wib * (m.maxM1 * (2 * m.maxM1 + 1));
  const long total = m.start[m.nlev];
  for (long g = (long)blockIdx.x * nw + wib; g < total; g += (long)gridDim.x * nw) {
    int l = 0;
    while (g >= m.start[l + 1]) ++l;
    blockinv_task<T>(m.L[l], m.Binv[l], m.nclass[l], m.cxx[l], m.cyy[l], flag, g - m.start[l], A);
  }
}

// ------------------------------------------------------------------ launchers
static inline int grid_for(long n, int bs) { return (int)std::max<long>(1, (n + bs - 1) / bs); }

template <typename T>
static cudaError_t set_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Levels with at least this many columns use the thread-per-column sigma
// operator (k_op_cols_tpc) when M1 <= 17.
constexpr long kTpcMinCols = 8192;

static inline int grid_cols(long ncols, int threads) {
  const long w = threads / 32;
  return (int)std::min<long>(std::max<long>(1, (ncols + w - 1) / w), (long)sm_count() * 64);
}

// Warp-per-column operator with the column length fixed at compile time where
// it is one of the common lengths (Nz = 4, 6, 8, 12, 16, 24, 32), else read
// from the level.
template <typename T, int DIM>
static cudaError_t launch_op_cols_m(const LevelView<T>& L, int g, size_t smem, cudaStream_t s, const T* p,
                                    const T* Px, const T* Py, T* Gx, T* Gy, T* part) {
#define WT_OPC(KM) launch_k(k_op_cols<T, DIM, KM>, dim3(g), dim3(256), smem, s, L, p, Px, Py, Gx, Gy, part)
  switch (L.M1) {
    case 5: return WT_OPC(5);
    case 7: return WT_OPC(7);
    case 9: return WT_OPC(9);
    case 13: return WT_OPC(13);
    case 17: return WT_OPC(17);
    case 25: return WT_OPC(25);
    case 33: return WT_OPC(33);
    default: return WT_OPC(0);
  }
#undef WT_OPC
}

template <typename T>
cudaError_t launch_op_cols(const LevelView<T>& L, const T* p, const T* Px, const T* Py, T* Gx,
                           T* Gy, T* part, cudaStream_t s, int df) {
  if constexpr (sizeof(T) == 8) {
    if (df && L.ncols >= kTpcMinCols && col_df_fits(L.M1))
      return launch_op_cols_df(L, p, Px, Py, Gx, Gy, part, s);
  }
  (void)df;
  const size_t smem = opcols_smem<T>(L.M1);
  if (L.ncols >= kTpcMinCols && L.M1 <= 17) {
    // many columns: one thread per column, coalesced sigma rows
    const dim3 G((unsigned)((L.ncols + 127) / 128)), B(128);
    if (L.Ny == 1) {
      if (L.M1 <= 9) return launch_k(k_op_cols_tpc<T, 2, 9>, G, B, smem, s, L, p, Px, Py, Gx, Gy, part);
      return launch_k(k_op_cols_tpc<T, 2, 17>, G, B, smem, s, L, p, Px, Py, Gx, Gy, part);
    }
    if (L.M1 <= 9) return launch_k(k_op_cols_tpc<T, 3, 9>, G, B, smem, s, L, p, Px, Py, Gx, Gy, part);
    return launch_k(k_op_cols_tpc<T, 3, 17>, G, B, smem, s, L, p, Px, Py, Gx, Gy, part);
  }
  const int g = grid_cols(L.ncols, 256);
  if (L.Ny == 1) return launch_op_cols_m<T, 2>(L, g, smem, s, p, Px, Py, Gx, Gy, part);
  return launch_op_cols_m<T, 3>(L, g, smem, s, p, Px, Py, Gx, Gy, part);
}

template <typename T>
cudaError_t launch_op_cols_T(const LevelView<T>& L, const T* lam, const T* Dlam, T* Mx, T* part,
                             cudaStream_t s) {
  if (L.Ny != 1) return cudaErrorInvalidValue;
  const int g = grid_cols(L.ncols, 256);
  return launch_k(k_op_cols_T<T>, dim3(g), dim3(256), opcols_smem<T>(L.M1), s, L, lam, Dlam, Mx, part);
}

template <typename T, int DIM, bool TR>
static cudaError_t launch_smooth_m(const LevelView<T>& L, dim3 G, dim3 B, cudaStream_t s, const T* r, const T* rhoX,
                                   const T* rhoY, const T* rhoXY, const T* Binv, T* x, T omega, int first) {
#define WT_SMOOTH(MM, EX) \
  launch_k(k_smooth_cols<T, DIM, TR, MM, EX>, G, B, 0, s, L, r, rhoX, rhoY, rhoXY, Binv, x, omega, first)
  switch (L.M1) {                           // the common column lengths: exact
    case 5: return WT_SMOOTH(5, true);
    case 7: return WT_SMOOTH(7, true);
    case 9: return WT_SMOOTH(9, true);
    case 13: return WT_SMOOTH(13, true);
    case 17: return WT_SMOOTH(17, true);
    case 25: return WT_SMOOTH(25, true);
    case 33: return WT_SMOOTH(33, true);
    default: break;
  }
  if (L.M1 <= 9) return WT_SMOOTH(9, false);
  if (L.M1 <= 17) return WT_SMOOTH(17, false);
  if (L.M1 <= 25) return WT_SMOOTH(25, false);
  return WT_SMOOTH(33, false);
#undef WT_SMOOTH
}

template <typename T>
cudaError_t launch_smooth_cols(const LevelView<T>& L, const T* r, const T* rhoX, const T* rhoY,
                               const T* rhoXY, const T* Binv, int nclass, T* x, T omega, int first,
                               int tr, cudaStream_t s) {
  (void)nclass;
  const int g = grid_cols(L.ncols, 256);
  const dim3 G(g), B(256);
  if (L.Ny == 1) {
    if (tr) return launch_smooth_m<T, 2, true>(L, G, B, s, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
    return launch_smooth_m<T, 2, false>(L, G, B, s, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
  }
  if (tr) return launch_smooth_m<T, 3, true>(L, G, B, s, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
  return launch_smooth_m<T, 3, false>(L, G, B, s, r, rhoX, rhoY, rhoXY, Binv, x, omega, first);
}

template <typename T>
cudaError_t launch_col_matrix(const T* M, int Mo, int Mi, const T* in, T* out, int ncols,
                              int accumulate, cudaStream_t s, int df) {
  if constexpr (sizeof(T) == 8) {
    if (df && ncols >= kTpcMinCols && Mo <= kMaxM1 && col_df_fits(Mi))
      return launch_col_matrix_df(M, Mo, Mi, in, out, ncols, accumulate, s);
  }
  (void)df;
  if (ncols >= kTpcMinCols && Mo <= kMaxM1) {
    // many columns (3D levels): one thread per column
    const dim3 G((unsigned)((ncols + 127) / 128)), B(128);
    const size_t sm = sizeof(T) * (size_t)Mo * Mi;
#define WT_CMT(MI) launch_k(k_col_matrix_tpc<T, MI>, G, B, sm, s, M, Mo, in, out, ncols, accumulate)
    switch (Mi) {
      case 5: return WT_CMT(5);
      case 9: return WT_CMT(9);
      case 13: return WT_CMT(13);
      case 17: return WT_CMT(17);
      case 25: return WT_CMT(25);
      case 33: return WT_CMT(33);
      default: break;
    }
#undef WT_CMT
  }
  const int g = grid_cols(ncols, 256);
  const size_t smem = sizeof(T) * (size_t)Mo * Mi;
  return launch_k(k_col_matrix<T>, dim3(g), dim3(256), smem, s, M, Mo, Mi, in, out, ncols, accumulate);
}

template <typename T>
cudaError_t launch_block_inverse_multi(const BlockInvMulti<T>& m, int* flag, cudaStream_t s) {
  if (m.nlev <= 0) return cudaSuccess;
  const int W = 2 * m.maxM1 + 1;
  const size_t smem = 4 * (size_t)m.maxM1 * W * sizeof(T);
  if (smem > 32 * 1024) {
    cudaError_t e = ensure_dyn_smem((const void*)k_block_inverse_multi<T>, smem);
    if (e != cudaSuccess) return e;
  }
  const long total = m.start[m.nlev];
  const int g = (int)std::min<long>(std::max<long>(1, (total + 3) / 4), sm_count() * 8);
  return launch_k(k_block_inverse_multi<T>, dim3(g), dim3(128), smem, s, m, flag);
}

#define WT_INST(T)                                                                              \
  template cudaError_t launch_op_cols<T>(const LevelView<T>&, const T*, const T*, const T*, T*,  \
                                         T*, T*, cudaStream_t, int);                            \
  template cudaError_t launch_smooth_cols<T>(const LevelView<T>&, const T*, const T*, const T*,  \
                                             const T*, const T*, int, T*, T, int, int,          \
                                             cudaStream_t);                                      \
  template cudaError_t launch_op_cols_T<T>(const LevelView<T>&, const T*, const T*, T*, T*,      \
                                           cudaStream_t);                                        \
  template cudaError_t launch_col_matrix<T>(const T*, int, int, const T*, T*, int, int,         \
                                            cudaStream_t, int);                                 \
  template cudaError_t launch_block_inverse_multi<T>(const BlockInvMulti<T>&, int*, cudaStream_t);
WT_INST(float)
WT_INST(double)

}  // namespace wt
