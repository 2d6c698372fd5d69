// Multi-right-hand-side supernodal solve with the nested-dissection LDL^T factor of
// the slab matrix (eq. StandardSmoother applies A_slab^{-1} to every slab at once;
// every slab of a time level shares one factor, Section 2.1) and of K_n
// (eq. AuxNodalSm).
//
// Per supernode s with columns [col0, col0+nc), below-structure rows (nr of
// them) and W_s = [L11^{-1}; -L21 L11^{-1}]:
//   forward  (leaves -> root):  f = Q[cols] + children's update rows;
//                               z_s = D^{-1} (L11^{-1} f),  u_s = f_r - L21 L11^{-1} f
//   backward (root -> leaves):  x_s = W_s^T [z_s ; x(rows)]
// Nodes of one tree depth are independent, so each depth is one launch over
// (node, row tile) x (right-hand-side tile) blocks.  The right-hand sides are the
// slabs of the level (contiguous in each row), so every operand row is a
// contiguous, coalesced vector.  Arithmetic is FP64 (double or double2 complex).
#include "device.h"

namespace stmg {
namespace {

template <typename T>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
};
template <>
struct Ar<double2> {
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void mac(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
};

constexpr int BM = kSnBM;   // rows of W per block
constexpr int BK = 16;      // depth of one shared-memory stage
constexpr int NT = 256;     // threads: 16 x 16, micro-tile rows ty + 16 i, cols tx + 16 j
constexpr int TM = BM / 16;

template <typename T, int BN>
__global__ void __launch_bounds__(NT) k_sn_forward(const DevNode* __restrict__ nodes, const T* __restrict__ W,
                                                   const T* __restrict__ Dinv, const int32_t* __restrict__ gsrc,
                                                   const int2* __restrict__ tiles, const T* __restrict__ Q,
                                                   T* __restrict__ Z, T* __restrict__ U, int nrhs, int ld) {
  constexpr int TN = BN / 16;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int2 tl = tiles[blockIdx.x];
  const DevNode nd = nodes[tl.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int row0 = tl.y * BM, c0 = blockIdx.y * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* Ws = W + nd.w_off;
  const int32_t* gs = gsrc + nd.g_off * 2;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Ar<T>::zero();
  // rows inside L11^{-1} (lower triangular) need no columns beyond the row
  const int kmax = (row0 + BM <= nc) ? (row0 + BM) : nc;
  for (int k0 = 0; k0 < kmax; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      const int i = t / BK, kk = t % BK;
      const int r = row0 + i, k = k0 + kk;
      As[kk][i] = (r < m && k < nc) ? Ws[(int64_t)r * nc + k] : Ar<T>::zero();
    }
    for (int t = threadIdx.x; t < BK * BN; t += NT) {
      const int kk = t / BN, j = t % BN;
      const int k = k0 + kk, c = c0 + j;
      T v = Ar<T>::zero();
      if (k < nc && c < nrhs) {
        v = Q[(int64_t)(nd.col0 + k) * ld + c];
        const int s0 = gs[2 * k], s1 = gs[2 * k + 1];
        if (s0 >= 0) v = Ar<T>::add(v, U[(int64_t)s0 * ld + c]);
        if (s1 >= 0) v = Ar<T>::add(v, U[(int64_t)s1 * ld + c]);
      }
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) Ar<T>::mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c >= nrhs) continue;
      if (r < nc) {
        Z[(int64_t)(nd.col0 + r) * ld + c] = Ar<T>::mul(Dinv[nd.col0 + r], acc[i][j]);
      } else {
        T v = acc[i][j];
        const int s0 = gs[2 * r], s1 = gs[2 * r + 1];
        if (s0 >= 0) v = Ar<T>::add(v, U[(int64_t)s0 * ld + c]);
        if (s1 >= 0) v = Ar<T>::add(v, U[(int64_t)s1 * ld + c]);
        U[(int64_t)(nd.u_off + r - nc) * ld + c] = v;
      }
    }
  }
}

template <typename T, int BN>
__global__ void __launch_bounds__(NT) k_sn_backward(const DevNode* __restrict__ nodes, const T* __restrict__ W,
                                                    const int32_t* __restrict__ rows,
                                                    const int2* __restrict__ tiles, const T* __restrict__ Z,
                                                    T* __restrict__ X, int nrhs, int ld) {
  constexpr int TN = BN / 16;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int2 tl = tiles[blockIdx.x];
  const DevNode nd = nodes[tl.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int row0 = tl.y * BM, c0 = blockIdx.y * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* Ws = W + nd.w_off;
  const int32_t* rw = rows + nd.row_off;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Ar<T>::zero();
  // W[k][i] = 0 for k < i inside L11^{-1}: start at the tile's first row
  const int kmin = (row0 / BK) * BK;
  for (int k0 = kmin; k0 < m; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      const int i = t % BM, kk = t / BM;
      const int r = row0 + i, k = k0 + kk;
      As[kk][i] = (r < nc && k < m) ? Ws[(int64_t)k * nc + r] : Ar<T>::zero();
    }
    for (int t = threadIdx.x; t < BK * BN; t += NT) {
      const int kk = t / BN, j = t % BN;
      const int k = k0 + kk, c = c0 + j;
      T v = Ar<T>::zero();
      if (k < m && c < nrhs) {
        const int64_t src = (k < nc) ? (int64_t)(nd.col0 + k) : (int64_t)rw[k - nc];
        v = (k < nc) ? Z[src * ld + c] : X[src * ld + c];
      }
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) Ar<T>::mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= nc) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < nrhs) X[(int64_t)(nd.col0 + r) * ld + c] = acc[i][j];
    }
  }
}

template <typename T, int BN>
cudaError_t sn_solve_impl(const DevFactor<T>& F, T* Q, T* Z, T* U, int nrhs, int ld, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  const unsigned gy = (unsigned)((nrhs + BN - 1) / BN);
  for (int d = F.max_depth; d >= 0; --d) {
    const int64_t a = F.h_fwd_off[d], b = F.h_fwd_off[d + 1];
    if (b > a)
      { k_sn_forward<T, BN><<<dim3((unsigned)(b - a), gy), NT, 0, st>>>(F.nodes, F.W, F.Dinv, F.gsrc,
                                                                       F.fwd_tiles + a, Q, Z, U, nrhs, ld); count_launches(1); }
  }
  for (int d = 0; d <= F.max_depth; ++d) {
    const int64_t a = F.h_bwd_off[d], b = F.h_bwd_off[d + 1];
    if (b > a)
      { k_sn_backward<T, BN><<<dim3((unsigned)(b - a), gy), NT, 0, st>>>(F.nodes, F.W, F.rows, F.bwd_tiles + a, Z,
                                                                        Q, nrhs, ld); count_launches(1); }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t sn_solve_real(const DevFactor<double>& F, double* Q, double* Z, double* U, int nrhs, int ld,
                          cudaStream_t st) {
  return sn_solve_impl<double, 64>(F, Q, Z, U, nrhs, ld, st);
}
cudaError_t sn_solve_cplx(const DevFactor<double2>& F, double2* Q, double2* Z, double2* U, int nrhs, int ld,
                          cudaStream_t st) {
  return sn_solve_impl<double2, 32>(F, Q, Z, U, nrhs, ld, st);
}

}  // namespace stmg
