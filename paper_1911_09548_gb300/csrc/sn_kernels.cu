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


// ---------------------------------------------------------------- split-K path
// With few right-hand sides (coarse time levels have 1..16 slabs) a 64 x 32 tile
// per block leaves most of the GPU idle and the top supernodes serialise on their
// long K loops.  Here every item is kSkRows rows x one K chunk of kSkK columns for
// all right-hand sides (one row per thread, NB accumulators); a second kernel sums
// the chunks of each row in a fixed order and applies the epilogue.
constexpr int SK_THREADS = kSkRows;
constexpr int SK_KS = 16;   // K columns staged in shared memory at a time

template <typename T, int NB, bool FWD>
__global__ void __launch_bounds__(SK_THREADS) k_sn_skinny_partial(
    const DevNode* __restrict__ nodes, const T* __restrict__ W, const int32_t* __restrict__ gsrc,
    const int32_t* __restrict__ rows, const int4* __restrict__ items, const T* __restrict__ Q,
    const T* __restrict__ Z, const T* __restrict__ U, const T* __restrict__ X, T* __restrict__ P, int nrhs, int ld) {
  __shared__ T As[SK_KS][kSkRows];
  __shared__ T Bs[SK_KS][NB];
  const int4 it = items[blockIdx.x];
  const DevNode nd = nodes[it.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int r0 = it.y, k0 = it.z, k1 = it.w;
  const int tid = threadIdx.x;
  const int cb = blockIdx.y * NB;           // first right-hand side of this column block
  const T* Ws = W + nd.w_off;
  const int32_t* gs = gsrc + nd.g_off * 2;
  const int32_t* rw = rows + nd.row_off;
  T acc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] = Ar<T>::zero();
  for (int ks = k0; ks < k1; ks += SK_KS) {
    for (int t = tid; t < SK_KS * kSkRows; t += SK_THREADS) {
      int i, kk;
      if (FWD) { i = t / SK_KS; kk = t % SK_KS; }     // W row-major: k fastest
      else { i = t % kSkRows; kk = t / kSkRows; }     // W^T: row index fastest
      const int r = r0 + i, k = ks + kk;
      T a = Ar<T>::zero();
      if (FWD) { if (r < m && k < k1) a = Ws[(int64_t)r * nc + k]; }
      else { if (r < nc && k < k1) a = Ws[(int64_t)k * nc + r]; }
      As[kk][i] = a;
    }
    for (int t = tid; t < SK_KS * NB; t += SK_THREADS) {
      const int kk = t / NB, cl = t % NB, c = cb + cl;
      const int k = ks + kk;
      T v = Ar<T>::zero();
      if (k < k1 && c < nrhs) {
        if (FWD) {
          v = Q[(int64_t)(nd.col0 + k) * ld + c];
          const int s0 = gs[2 * k], s1 = gs[2 * k + 1];
          if (s0 >= 0) v = Ar<T>::add(v, U[(int64_t)s0 * ld + c]);
          if (s1 >= 0) v = Ar<T>::add(v, U[(int64_t)s1 * ld + c]);
        } else {
          v = (k < nc) ? Z[(int64_t)(nd.col0 + k) * ld + c] : X[(int64_t)rw[k - nc] * ld + c];
        }
      }
      Bs[kk][cl] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK_KS; ++kk) {
      const T a = As[kk][tid];
#pragma unroll
      for (int j = 0; j < NB; ++j) Ar<T>::mac(acc[j], a, Bs[kk][j]);
    }
    __syncthreads();
  }
  T* out = P + (((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kSkRows + tid) * NB;
#pragma unroll
  for (int j = 0; j < NB; ++j) out[j] = acc[j];
}

// One block per unit (node, row0, item range): thread (row, column) sums the
// unit's items in order, then the forward or backward epilogue.
template <typename T, int NB, bool FWD>
__global__ void __launch_bounds__(kSkRows * NB) k_sn_skinny_reduce(
    const DevNode* __restrict__ nodes, const T* __restrict__ Dinv, const int32_t* __restrict__ gsrc,
    const int4* __restrict__ units, int64_t item_base, int64_t n_items, const T* __restrict__ P,
    T* __restrict__ Z, T* __restrict__ U, T* __restrict__ X, int nrhs, int ld) {
  const int4 un = units[blockIdx.x];
  const DevNode nd = nodes[un.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int i = threadIdx.x / NB, cl = threadIdx.x % NB, c = blockIdx.y * NB + cl;
  const int r = un.y + i;
  if (c >= nrhs) return;
  const T* Pc = P + (int64_t)blockIdx.y * n_items * kSkRows * NB;
  T acc = Ar<T>::zero();
  for (int q = un.z; q < un.w; ++q) acc = Ar<T>::add(acc, Pc[(((int64_t)(q - item_base)) * kSkRows + i) * NB + cl]);
  if (FWD) {
    if (r >= m) return;
    if (r < nc) {
      Z[(int64_t)(nd.col0 + r) * ld + c] = Ar<T>::mul(Dinv[nd.col0 + r], acc);
    } else {
      const int32_t* gs = gsrc + nd.g_off * 2;
      const int s0 = gs[2 * r], s1 = gs[2 * r + 1];
      if (s0 >= 0) acc = Ar<T>::add(acc, U[(int64_t)s0 * ld + c]);
      if (s1 >= 0) acc = Ar<T>::add(acc, U[(int64_t)s1 * ld + c]);
      U[(int64_t)(nd.u_off + r - nc) * ld + c] = acc;
    }
  } else {
    if (r < nc) X[(int64_t)(nd.col0 + r) * ld + c] = acc;
  }
}

template <typename T, int NB>
void skinny_depth(const DevFactor<T>& F, int d, bool fwd, T* Q, T* Z, T* U, T* P, int nrhs, int ld,
                  cudaStream_t st) {
  const int64_t* io = fwd ? F.h_fs_item_off : F.h_bs_item_off;
  const int64_t* uo = fwd ? F.h_fs_unit_off : F.h_bs_unit_off;
  const int64_t ia = io[d], ib = io[d + 1], ua = uo[d], ub = uo[d + 1];
  if (ib <= ia) return;
  const unsigned gy = (unsigned)((nrhs + NB - 1) / NB);
  if (fwd) {
    k_sn_skinny_partial<T, NB, true><<<dim3((unsigned)(ib - ia), gy), SK_THREADS, 0, st>>>(
        F.nodes, F.W, F.gsrc, F.rows, F.fs_items + ia, Q, Z, U, Q, P, nrhs, ld);
    k_sn_skinny_reduce<T, NB, true><<<dim3((unsigned)(ub - ua), gy), kSkRows * NB, 0, st>>>(
        F.nodes, F.Dinv, F.gsrc, F.fs_units + ua, ia, ib - ia, P, Z, U, Q, nrhs, ld);
  } else {
    k_sn_skinny_partial<T, NB, false><<<dim3((unsigned)(ib - ia), gy), SK_THREADS, 0, st>>>(
        F.nodes, F.W, F.gsrc, F.rows, F.bs_items + ia, Q, Z, U, Q, P, nrhs, ld);
    k_sn_skinny_reduce<T, NB, false><<<dim3((unsigned)(ub - ua), gy), kSkRows * NB, 0, st>>>(
        F.nodes, F.Dinv, F.gsrc, F.bs_units + ua, ia, ib - ia, P, Z, U, Q, nrhs, ld);
  }
  count_launches(2);
}

template <typename T, int NB>
cudaError_t sn_solve_skinny(const DevFactor<T>& F, T* Q, T* Z, T* U, T* P, int nrhs, int ld, cudaStream_t st) {
  for (int d = F.max_depth; d >= 0; --d) skinny_depth<T, NB>(F, d, true, Q, Z, U, P, nrhs, ld, st);
  for (int d = 0; d <= F.max_depth; ++d) skinny_depth<T, NB>(F, d, false, Q, Z, U, P, nrhs, ld, st);
  return cudaGetLastError();
}

// Tiled products for many right-hand sides; a depth whose tile grid would not
// fill two waves of the GPU (the few large supernodes near the root) goes through
// the split-K kernels instead, with NBK right-hand sides per column block.
template <typename T, int BN, int NBK>
cudaError_t sn_solve_impl(const DevFactor<T>& F, T* Q, T* Z, T* U, T* P, int nrhs, int ld, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  const unsigned gy = (unsigned)((nrhs + BN - 1) / BN);
  const int64_t two_waves = 2 * (int64_t)F.n_sm;
  for (int d = F.max_depth; d >= 0; --d) {
    const int64_t a = F.h_fwd_off[d], b = F.h_fwd_off[d + 1];
    if (b <= a) continue;
    if (P && (b - a) * gy < two_waves) {
      skinny_depth<T, NBK>(F, d, true, Q, Z, U, P, nrhs, ld, st);
      continue;
    }
    { k_sn_forward<T, BN><<<dim3((unsigned)(b - a), gy), NT, 0, st>>>(F.nodes, F.W, F.Dinv, F.gsrc,
                                                                       F.fwd_tiles + a, Q, Z, U, nrhs, ld); count_launches(1); }
  }
  for (int d = 0; d <= F.max_depth; ++d) {
    const int64_t a = F.h_bwd_off[d], b = F.h_bwd_off[d + 1];
    if (b <= a) continue;
    if (P && (b - a) * gy < two_waves) {
      skinny_depth<T, NBK>(F, d, false, Q, Z, U, P, nrhs, ld, st);
      continue;
    }
    { k_sn_backward<T, BN><<<dim3((unsigned)(b - a), gy), NT, 0, st>>>(F.nodes, F.W, F.rows, F.bwd_tiles + a, Z,
                                                                        Q, nrhs, ld); count_launches(1); }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t sn_solve_real(const DevFactor<double>& F, double* Q, double* Z, double* U, double* P, int nrhs, int ld,
                          cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (P && nrhs <= 4) return sn_solve_skinny<double, 4>(F, Q, Z, U, P, nrhs, ld, st);
  if (P && nrhs <= 16) return sn_solve_skinny<double, 16>(F, Q, Z, U, P, nrhs, ld, st);
  if (P && nrhs <= kSkMaxRhsR) return sn_solve_skinny<double, kSkMaxRhsR>(F, Q, Z, U, P, nrhs, ld, st);
  return sn_solve_impl<double, 64, kSkMaxRhsR>(F, Q, Z, U, P, nrhs, ld, st);
}
cudaError_t sn_solve_cplx(const DevFactor<double2>& F, double2* Q, double2* Z, double2* U, double2* P, int nrhs,
                          int ld, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (P && nrhs <= 2) return sn_solve_skinny<double2, 2>(F, Q, Z, U, P, nrhs, ld, st);
  if (P && nrhs <= 8) return sn_solve_skinny<double2, 8>(F, Q, Z, U, P, nrhs, ld, st);
  if (P && nrhs <= kSkMaxRhsC) return sn_solve_skinny<double2, kSkMaxRhsC>(F, Q, Z, U, P, nrhs, ld, st);
  return sn_solve_impl<double2, 32, kSkMaxRhsC>(F, Q, Z, U, P, nrhs, ld, st);
}

}  // namespace stmg
