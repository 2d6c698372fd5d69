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
// contiguous, coalesced vector.
//
// Arithmetic policies (template parameter P):
//   PolNative<T>  T = double / double2 / float / float2: storage = arithmetic.
//   PolDF / PolDFC: FP64-accurate "double-float" arithmetic for GB300, whose FP64
//     pipe runs at 1/58 of its FP32 pipe.  W is stored as (hi, lo) FP32 pairs,
//     right-hand sides stay FP64 in memory and are split on load, products are
//     exact (fma error term) plus the two cross terms, and sums use the
//     error-free two-sum (Knuth), so one multiply-add costs 12 FP32 instructions
//     and keeps ~48 significant bits.  Epilogues (pivots, update sums) run in FP64.
//
// Included by the translation units that instantiate the solves (sn_kernels.cu: FP64,
// sn_mixed.cu: FP32 and real double-float, sn_dfc.cu: complex double-float, sn_tc.cu:
// 16-bit factors), so that they compile in parallel; everything here has internal linkage.
#pragma once

#include <algorithm>
#include <type_traits>

#include "device.h"
#include "launch.cuh"

namespace stmg {
namespace {

// ---------------------------------------------------------------- arithmetic
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
  // one rounded product and one fused multiply-add per part, spelled out so that every
  // kernel rounds the same way
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
  }
};
template <>
struct Ar<float> {
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
};
template <>
struct Ar<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void mac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
  }
};

// Load of a value that another warp of the same kernel may have written (CG: through
// L2 only, never a stale line of this SM's L1 or read-only cache).
template <bool CG, typename S>
__device__ __forceinline__ S ldx(const S* p) {
  if (CG) return __ldcg(p);
  return *p;
}

template <typename T>
struct PolNative {
  using S = T;   // memory type of right-hand sides, updates, pivots
  using WT = T;  // memory type of W
  using A = T;   // arithmetic type
  static __device__ __forceinline__ A zero() { return Ar<T>::zero(); }
  static __device__ __forceinline__ A from_w(WT w) { return w; }
  static __device__ __forceinline__ A from_s(S v) { return v; }
  static __device__ __forceinline__ S to_s(A a) { return a; }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { Ar<T>::mac(acc, a, b); }
};

// FP64 complex products with three real multiplications (Gauss): for y = sum_k a_k b_k
// keep p = sum Re a Re b, q = sum Im a Im b, r = sum (Re a + Im a)(Re b + Im b); then
// Re y = p - q, Im y = r - p - q.  Operands are staged as (Re, Im, Re + Im), the sums
// formed once per staged element and reused across the whole tile, so a complex
// multiply-add costs 3 FP64 FMAs instead of 4 on the FP64 pipe that bounds this path.
struct c3 {
  double x, y, z;
};
struct PolC3M {
  using S = double2;
  using WT = double2;
  using A = c3;
  static __device__ __forceinline__ A zero() { return c3{0.0, 0.0, 0.0}; }
  static __device__ __forceinline__ A from_w(WT w) { return c3{w.x, w.y, w.x + w.y}; }
  static __device__ __forceinline__ A from_s(S v) { return c3{v.x, v.y, v.x + v.y}; }
  static __device__ __forceinline__ S to_s(A a) { return make_double2(a.x - a.y, a.z - a.x - a.y); }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.y = fma(a.y, b.y, acc.y);
    acc.z = fma(a.z, b.z, acc.z);
  }
};

// double-float value h + l
struct dfr {
  float h, l;
};
struct dfc {
  dfr re, im;
};

__device__ __forceinline__ dfr df_split(double v) {
  dfr r;
  r.h = __double2float_rn(v);
  r.l = __double2float_rn(v - (double)r.h);
  return r;
}
__device__ __forceinline__ double df_join(dfr a) { return (double)a.h + (double)a.l; }

// acc += sgn * a * b (sgn = +1 or -1 folded into the first factor).
__device__ __forceinline__ void df_mac(dfr& acc, dfr a, dfr b, float sgn) {
  const float ah = sgn * a.h, al = sgn * a.l;
  const float p = ah * b.h;
  float e = fmaf(ah, b.h, -p);          // exact error of the leading product
  e = fmaf(ah, b.l, e);
  e = fmaf(al, b.h, e);
  const float s = acc.h + p;            // two-sum of the leading parts
  const float bb = s - acc.h;
  const float t = (acc.h - (s - bb)) + (p - bb);
  acc.l = acc.l + (t + e);
  acc.h = s;
}

struct PolDF {
  using S = double;
  using WT = float2;   // (hi, lo)
  using A = dfr;
  static __device__ __forceinline__ A zero() { return dfr{0.f, 0.f}; }
  static __device__ __forceinline__ A from_w(WT w) { return dfr{w.x, w.y}; }
  static __device__ __forceinline__ A from_s(S v) { return df_split(v); }
  static __device__ __forceinline__ S to_s(A a) { return df_join(a); }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { df_mac(acc, a, b, 1.f); }
};

struct PolDFC {
  using S = double2;
  using WT = float4;   // (re hi, re lo, im hi, im lo)
  using A = dfc;
  static __device__ __forceinline__ A zero() { return dfc{dfr{0.f, 0.f}, dfr{0.f, 0.f}}; }
  static __device__ __forceinline__ A from_w(WT w) { return dfc{dfr{w.x, w.y}, dfr{w.z, w.w}}; }
  static __device__ __forceinline__ A from_s(S v) { return dfc{df_split(v.x), df_split(v.y)}; }
  static __device__ __forceinline__ S to_s(A a) { return make_double2(df_join(a.re), df_join(a.im)); }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) {
    df_mac(acc.re, a.re, b.re, 1.f);
    df_mac(acc.re, a.im, b.im, -1.f);
    df_mac(acc.im, a.re, b.im, 1.f);
    df_mac(acc.im, a.im, b.re, 1.f);
  }
};

// BF16 factor, FP32 arithmetic (split-K path of the tensor-core solve)
struct PolBF16C {
  using S = float2;
  using WT = __nv_bfloat162;
  using A = float2;
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ A from_w(WT w) { return __bfloat1622float2(w); }
  static __device__ __forceinline__ A from_s(S v) { return v; }
  static __device__ __forceinline__ S to_s(A a) { return a; }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { Ar<float2>::mac(acc, a, b); }
};

// BF16 factor and right-hand sides rounded to BF16 where they enter a product, FP32
// products and sums: the arithmetic of the tensor-core kernels (whose operand tiles
// hold BF16 copies of the gathered FP32 right-hand sides) on the CUDA cores, as their
// element-wise reference.  Only the FP32 summation order differs.
struct PolBF16CR {
  using S = float2;
  using WT = __nv_bfloat162;
  using A = float2;
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ A from_w(WT w) { return __bfloat1622float2(w); }
  static __device__ __forceinline__ A from_s(S v) { return __bfloat1622float2(__floats2bfloat162_rn(v.x, v.y)); }
  static __device__ __forceinline__ S to_s(A a) { return a; }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { Ar<float2>::mac(acc, a, b); }
};

// FP16 factor, FP32 arithmetic (split-K path of the FP16 tensor-core solve; its
// right-hand-side columns arrive scaled by powers of two, see col_scale)
struct PolF16C {
  using S = float2;
  using WT = __half2;
  using A = float2;
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ A from_w(WT w) { return __half22float2(w); }
  static __device__ __forceinline__ A from_s(S v) { return v; }
  static __device__ __forceinline__ S to_s(A a) { return a; }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { Ar<float2>::mac(acc, a, b); }
};

// ... and with the right-hand sides rounded to FP16 where they enter a product: the
// element-wise reference of the FP16 tensor-core kernels, as PolBF16CR is of the BF16 ones
struct PolF16CR {
  using S = float2;
  using WT = __half2;
  using A = float2;
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ A from_w(WT w) { return __half22float2(w); }
  static __device__ __forceinline__ A from_s(S v) { return __half22float2(__floats2half2_rn(v.x, v.y)); }
  static __device__ __forceinline__ S to_s(A a) { return a; }
  static __device__ __forceinline__ void mac(A& acc, A a, A b) { Ar<float2>::mac(acc, a, b); }
};

constexpr int BK = 16;      // depth of one shared-memory stage
constexpr int NT = 256;     // threads: 16 x 16, micro-tile rows ty + 16 i, cols tx + 16 j

// ---------------------------------------------------------------- tiled path
// BM rows of W (forward) or output rows (backward) per block, BN right-hand sides.  The
// factor's tile lists are built for its BM (DevFactor::bm): 64 for the FP32 / BF16 /
// double-float factors, 16 for the FP64 ones, whose kernels are bound by the FP64 pipe,
// so that small supernodes waste few multiply-adds on padded rows and on the zero
// triangle of L11^{-1} (shared-memory and L2 traffic per multiply-add rise, but far
// below what that pipe's rate leaves room for).
template <typename P, int BN, int BM>
__global__ void __launch_bounds__(NT) k_sn_forward(const DevNode* __restrict__ nodes,
                                                   const typename P::WT* __restrict__ W,
                                                   const typename P::S* __restrict__ Dinv,
                                                   const int32_t* __restrict__ gsrc, const int2* __restrict__ tiles,
                                                   const typename P::S* __restrict__ Q, typename P::S* __restrict__ Z,
                                                   typename P::S* __restrict__ U, int nrhs, int ld) {
  pdl_entry();
  using S = typename P::S;
  using A = typename P::A;
  constexpr int TN = BN / 16;
  constexpr int TM = BM / 16;
  __shared__ A As[BK][BM];
  __shared__ A Bs[BK][BN];
  const int2 tl = tiles[blockIdx.x];
  const DevNode nd = nodes[tl.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int row0 = tl.y * BM, c0 = blockIdx.y * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const typename P::WT* Ws = W + nd.w_off;
  const int32_t* gs = gsrc + nd.g_off * 2;
  A acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = P::zero();
  // rows inside L11^{-1} (lower triangular) need no columns beyond the row
  const int kmax = (row0 + BM <= nc) ? (row0 + BM) : nc;
  for (int k0 = 0; k0 < kmax; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      const int i = t / BK, kk = t % BK;
      const int r = row0 + i, k = k0 + kk;
      As[kk][i] = (r < m && k < nc) ? P::from_w(Ws[(int64_t)r * nc + k]) : P::zero();
    }
    for (int t = threadIdx.x; t < BK * BN; t += NT) {
      const int kk = t / BN, j = t % BN;
      const int k = k0 + kk, c = c0 + j;
      S v = Ar<S>::zero();
      if (k < nc && c < nrhs) {
        v = Q[(int64_t)(nd.col0 + k) * ld + c];
        const int s0 = gs[2 * k], s1 = gs[2 * k + 1];
        if (s0 >= 0) v = Ar<S>::add(v, U[(int64_t)s0 * ld + c]);
        if (s1 >= 0) v = Ar<S>::add(v, U[(int64_t)s1 * ld + c]);
      }
      Bs[kk][j] = P::from_s(v);
    }
    __syncthreads();
    const int klim = kmax - k0;   // the stage's last K column (block-uniform)
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      // FP64 tiles (BM == kSnBmFP64) skip the zero-padded K columns: the FP64 pipe bounds them
      if (BM == kSnBmFP64 && kk >= klim) break;
      A a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) P::mac(acc[i][j], a[i], b[j]);
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
      const S v0 = P::to_s(acc[i][j]);
      if (r < nc) {
        Z[(int64_t)(nd.col0 + r) * ld + c] = Ar<S>::mul(Dinv[nd.col0 + r], v0);
      } else {
        S v = v0;
        const int s0 = gs[2 * r], s1 = gs[2 * r + 1];
        if (s0 >= 0) v = Ar<S>::add(v, U[(int64_t)s0 * ld + c]);
        if (s1 >= 0) v = Ar<S>::add(v, U[(int64_t)s1 * ld + c]);
        U[(int64_t)(nd.u_off + r - nc) * ld + c] = v;
      }
    }
  }
}

template <typename P, int BN, int BM>
__global__ void __launch_bounds__(NT) k_sn_backward(const DevNode* __restrict__ nodes,
                                                    const typename P::WT* __restrict__ W,
                                                    const int32_t* __restrict__ rows,
                                                    const int2* __restrict__ tiles,
                                                    const typename P::S* __restrict__ Z,
                                                    typename P::S* __restrict__ X, int nrhs, int ld) {
  pdl_entry();
  using S = typename P::S;
  using A = typename P::A;
  constexpr int TN = BN / 16;
  constexpr int TM = BM / 16;
  __shared__ A As[BK][BM];
  __shared__ A Bs[BK][BN];
  const int2 tl = tiles[blockIdx.x];
  const DevNode nd = nodes[tl.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int row0 = tl.y * BM, c0 = blockIdx.y * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const typename P::WT* Ws = W + nd.w_off;
  const int32_t* rw = rows + nd.row_off;
  A acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = P::zero();
  // W[k][i] = 0 for k < i inside L11^{-1}: start at the tile's first row
  const int kmin = (row0 / BK) * BK;
  for (int k0 = kmin; k0 < m; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      const int i = t % BM, kk = t / BM;
      const int r = row0 + i, k = k0 + kk;
      As[kk][i] = (r < nc && k < m) ? P::from_w(Ws[(int64_t)k * nc + r]) : P::zero();
    }
    for (int t = threadIdx.x; t < BK * BN; t += NT) {
      const int kk = t / BN, j = t % BN;
      const int k = k0 + kk, c = c0 + j;
      S v = Ar<S>::zero();
      if (k < m && c < nrhs) {
        const int64_t src = (k < nc) ? (int64_t)(nd.col0 + k) : (int64_t)rw[k - nc];
        v = (k < nc) ? Z[src * ld + c] : X[src * ld + c];
      }
      Bs[kk][j] = P::from_s(v);
    }
    __syncthreads();
    const int klim = m - k0;      // the stage's last K column (block-uniform)
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      // FP64 tiles (BM == kSnBmFP64) skip the zero-padded K columns: the FP64 pipe bounds them
      if (BM == kSnBmFP64 && kk >= klim) break;
      A a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) P::mac(acc[i][j], a[i], b[j]);
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
      if (c < nrhs) X[(int64_t)(nd.col0 + r) * ld + c] = P::to_s(acc[i][j]);
    }
  }
}

// ---------------------------------------------------------------- split-K path
// With few right-hand sides (coarse time levels have 1..16 slabs), or at the few
// large supernodes near the root, the tiles of the tiled path leave most of the GPU
// idle and the top supernodes serialise on their long K loops.  Here every item is kSkRows rows
// x one K chunk of kSkK columns x one column block of NB right-hand sides (one row
// per thread, NB accumulators); a second kernel sums the chunks of each row in a
// fixed order (in the memory type S) and applies the epilogue.
constexpr int SK_THREADS = kSkRows;
constexpr int SK_KS = 16;   // K columns staged in shared memory at a time

// One item (kSkRows rows x one K chunk) x one column block of NB right-hand sides,
// computed by one warp (lane = row); As, Bs: the warp's shared-memory stage.  The
// kSkRows x NB partial product goes to out (row-major).
template <typename P, int NB, bool FWD, bool CG = false>
__device__ __forceinline__ void sk_item(const DevNode* __restrict__ nodes, const typename P::WT* __restrict__ W,
                                        const int32_t* __restrict__ gsrc, const int32_t* __restrict__ rows, int4 it,
                                        int cb, const typename P::S* __restrict__ Q,
                                        const typename P::S* __restrict__ Z, const typename P::S* __restrict__ U,
                                        const typename P::S* __restrict__ X, typename P::S* __restrict__ out,
                                        int nrhs, int ld, typename P::A (*As)[kSkRows + 1],
                                        typename P::A (*Bs)[NB], int lane, bool pdl_wait = false) {
  using S = typename P::S;
  using A = typename P::A;
  static_assert(SK_THREADS == 32, "one warp per item: warp-level synchronisation below");
  constexpr int NA = SK_KS * kSkRows / SK_THREADS;              // factor entries per thread per stage
  constexpr int NBL = (SK_KS * NB + SK_THREADS - 1) / SK_THREADS;   // right-hand-side entries per thread
  const DevNode nd = nodes[it.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int r0 = it.y, k0 = it.z, k1 = it.w;
  const int tid = lane;
  const typename P::WT* Ws = W + nd.w_off;
  const int32_t* gs = gsrc + nd.g_off * 2;
  const int32_t* rw = rows + nd.row_off;
  A acc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] = P::zero();
  // software pipeline: the next stage's global loads are in registers while the
  // current stage is multiplied out of shared memory
  typename P::WT ra[NA];   // raw factor entries (converted on the way into shared memory)
  S rb[NBL];
  auto load_w = [&](int ks) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int t = tid + u * SK_THREADS;
      int i, kk;
      if (FWD) { i = t / SK_KS; kk = t % SK_KS; }     // W row-major: k fastest
      else { i = t % kSkRows; kk = t / kSkRows; }     // W^T: row index fastest
      const int r = r0 + i, k = ks + kk;
      typename P::WT a{};
      if (FWD) { if (r < m && k < k1) a = Ws[(int64_t)r * nc + k]; }
      else { if (r < nc && k < k1) a = Ws[(int64_t)k * nc + r]; }
      ra[u] = a;
    }
  };
  auto load_b = [&](int ks) {
#pragma unroll
    for (int u = 0; u < NBL; ++u) {
      const int t = tid + u * SK_THREADS;
      S v = Ar<S>::zero();
      if (t < SK_KS * NB) {
        const int kk = t / NB, cl = t % NB, c = cb + cl;
        const int k = ks + kk;
        if (k < k1 && c < nrhs) {
          if (FWD) {
            v = Q[(int64_t)(nd.col0 + k) * ld + c];
            const int s0 = gs[2 * k], s1 = gs[2 * k + 1];
            if (s0 >= 0) v = Ar<S>::add(v, ldx<CG>(U + (int64_t)s0 * ld + c));
            if (s1 >= 0) v = Ar<S>::add(v, ldx<CG>(U + (int64_t)s1 * ld + c));
          } else {
            v = (k < nc) ? Z[(int64_t)(nd.col0 + k) * ld + c] : ldx<CG>(X + (int64_t)rw[k - nc] * ld + c);
          }
        }
      }
      rb[u] = v;
    }
  };
  // the factor is static: its first stage is requested before waiting for the kernel
  // that wrote the right-hand sides (pdl_wait: launched with programmatic serialisation)
  if (k0 < k1) load_w(k0);
  if (pdl_wait) pdl_entry();
  if (k0 < k1) load_b(k0);
  for (int ks = k0; ks < k1; ks += SK_KS) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int t = tid + u * SK_THREADS;
      if (FWD) As[t % SK_KS][t / SK_KS] = P::from_w(ra[u]);
      else As[t / kSkRows][t % kSkRows] = P::from_w(ra[u]);
    }
#pragma unroll
    for (int u = 0; u < NBL; ++u) {
      const int t = tid + u * SK_THREADS;
      if (t < SK_KS * NB) Bs[t / NB][t % NB] = P::from_s(rb[u]);
    }
    __syncwarp();
    if (ks + SK_KS < k1) {
      load_w(ks + SK_KS);
      load_b(ks + SK_KS);
    }
#pragma unroll
    for (int kk = 0; kk < SK_KS; ++kk) {
      const A a = As[kk][tid];
#pragma unroll
      for (int j = 0; j < NB; ++j) P::mac(acc[j], a, Bs[kk][j]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) out[tid * NB + j] = P::to_s(acc[j]);
}

// The kSkRows x NB outputs of one unit (node, kSkRows rows) and column block: the
// unit's K-chunk partials summed in item order, then the forward or backward
// epilogue.  One warp; lane t handles outputs t, t + 32, ... (row t / NB, column t % NB).
template <typename P, int NB, bool FWD, bool CG = false>
__device__ __forceinline__ void sk_unit(const DevNode* __restrict__ nodes, const typename P::S* __restrict__ Dinv,
                                        const int32_t* __restrict__ gsrc, int4 un, int64_t item_base,
                                        int64_t n_items, int by, const typename P::S* __restrict__ Pt,
                                        typename P::S* __restrict__ Z, typename P::S* __restrict__ U,
                                        typename P::S* __restrict__ X, int nrhs, int ld, int lane) {
  using S = typename P::S;
  const DevNode nd = nodes[un.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const S* Pc = Pt + (int64_t)by * n_items * kSkRows * NB;
  for (int t = lane; t < kSkRows * NB; t += 32) {
    const int i = t / NB, cl = t % NB, c = by * NB + cl;
    const int r = un.y + i;
    if (c >= nrhs) continue;
    S acc = Ar<S>::zero();
    for (int q = un.z; q < un.w; ++q)
      acc = Ar<S>::add(acc, ldx<CG>(Pc + (((int64_t)(q - item_base)) * kSkRows + i) * NB + cl));
    if (FWD) {
      if (r >= m) continue;
      if (r < nc) {
        Z[(int64_t)(nd.col0 + r) * ld + c] = Ar<S>::mul(Dinv[nd.col0 + r], acc);
      } else {
        const int32_t* gs = gsrc + nd.g_off * 2;
        const int s0 = gs[2 * r], s1 = gs[2 * r + 1];
        if (s0 >= 0) acc = Ar<S>::add(acc, ldx<CG>(U + (int64_t)s0 * ld + c));
        if (s1 >= 0) acc = Ar<S>::add(acc, ldx<CG>(U + (int64_t)s1 * ld + c));
        U[(int64_t)(nd.u_off + r - nc) * ld + c] = acc;
      }
    } else {
      if (r < nc) X[(int64_t)(nd.col0 + r) * ld + c] = acc;
    }
  }
}

template <typename P, int NB, bool FWD>
__global__ void __launch_bounds__(SK_THREADS) k_sn_skinny_partial(
    const DevNode* __restrict__ nodes, const typename P::WT* __restrict__ W, const int32_t* __restrict__ gsrc,
    const int32_t* __restrict__ rows, const int4* __restrict__ items, const typename P::S* __restrict__ Q,
    const typename P::S* __restrict__ Z, const typename P::S* __restrict__ U, const typename P::S* __restrict__ X,
    typename P::S* __restrict__ Pt, int nrhs, int ld) {
  // sk_item calls pdl_entry() after requesting the item's first factor stage (static
  // data), before it reads a right-hand side or writes its partial, so that under
  // programmatic serialisation the request overlaps the end of the previous kernel
  static_assert(SK_THREADS == 32, "one warp per item: warp-level synchronisation");
  __shared__ typename P::A As[SK_KS][kSkRows + 1];   // + 1: conflict-free stores of row-major factor rows
  __shared__ typename P::A Bs[SK_KS][NB];
  typename P::S* out = Pt + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kSkRows * NB;
  sk_item<P, NB, FWD>(nodes, W, gsrc, rows, items[blockIdx.x], blockIdx.y * NB, Q, Z, U, X, out, nrhs, ld, As, Bs,
                      threadIdx.x, true);
}

template <typename P, int NB, bool FWD>
__global__ void __launch_bounds__(kSkRows * NB) k_sn_skinny_reduce(
    const DevNode* __restrict__ nodes, const typename P::S* __restrict__ Dinv, const int32_t* __restrict__ gsrc,
    const int4* __restrict__ units, int64_t item_base, int64_t n_items, const typename P::S* __restrict__ Pt,
    typename P::S* __restrict__ Z, typename P::S* __restrict__ U, typename P::S* __restrict__ X, int nrhs, int ld) {
  // the unit's static description is read before waiting for the partials' kernel (an
  // overlap under programmatic serialisation)
  using S = typename P::S;
  const int4 un = units[blockIdx.x];
  const DevNode nd = nodes[un.x];
  pdl_entry();
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int i = threadIdx.x / NB, cl = threadIdx.x % NB, c = blockIdx.y * NB + cl;
  const int r = un.y + i;
  if (c >= nrhs) return;
  const S* Pc = Pt + (int64_t)blockIdx.y * n_items * kSkRows * NB;
  S acc = Ar<S>::zero();
  for (int q = un.z; q < un.w; ++q) acc = Ar<S>::add(acc, Pc[(((int64_t)(q - item_base)) * kSkRows + i) * NB + cl]);
  if (FWD) {
    if (r >= m) return;
    if (r < nc) {
      Z[(int64_t)(nd.col0 + r) * ld + c] = Ar<S>::mul(Dinv[nd.col0 + r], acc);
    } else {
      const int32_t* gs = gsrc + nd.g_off * 2;
      const int s0 = gs[2 * r], s1 = gs[2 * r + 1];
      if (s0 >= 0) acc = Ar<S>::add(acc, U[(int64_t)s0 * ld + c]);
      if (s1 >= 0) acc = Ar<S>::add(acc, U[(int64_t)s1 * ld + c]);
      U[(int64_t)(nd.u_off + r - nc) * ld + c] = acc;
    }
  } else {
    if (r < nc) X[(int64_t)(nd.col0 + r) * ld + c] = acc;
  }
}

template <typename P, int NB>
void skinny_depth(const DevFactor<typename P::S, typename P::WT>& F, int d, bool fwd, typename P::S* Q,
                  typename P::S* Z, typename P::S* U, typename P::S* Pt, int nrhs, int ld, const SkSync& sy,
                  cudaStream_t st) {
  const int64_t* io = fwd ? F.h_fs_item_off : F.h_bs_item_off;
  const int64_t* uo = fwd ? F.h_fs_unit_off : F.h_bs_unit_off;
  const int64_t ia = io[d], ib = io[d + 1], ua = uo[d], ub = uo[d + 1];
  if (ib <= ia) return;
  const unsigned gy = (unsigned)((nrhs + NB - 1) / NB);
  // FP32 right-hand sides (FP32 and 16-bit factors): each kernel's static prologue overlaps
  // the previous kernel's end.  The FP64 and double-float solves measured slower that way
  // (their kernels keep the FP64 or FP32 pipe busy to the end), so they queue plainly.
  constexpr bool fp32_rhs = std::is_same<typename P::S, float>::value || std::is_same<typename P::S, float2>::value;
  const bool ov = fp32_rhs || launch_overlap();
  if (fwd) {
    launch_cfg(ov, k_sn_skinny_partial<P, NB, true>, dim3((unsigned)(ib - ia), gy), SK_THREADS, 0, st,
        F.nodes, F.W, F.gsrc, F.rows, F.fs_items + ia, Q, Z, U, Q, Pt, nrhs, ld);
    launch_cfg(ov, k_sn_skinny_reduce<P, NB, true>, dim3((unsigned)(ub - ua), gy), kSkRows * NB, 0, st,
        F.nodes, F.Dinv, F.gsrc, F.fs_units + ua, ia, ib - ia, Pt, Z, U, Q, nrhs, ld);
  } else {
    launch_cfg(ov, k_sn_skinny_partial<P, NB, false>, dim3((unsigned)(ib - ia), gy), SK_THREADS, 0, st,
        F.nodes, F.W, F.gsrc, F.rows, F.bs_items + ia, Q, Z, U, Q, Pt, nrhs, ld);
    launch_cfg(ov, k_sn_skinny_reduce<P, NB, false>, dim3((unsigned)(ub - ua), gy), kSkRows * NB, 0, st,
        F.nodes, F.Dinv, F.gsrc, F.bs_units + ua, ia, ib - ia, Pt, Z, U, Q, nrhs, ld);
  }
  count_launches(2);
}

// ---------------------------------------------------------------- persistent split-K solve
// The whole solve (every tree depth, forward then backward) in one cooperative
// launch: PS_WARPS warps per block, each taking (item, column block) pairs and then
// (unit, column block) pairs grid-stride, with a grid barrier after every phase in
// place of a kernel boundary.  Same items, partial layout, summation order and
// epilogue as the per-depth kernels.
constexpr int PS_WARPS = 8;
constexpr int GRID_WAIT_LIMIT = 1 << 22;   // polls of one barrier (with a short sleep each)

// Grid barrier on bar[0] (arrivals) and bar[1] (generation).  Bounded: a block that
// gives up sets *err and returns false; the kernel then returns (its results are
// invalid and the host reports ST_MG_ERR_TIMEOUT).  Co-residency of all blocks is
// guaranteed by the cooperative launch.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      int it = 0;
      while (*vgen == g && it < GRID_WAIT_LIMIT) {
        __nanosleep(32);
        ++it;
      }
      if (*vgen == g) {
        atomicExch(err, 1);
        ok = 0;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename P, int NB, bool FWD>
__global__ void __launch_bounds__(PS_WARPS * 32) k_sn_skinny_solve(
    const DevNode* __restrict__ nodes, const typename P::WT* __restrict__ W, const typename P::S* __restrict__ Dinv,
    const int32_t* __restrict__ gsrc, const int32_t* __restrict__ rows, const int4* __restrict__ items,
    const int4* __restrict__ units, const int64_t* __restrict__ item_off, const int64_t* __restrict__ unit_off,
    int max_depth, typename P::S* __restrict__ Q, typename P::S* __restrict__ Z, typename P::S* __restrict__ U,
    typename P::S* __restrict__ Pt, int nrhs, int ld, unsigned* bar, int* err) {
  using A = typename P::A;
  extern __shared__ __align__(16) unsigned char ps_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  A (*As)[kSkRows + 1] = reinterpret_cast<A (*)[kSkRows + 1]>(ps_smem) + (int64_t)w * SK_KS;
  A (*Bs)[NB] = reinterpret_cast<A (*)[NB]>(ps_smem + (size_t)PS_WARPS * SK_KS * (kSkRows + 1) * sizeof(A)) +
                (int64_t)w * SK_KS;
  const int64_t gw = (int64_t)blockIdx.x * PS_WARPS + w, nw = (int64_t)gridDim.x * PS_WARPS;
  const int gy = (nrhs + NB - 1) / NB;
  for (int step = 0; step <= max_depth; ++step) {
    const int d = FWD ? max_depth - step : step;
    const int64_t ia = item_off[d], ni = item_off[d + 1] - ia;
    const int64_t ua = unit_off[d], nu = unit_off[d + 1] - ua;
    if (ni <= 0) continue;
    for (int64_t t = gw; t < ni * gy; t += nw) {
      const int64_t q = t % ni;
      const int by = (int)(t / ni);
      sk_item<P, NB, FWD>(nodes, W, gsrc, rows, items[ia + q], by * NB, Q, Z, U, Q,
                          Pt + ((int64_t)by * ni + q) * kSkRows * NB, nrhs, ld, As, Bs, lane);
    }
    if (!grid_barrier(bar, err)) return;
    for (int64_t t = gw; t < nu * gy; t += nw)
      sk_unit<P, NB, FWD>(nodes, Dinv, gsrc, units[ua + t % nu], ia, ni, (int)(t / nu), Pt, Z, U, Q, nrhs, ld, lane);
    if (!grid_barrier(bar, err)) return;
  }
}

// ---------------------------------------------------------------- dataflow split-K solve
// One sweep (forward or backward) of the split-K solve in one launch, ordered by data
// dependences instead of by tree depth.  Every warp claims tasks from a global counter
// in a fixed topological order (forward: depth max .. 0, backward: 0 .. max; in each
// depth its items, then its units).  An item of node s first waits until the nodes it
// reads from are complete (forward: the children, whose update rows it gathers;
// backward: the parent, whose completion implies every ancestor's, whose solution rows
// it gathers), a unit until all of its items are; a finished item counts towards its
// unit, a finished unit towards its node.  A task only waits on tasks claimed before it,
// and those are held by running warps that wait only on tasks claimed before theirs, so
// the sweep always progresses.  Items, partial layout (one partial block per item),
// summation order and epilogue are those of the per-depth kernels: results agree bit for
// bit.  Values written in this launch are read through L2 (ldx<true>).  Waits are
// bounded: a wait that gives up sets *err and the task runs anyway (its result is then
// invalid and reported), so no other wait hangs behind it.
// ctr: [0] task counter, [1, 1 + n_units) items finished per unit, then units finished
// per node; zero before the launch.
constexpr int DF_WARPS = 8;
constexpr int DF_WAIT_LIMIT = 1 << 22;   // polls (each after a short sleep) before a wait gives up

// Lane 0 of a warp: wait until *p >= target.  Gives up at once once *err is set (an
// earlier wait gave up: the sweep's result is already invalid), else after the limit.
__device__ __forceinline__ bool df_wait(const unsigned* p, unsigned target, const int* err) {
  for (int it = 0; it < DF_WAIT_LIMIT; ++it) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    if (*reinterpret_cast<const volatile int*>(err)) return false;
    __nanosleep(64);
  }
  return false;
}

template <typename P, int NB, bool FWD>
__global__ void __launch_bounds__(DF_WARPS * 32) k_sn_skinny_df(
    const DevNode* __restrict__ nodes, const typename P::WT* __restrict__ W, const typename P::S* __restrict__ Dinv,
    const int32_t* __restrict__ gsrc, const int32_t* __restrict__ rows, const int4* __restrict__ items,
    const int4* __restrict__ units, const int2* __restrict__ tasks, int ntasks,
    const int32_t* __restrict__ item_unit, const int32_t* __restrict__ node_units, const int2* __restrict__ node_dep,
    int n_units, typename P::S* Q, typename P::S* Z, typename P::S* U, typename P::S* Pt, int nrhs, int ld,
    unsigned* ctr, int* err) {
  pdl_entry();
  using A = typename P::A;
  extern __shared__ __align__(16) unsigned char df_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  A (*As)[kSkRows + 1] = reinterpret_cast<A (*)[kSkRows + 1]>(df_smem) + (int64_t)w * SK_KS;
  A (*Bs)[NB] = reinterpret_cast<A (*)[NB]>(df_smem + (size_t)DF_WARPS * SK_KS * (kSkRows + 1) * sizeof(A)) +
                (int64_t)w * SK_KS;
  unsigned* unit_done = ctr + 1;
  unsigned* node_done = ctr + 1 + n_units;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(ctr, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntasks) break;
    const int2 tk = tasks[t];
    if (tk.x == 0) {
      const int4 it = items[tk.y];
      if (lane == 0) {
        const int2 dp = node_dep[it.x];
        bool ok = true;
        if (dp.x >= 0) ok = df_wait(node_done + dp.x, (unsigned)node_units[dp.x], err);
        if (ok && dp.y >= 0) ok = df_wait(node_done + dp.y, (unsigned)node_units[dp.y], err);
        if (!ok) atomicExch(err, 1);
      }
      __syncwarp();
      __threadfence();
      sk_item<P, NB, FWD, true>(nodes, W, gsrc, rows, it, 0, Q, Z, U, Q, Pt + (int64_t)tk.y * kSkRows * NB, nrhs,
                                ld, As, Bs, lane);
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(unit_done + item_unit[tk.y], 1u);
    } else {
      const int4 un = units[tk.y];
      if (lane == 0 && !df_wait(unit_done + tk.y, (unsigned)(un.w - un.z), err)) atomicExch(err, 1);
      __syncwarp();
      __threadfence();
      sk_unit<P, NB, FWD, true>(nodes, Dinv, gsrc, un, 0, 0, 0, Pt, Z, U, Q, nrhs, ld, lane);
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(node_done + un.x, 1u);
    }
  }
}

template <typename P, int NB>
cudaError_t sn_solve_skinny(const DevFactor<typename P::S, typename P::WT>& F, typename P::S* Q, typename P::S* Z,
                            typename P::S* U, typename P::S* Pt, int nrhs, int ld, const SkSync& sy,
                            cudaStream_t st) {
  if (sy.df && sy.err && F.df_tasks_f && nrhs <= NB) {
    // two dataflow launches (forward, backward), each after zeroing its counters
    static int grid[2] = {-1, -1};   // per instantiation: depends only on the kernel and the device
    const size_t smem = (size_t)DF_WARPS * SK_KS * ((kSkRows + 1) + NB) * sizeof(typename P::A);
    for (int dir = 0; dir < 2; ++dir) {
      auto kern = dir == 0 ? k_sn_skinny_df<P, NB, true> : k_sn_skinny_df<P, NB, false>;
      if (grid[dir] < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DF_WARPS * 32, smem);
        if (e != cudaSuccess) return e;
        grid[dir] = std::max(per_sm, 1) * F.n_sm;
      }
    }
    for (int dir = 0; dir < 2; ++dir) {
      const bool fwd = dir == 0;
      const int nunits = (int)(fwd ? F.n_fs_units : F.n_bs_units);
      const int ntasks = (int)(fwd ? F.n_df_tasks_f : F.n_df_tasks_b);
      cudaError_t e = cudaMemsetAsync(sy.df, 0, sizeof(unsigned) * (size_t)(1 + nunits + F.nnodes), st);
      if (e != cudaSuccess) return e;
      if (fwd)
        launch_k(k_sn_skinny_df<P, NB, true>, dim3((unsigned)grid[0]), DF_WARPS * 32, smem, st, F.nodes, F.W, F.Dinv,
                 F.gsrc, F.rows, F.fs_items, F.fs_units, F.df_tasks_f, ntasks, F.df_item_unit_f, F.df_node_units_f,
                 F.df_children, nunits, Q, Z, U, Pt, nrhs, ld, sy.df, sy.err);
      else
        launch_k(k_sn_skinny_df<P, NB, false>, dim3((unsigned)grid[1]), DF_WARPS * 32, smem, st, F.nodes, F.W, F.Dinv,
                 F.gsrc, F.rows, F.bs_items, F.bs_units, F.df_tasks_b, ntasks, F.df_item_unit_b, F.df_node_units_b,
                 F.df_parent, nunits, Q, Z, U, Pt, nrhs, ld, sy.df, sy.err);
      count_launches(1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (sy.bar && sy.err && F.d_fs_item_off) {
    // two cooperative launches (forward, backward), as many blocks as can be resident
    static int grid[2] = {-1, -1};   // per instantiation: depends only on the kernel and the device
    const size_t smem = (size_t)PS_WARPS * SK_KS * ((kSkRows + 1) + NB) * sizeof(typename P::A);
    for (int dir = 0; dir < 2; ++dir) {
      auto kern = dir == 0 ? k_sn_skinny_solve<P, NB, true> : k_sn_skinny_solve<P, NB, false>;
      if (grid[dir] < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PS_WARPS * 32, smem);
        if (e != cudaSuccess) return e;
        grid[dir] = per_sm * F.n_sm;
      }
    }
    if (grid[0] > 0 && grid[1] > 0) {
      for (int dir = 0; dir < 2; ++dir) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid[dir]);
        cfg.blockDim = dim3(PS_WARPS * 32);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const bool fwd = dir == 0;
        cudaError_t e = cudaLaunchKernelEx(
            &cfg, fwd ? k_sn_skinny_solve<P, NB, true> : k_sn_skinny_solve<P, NB, false>, F.nodes, F.W, F.Dinv,
            F.gsrc, F.rows, fwd ? F.fs_items : F.bs_items, fwd ? F.fs_units : F.bs_units,
            fwd ? F.d_fs_item_off : F.d_bs_item_off, fwd ? F.d_fs_unit_off : F.d_bs_unit_off, F.max_depth, Q, Z, U, Pt,
            nrhs, ld, sy.bar, sy.err);
        count_launches(1);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  for (int d = F.max_depth; d >= 0; --d) skinny_depth<P, NB>(F, d, true, Q, Z, U, Pt, nrhs, ld, sy, st);
  for (int d = 0; d <= F.max_depth; ++d) skinny_depth<P, NB>(F, d, false, Q, Z, U, Pt, nrhs, ld, sy, st);
  return cudaGetLastError();
}

// Tiled products for many right-hand sides; a depth whose tile grid would not
// fill two waves of the GPU (the few large supernodes near the root) goes through
// the split-K kernels instead, with NBK right-hand sides per column block.
template <typename P, int BN, int NBK, int BM>
cudaError_t sn_solve_tiled(const DevFactor<typename P::S, typename P::WT>& F, typename P::S* Q, typename P::S* Z,
                           typename P::S* U, typename P::S* Pt, int nrhs, int ld, const SkSync& sy,
                           cudaStream_t st) {
  const unsigned gy = (unsigned)((nrhs + BN - 1) / BN);
  const int64_t two_waves = (int64_t)sy.split_waves * F.n_sm;
  for (int d = F.max_depth; d >= 0; --d) {
    const int64_t a = F.h_fwd_off[d], b = F.h_fwd_off[d + 1];
    if (b <= a) continue;
    if (Pt && (b - a) * gy < two_waves) {
      skinny_depth<P, NBK>(F, d, true, Q, Z, U, Pt, nrhs, ld, sy, st);
      continue;
    }
    launch_k(k_sn_forward<P, BN, BM>, dim3((unsigned)(b - a), gy), NT, 0, st, F.nodes, F.W, F.Dinv, F.gsrc, F.fwd_tiles + a,
                                                                     Q, Z, U, nrhs, ld);
    count_launches(1);
  }
  for (int d = 0; d <= F.max_depth; ++d) {
    const int64_t a = F.h_bwd_off[d], b = F.h_bwd_off[d + 1];
    if (b <= a) continue;
    if (Pt && (b - a) * gy < two_waves) {
      skinny_depth<P, NBK>(F, d, false, Q, Z, U, Pt, nrhs, ld, sy, st);
      continue;
    }
    launch_k(k_sn_backward<P, BN, BM>, dim3((unsigned)(b - a), gy), NT, 0, st, F.nodes, F.W, F.rows, F.bwd_tiles + a, Z, Q,
                                                                      nrhs, ld);
    count_launches(1);
  }
  return cudaGetLastError();
}

// Real matrices: column blocks of 4 / 16 / 32 on the split-K path, 64-wide tiles.
template <typename P, int BM = kSnBM>
cudaError_t solve_real(const DevFactor<typename P::S, typename P::WT>& F, typename P::S* Q, typename P::S* Z,
                       typename P::S* U, typename P::S* Pt, int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (Pt && nrhs <= 4) return sn_solve_skinny<P, 4>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  if (Pt && nrhs <= 16) return sn_solve_skinny<P, 16>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  if (Pt && nrhs <= kSkMaxRhsR) return sn_solve_skinny<P, kSkMaxRhsR>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  return sn_solve_tiled<P, 64, kSkMaxRhsR, BM>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
}
// Complex matrices: column blocks of 2 / 8 / 16, 32-wide tiles.
template <typename P, int BM = kSnBM>
cudaError_t solve_cplx(const DevFactor<typename P::S, typename P::WT>& F, typename P::S* Q, typename P::S* Z,
                       typename P::S* U, typename P::S* Pt, int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (Pt && nrhs <= 2) return sn_solve_skinny<P, 2>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  if (Pt && nrhs <= 8) return sn_solve_skinny<P, 8>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  if (Pt && nrhs <= kSkMaxRhsC) return sn_solve_skinny<P, kSkMaxRhsC>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
  return sn_solve_tiled<P, 32, kSkMaxRhsC, BM>(F, Q, Z, U, Pt, nrhs, ld, sy, st);
}

}  // namespace

}  // namespace stmg
