// Space-time kernels of the V-cycle (Sections 2.1, 2.2, 3.3 of the paper), all on
// the edge-major layout v[e * ncols + n*q + i] (q = DG degree + 1): the row of one
// spatial unknown holds all slabs, so a CSR gather of a neighbour reads one
// contiguous vector and a warp's loads coalesce.
#include <atomic>

#include <type_traits>

#include "device.h"
#include "launch.cuh"

namespace stmg {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RES_WARPS = 8;   // rows (warps) per block of the residual kernels
constexpr int SPL = 8;         // slabs per lane per pass (32 * SPL slabs per pass), FP64 kernels
constexpr int SPL_DF = 2;      // the same for the double-float kernels (4 pairs of accumulators per
                               // slab: fewer slabs per pass keep enough warps resident)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block sum of per-thread values in a fixed order -> out (thread 0 writes).
template <int NTH>
__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double red[NTH / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NTH / 32; ++w) s += red[w];
    *out = s;
  }
}

// T = double: the FP64 residual.  T = float: the same operations in FP32 on an FP32 copy
// of x and FP32 coefficients, f and r in FP64 (the residual of a correction equation,
// whose right-hand side is itself a residual: the rounding error is relative to it).
// r_n = f_n - (K_t (x) M + M_t (x) K) x_n - (N_t (x) M) x_{n-1} for DG(1), with
// K_t = [[1,1],[-1,1]], M_t = tau diag(1, 1/3), N_t = [[-1,-1],[1,1]]:
//   r0 = f0 - (A0 + A1 + B0) + c,  r1 = f1 - (A1 - A0 + B1) - c
// where A_i = M x_i, B0 = tau K x0, B1 = (tau/3) K x1 on slab n and
// c = (M (x0 + x1)) of slab n-1 = A0 + A1 of the previous slab.
template <int LPR, typename T>
__global__ void __launch_bounds__(RES_WARPS * 32) k_residual_dg1(int nrows, const int64_t* __restrict__ rowptr,
                                                                 const int32_t* __restrict__ col,
                                                                 const T* __restrict__ m,
                                                                 const T* __restrict__ k0,
                                                                 const T* __restrict__ k1,
                                                                 const double* __restrict__ f,
                                                                 const T* __restrict__ x,
                                                                 double* __restrict__ r, int N_t,
                                                                 double* __restrict__ partial, int seg) {
  pdl_entry();
  using V2 = typename std::conditional<std::is_same<T, double>::value, double2, float2>::type;
  // LPR lanes per row, 32 / LPR rows per warp (few slabs on coarse time levels)
  const int lane = threadIdx.x & (LPR - 1);
  const int row = (blockIdx.x * RES_WARPS + (threadIdx.x >> 5)) * (32 / LPR) + ((threadIdx.x & 31) / LPR);
  double sq = 0.0;
  {
    // rows past the end keep the warp's shuffles uniform: empty, no loads or stores
    const bool valid = row < nrows;
    const int64_t beg = valid ? rowptr[row] : 0, end = valid ? rowptr[row + 1] : 0;
    const int64_t ld = 2 * (int64_t)N_t;
    const double2* f2 = reinterpret_cast<const double2*>(f + row * ld);
    double2* r2 = reinterpret_cast<double2*>(r + row * ld);
    T carry = T(0);   // A0 + A1 of the slab before this pass
    for (int n0 = 0; n0 < N_t; n0 += LPR * SPL) {
      T A0[SPL], A1[SPL], B0[SPL], B1[SPL];
#pragma unroll
      for (int j = 0; j < SPL; ++j) A0[j] = A1[j] = B0[j] = B1[j] = T(0);
      for (int64_t q = beg; q < end; ++q) {
        const int64_t c = col[q];
        const T mv = m[q], kv0 = k0[q], kv1 = k1[q];
        const V2* xr = reinterpret_cast<const V2*>(x + c * ld);
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
          const int n = n0 + LPR * j + lane;
          if (n < N_t) {
            const V2 v = xr[n];
            A0[j] = fma(mv, v.x, A0[j]);
            A1[j] = fma(mv, v.y, A1[j]);
            B0[j] = fma(kv0, v.x, B0[j]);
            B1[j] = fma(kv1, v.y, B1[j]);
          }
        }
      }
      T prevA = carry;
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        const T As = A0[j] + A1[j];
        const T up = __shfl_up_sync(FULL, As, 1, LPR);
        const T from31 = __shfl_sync(FULL, prevA, LPR - 1, LPR);
        T c = (lane > 0) ? up : (j == 0 ? carry : from31);
        prevA = As;
        const int n = n0 + LPR * j + lane;
        if (n % seg == 0) c = T(0);   // first slab of a problem: no history
        if (valid && n < N_t) {
          const double2 fv = f2[n];
          double2 rv;
          if (std::is_same<T, double>::value) {
            rv.x = fv.x - (double)(As + B0[j]) + (double)c;
            rv.y = fv.y - (double)((A1[j] - A0[j]) + B1[j]) - (double)c;
          } else {
            // FP32: the operator applied in FP32 and one FP64 subtraction from f per value
            // (the FP64 pipe is the scarce one)
            rv.x = fv.x - (double)((As + B0[j]) - c);
            rv.y = fv.y - (double)(((A1[j] - A0[j]) + B1[j]) + c);
          }
          r2[n] = rv;
          if (partial) {
            sq = fma(rv.x, rv.x, sq);
            sq = fma(rv.y, rv.y, sq);
          }
        }
      }
      carry = __shfl_sync(FULL, prevA, LPR - 1, LPR);
    }
  }
  if (partial) block_sum_store<RES_WARPS * 32>(sq, partial + blockIdx.x);
}

// DG(0) (implicit Euler, eq. timeStepping): r_n = f_n - (M + tau K) x_n + M x_{n-1}.
template <int LPR, typename T>
__global__ void __launch_bounds__(RES_WARPS * 32) k_residual_dg0(int nrows, const int64_t* __restrict__ rowptr,
                                                                 const int32_t* __restrict__ col,
                                                                 const T* __restrict__ a,
                                                                 const T* __restrict__ m,
                                                                 const double* __restrict__ f,
                                                                 const T* __restrict__ x,
                                                                 double* __restrict__ r, int N_t,
                                                                 double* __restrict__ partial, int seg) {
  pdl_entry();
  // LPR lanes per row, 32 / LPR rows per warp (few slabs on coarse time levels)
  const int lane = threadIdx.x & (LPR - 1);
  const int row = (blockIdx.x * RES_WARPS + (threadIdx.x >> 5)) * (32 / LPR) + ((threadIdx.x & 31) / LPR);
  double sq = 0.0;
  {
    // rows past the end keep the warp's shuffles uniform: empty, no loads or stores
    const bool valid = row < nrows;
    const int64_t beg = valid ? rowptr[row] : 0, end = valid ? rowptr[row + 1] : 0;
    const int64_t ld = N_t;
    T carry = T(0);
    for (int n0 = 0; n0 < N_t; n0 += LPR * SPL) {
      T Ax[SPL], Mx[SPL];
#pragma unroll
      for (int j = 0; j < SPL; ++j) Ax[j] = Mx[j] = T(0);
      for (int64_t q = beg; q < end; ++q) {
        const int64_t c = col[q];
        const T av = a[q], mv = m[q];
        const T* xr = x + c * ld;
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
          const int n = n0 + LPR * j + lane;
          if (n < N_t) {
            const T v = xr[n];
            Ax[j] = fma(av, v, Ax[j]);
            Mx[j] = fma(mv, v, Mx[j]);
          }
        }
      }
      T prev = carry;
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        const T up = __shfl_up_sync(FULL, Mx[j], 1, LPR);
        const T from31 = __shfl_sync(FULL, prev, LPR - 1, LPR);
        T c = (lane > 0) ? up : (j == 0 ? carry : from31);
        prev = Mx[j];
        const int n = n0 + LPR * j + lane;
        if (n % seg == 0) c = T(0);   // first slab of a problem: no history
        if (valid && n < N_t) {
          const double rv = f[row * ld + n] - (double)Ax[j] + (double)c;
          r[row * ld + n] = rv;
          sq = fma(rv, rv, sq);
        }
      }
      carry = __shfl_sync(FULL, prev, LPR - 1, LPR);
    }
  }
  if (partial) block_sum_store<RES_WARPS * 32>(sq, partial + blockIdx.x);
}

// ---------------------------------------------------------------- double-float residual
// FP64-accurate residual on the FP32 pipes: x is split once per call into (hi, lo)
// FP32 pairs, matrix coefficients are stored as pairs, every product is exact
// (fma error term) plus cross terms and every sum an error-free two-sum; the
// accumulated pairs are joined in FP64 for the time-block combination with f.
struct dpair {
  float h, l;
};

__device__ __forceinline__ void dp_mac(dpair& acc, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float t = (acc.h - (s - bb)) + (p - bb);
  acc.l = acc.l + (t + e);
  acc.h = s;
}
__device__ __forceinline__ double dp_join(dpair a) { return (double)a.h + (double)a.l; }

__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ xf, int64_t n) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xf[i] = (float)x[i];
}

// b += a
__global__ void k_vec_add(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] += a[i];
}

__global__ void k_split_pairs(const double* __restrict__ x, float2* __restrict__ xs, int64_t n) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = __double2float_rn(v);
    xs[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

template <int LPR>
__global__ void __launch_bounds__(RES_WARPS * 32) k_residual_dg1_df(int nrows, const int64_t* __restrict__ rowptr,
                                                                    const int32_t* __restrict__ col,
                                                                    const float2* __restrict__ m,
                                                                    const float2* __restrict__ k0,
                                                                    const float2* __restrict__ k1,
                                                                    const double* __restrict__ f,
                                                                    const float2* __restrict__ xs,
                                                                    double* __restrict__ r, int N_t,
                                                                    double* __restrict__ partial, int seg) {
  pdl_entry();
  // LPR lanes per row, 32 / LPR rows per warp (few slabs on coarse time levels)
  const int lane = threadIdx.x & (LPR - 1);
  const int row = (blockIdx.x * RES_WARPS + (threadIdx.x >> 5)) * (32 / LPR) + ((threadIdx.x & 31) / LPR);
  double sq = 0.0;
  {
    // rows past the end keep the warp's shuffles uniform: empty, no loads or stores
    const bool valid = row < nrows;
    const int64_t beg = valid ? rowptr[row] : 0, end = valid ? rowptr[row + 1] : 0;
    const int64_t ld = 2 * (int64_t)N_t;
    const double2* f2 = reinterpret_cast<const double2*>(f + row * ld);
    double2* r2 = reinterpret_cast<double2*>(r + row * ld);
    double carry = 0.0;
    for (int n0 = 0; n0 < N_t; n0 += LPR * SPL_DF) {
      dpair A0[SPL_DF], A1[SPL_DF], B0[SPL_DF], B1[SPL_DF];
#pragma unroll
      for (int j = 0; j < SPL_DF; ++j) A0[j] = A1[j] = B0[j] = B1[j] = dpair{0.f, 0.f};
      for (int64_t q = beg; q < end; ++q) {
        const int64_t c = col[q];
        const float2 mv = m[q], kv0 = k0[q], kv1 = k1[q];
        const float4* xr = reinterpret_cast<const float4*>(xs + c * ld);
#pragma unroll
        for (int j = 0; j < SPL_DF; ++j) {
          const int n = n0 + LPR * j + lane;
          if (n < N_t) {
            const float4 v = xr[n];   // (x0 hi, x0 lo, x1 hi, x1 lo)
            const float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
            dp_mac(A0[j], mv, x0);
            dp_mac(A1[j], mv, x1);
            dp_mac(B0[j], kv0, x0);
            dp_mac(B1[j], kv1, x1);
          }
        }
      }
      double prevA = carry;
#pragma unroll
      for (int j = 0; j < SPL_DF; ++j) {
        const double a0 = dp_join(A0[j]), a1 = dp_join(A1[j]);
        const double As = a0 + a1;
        const double up = __shfl_up_sync(FULL, As, 1, LPR);
        const double from31 = __shfl_sync(FULL, prevA, LPR - 1, LPR);
        double c = (lane > 0) ? up : (j == 0 ? carry : from31);
        prevA = As;
        const int n = n0 + LPR * j + lane;
        if (n % seg == 0) c = 0.0;   // first slab of a problem: no history
        if (valid && n < N_t) {
          const double2 fv = f2[n];
          double2 rv;
          rv.x = fv.x - (As + dp_join(B0[j])) + c;
          rv.y = fv.y - ((a1 - a0) + dp_join(B1[j])) - c;
          r2[n] = rv;
          sq = fma(rv.x, rv.x, sq);
          sq = fma(rv.y, rv.y, sq);
        }
      }
      carry = __shfl_sync(FULL, prevA, LPR - 1, LPR);
    }
  }
  if (partial) block_sum_store<RES_WARPS * 32>(sq, partial + blockIdx.x);
}

template <int LPR>
__global__ void __launch_bounds__(RES_WARPS * 32) k_residual_dg0_df(int nrows, const int64_t* __restrict__ rowptr,
                                                                    const int32_t* __restrict__ col,
                                                                    const float2* __restrict__ a,
                                                                    const float2* __restrict__ m,
                                                                    const double* __restrict__ f,
                                                                    const float2* __restrict__ xs,
                                                                    double* __restrict__ r, int N_t,
                                                                    double* __restrict__ partial, int seg) {
  pdl_entry();
  // LPR lanes per row, 32 / LPR rows per warp (few slabs on coarse time levels)
  const int lane = threadIdx.x & (LPR - 1);
  const int row = (blockIdx.x * RES_WARPS + (threadIdx.x >> 5)) * (32 / LPR) + ((threadIdx.x & 31) / LPR);
  double sq = 0.0;
  {
    // rows past the end keep the warp's shuffles uniform: empty, no loads or stores
    const bool valid = row < nrows;
    const int64_t beg = valid ? rowptr[row] : 0, end = valid ? rowptr[row + 1] : 0;
    const int64_t ld = N_t;
    double carry = 0.0;
    for (int n0 = 0; n0 < N_t; n0 += LPR * SPL_DF) {
      dpair Ax[SPL_DF], Mx[SPL_DF];
#pragma unroll
      for (int j = 0; j < SPL_DF; ++j) Ax[j] = Mx[j] = dpair{0.f, 0.f};
      for (int64_t q = beg; q < end; ++q) {
        const int64_t c = col[q];
        const float2 av = a[q], mv = m[q];
        const float2* xr = xs + c * ld;
#pragma unroll
        for (int j = 0; j < SPL_DF; ++j) {
          const int n = n0 + LPR * j + lane;
          if (n < N_t) {
            const float2 v = xr[n];
            dp_mac(Ax[j], av, v);
            dp_mac(Mx[j], mv, v);
          }
        }
      }
      double prev = carry;
#pragma unroll
      for (int j = 0; j < SPL_DF; ++j) {
        const double mx = dp_join(Mx[j]);
        const double up = __shfl_up_sync(FULL, mx, 1, LPR);
        const double from31 = __shfl_sync(FULL, prev, LPR - 1, LPR);
        double c = (lane > 0) ? up : (j == 0 ? carry : from31);
        prev = mx;
        const int n = n0 + LPR * j + lane;
        if (n % seg == 0) c = 0.0;   // first slab of a problem: no history
        if (valid && n < N_t) {
          const double rv = f[row * ld + n] - dp_join(Ax[j]) + c;
          r[row * ld + n] = rv;
          sq = fma(rv, rv, sq);
        }
      }
      carry = __shfl_sync(FULL, prev, LPR - 1, LPR);
    }
  }
  if (partial) block_sum_store<RES_WARPS * 32>(sq, partial + blockIdx.x);
}

__global__ void k_reduce_partials(const double* __restrict__ p, int n, double* __restrict__ out) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  block_sum_store<256>(s, out);
}

constexpr int NORM_BLOCKS = 1024;
__global__ void k_norm_partial(const double* __restrict__ v, int64_t n, double* __restrict__ partial) {
  pdl_entry();
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(v[i], v[i], s);
  block_sum_store<256>(s, partial + blockIdx.x);
}

constexpr int SLAB_ROWS = 4;   // rows (one per warp) per block of the permutation / transform kernels

__global__ void k_slab_pre_dg0(int nrows, const double* __restrict__ r, int src_ld, int slab0, int cnt,
                               const int32_t* __restrict__ iperm, double* __restrict__ Q, int ld) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double* src = r + (int64_t)e * src_ld;
  double* dst = Q + (int64_t)iperm[e] * ld;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) dst[k] = src[slab0 + k];
}

__global__ void k_slab_pre_dg1(int nrows, const double* __restrict__ r, int src_ld, int slab0, int cnt,
                               const int32_t* __restrict__ iperm, double2 c0, double2 c1,
                               double2* __restrict__ Q, int ld) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double2* src = reinterpret_cast<const double2*>(r + (int64_t)e * src_ld);
  double2* dst = Q + (int64_t)iperm[e] * ld;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const double2 v = src[slab0 + k];
    dst[k] = make_double2(c0.x * v.x + c1.x * v.y, c0.y * v.x + c1.y * v.y);
  }
}

__global__ void k_slab_post_dg0(int nrows, const double* __restrict__ X, int ld, const int32_t* __restrict__ iperm,
                                double* __restrict__ x, int dst_ld, int slab0, int cnt, double omega, int mode) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double* src = X + (int64_t)iperm[e] * ld;
  double* dst = x + (int64_t)e * dst_ld + slab0;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const double v = src[k];
    if (mode == 0) dst[k] = v;
    else dst[k] = fma(omega, v, dst[k]);
  }
}

__global__ void k_slab_post_dg1(int nrows, const double2* __restrict__ X, int ld, const int32_t* __restrict__ iperm,
                                double2 s1, double* __restrict__ x, int dst_ld, int slab0, int cnt,
                                double omega, int mode) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double2* src = X + (int64_t)iperm[e] * ld;
  double2* dst = reinterpret_cast<double2*>(x + (int64_t)e * dst_ld) + slab0;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const double2 v = src[k];
    const double u0 = 2.0 * v.x;
    const double u1 = 2.0 * (s1.x * v.x - s1.y * v.y);
    if (mode == 0) {
      dst[k] = make_double2(u0, u1);
    } else {
      double2 o = dst[k];
      o.x = fma(omega, u0, o.x);
      o.y = fma(omega, u1, o.y);
      dst[k] = o;
    }
  }
}

__global__ void k_slab_pre_dg0f(int nrows, const double* __restrict__ r, int src_ld, int slab0, int cnt,
                                const int32_t* __restrict__ iperm, float* __restrict__ Q, int ld) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double* src = r + (int64_t)e * src_ld;
  float* dst = Q + (int64_t)iperm[e] * ld;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) dst[k] = (float)src[slab0 + k];
}

__global__ void k_slab_pre_dg1f(int nrows, const double* __restrict__ r, int src_ld, int slab0, int cnt,
                                const int32_t* __restrict__ iperm, double2 c0, double2 c1,
                                float2* __restrict__ Q, int ld) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const double2* src = reinterpret_cast<const double2*>(r + (int64_t)e * src_ld);
  float2* dst = Q + (int64_t)iperm[e] * ld;
  // the transform in FP32 (its result is rounded to FP32 anyway): two conversions per
  // value on the FP64 pipe instead of four FP64 multiply-adds and two conversions
  const float a0 = (float)c0.x, a1 = (float)c1.x, b0 = (float)c0.y, b1 = (float)c1.y;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const double2 v = src[slab0 + k];
    const float vx = (float)v.x, vy = (float)v.y;
    dst[k] = make_float2(fmaf(a0, vx, a1 * vy), fmaf(b0, vx, b1 * vy));
  }
}

__global__ void k_slab_post_dg0f(int nrows, const float* __restrict__ X, int ld, const int32_t* __restrict__ iperm,
                                 double* __restrict__ x, int dst_ld, int slab0, int cnt, double omega, int mode) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const float* src = X + (int64_t)iperm[e] * ld;
  double* dst = x + (int64_t)e * dst_ld + slab0;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const double v = (double)src[k];
    if (mode == 0) dst[k] = v;
    else dst[k] = fma(omega, v, dst[k]);
  }
}

__global__ void k_slab_post_dg1f(int nrows, const float2* __restrict__ X, int ld, const int32_t* __restrict__ iperm,
                                 double2 s1, double* __restrict__ x, int dst_ld, int slab0, int cnt,
                                 double omega, int mode) {
  pdl_entry();
  const int e = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (e >= nrows) return;
  const float2* src = X + (int64_t)iperm[e] * ld;
  double2* dst = reinterpret_cast<double2*>(x + (int64_t)e * dst_ld) + slab0;
  // the back transform and the damping in FP32 (the solution is an FP32 value), then one
  // FP64 addition per value
  const float w = (float)(mode == 0 ? 1.0 : omega);
  const float t0 = 2.0f * w, t1 = (float)(2.0 * s1.x) * w, t2 = (float)(2.0 * s1.y) * w;
#pragma unroll 4
  for (int k = threadIdx.x & 31; k < cnt; k += 32) {
    const float2 vf = src[k];
    const float u0 = t0 * vf.x;
    const float u1 = fmaf(t1, vf.x, -(t2 * vf.y));
    if (mode == 0) {
      dst[k] = make_double2((double)u0, (double)u1);
    } else {
      double2 o = dst[k];
      o.x += (double)u0;
      o.y += (double)u1;
      dst[k] = o;
    }
  }
}

template <typename TQ>
__global__ void k_gather_perm(int nrows, const double* __restrict__ y, int ncols, const int32_t* __restrict__ iperm,
                              TQ* __restrict__ Q, int ld) {
  pdl_entry();
  const int v = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (v >= nrows) return;
  const double* src = y + (int64_t)v * ncols;
  TQ* dst = Q + (int64_t)iperm[v] * ld;
#pragma unroll 4
  for (int j = threadIdx.x & 31; j < ncols; j += 32) dst[j] = (TQ)src[j];
}

template <typename TQ>
__global__ void k_scatter_perm(int nrows, const TQ* __restrict__ X, int ld, const int32_t* __restrict__ iperm,
                               double* __restrict__ z, int ncols) {
  pdl_entry();
  const int v = blockIdx.x * SLAB_ROWS + (threadIdx.x >> 5);   // one warp per row
  if (v >= nrows) return;
  const TQ* src = X + (int64_t)iperm[v] * ld;
  double* dst = z + (int64_t)v * ncols;
#pragma unroll 4
  for (int j = threadIdx.x & 31; j < ncols; j += 32) dst[j] = (double)src[j];
}

// y = G^T r: warp per node, lanes over the time columns.
// y = G^T r: one warp per interior vertex.  The vertex's (at most 32) edges and signs
// are staged in shared memory; each lane sums double2 column pairs over them, four
// loads issued before their sums (the edge order of the sum is fixed).
constexpr int GT_WARPS = 8;
constexpr int GT_CHUNK = 64;   // column pairs per warp
__global__ void __launch_bounds__(GT_WARPS * 32) k_grad_T(int nrows, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const int8_t* __restrict__ sgn,
                                                          const double* __restrict__ r, double* __restrict__ y,
                                                          int ncols) {
  pdl_entry();
  __shared__ int s_col[GT_WARPS][32];
  __shared__ double s_sgn[GT_WARPS][32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int v = blockIdx.x * GT_WARPS + wb;
  if (v >= nrows) return;
  const int64_t beg = rowptr[v];
  const int nq = (int)(rowptr[v + 1] - beg);
  if (nq > 32 || (ncols & 1)) {   // general case (not reached on Kuhn meshes: <= 14 edges per vertex)
    if (blockIdx.y > 0) return;
    for (int j = lane; j < ncols; j += 32) {
      double sum = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double rv = r[(int64_t)col[beg + q] * ncols + j];
        sum = sgn[beg + q] > 0 ? sum + rv : sum - rv;
      }
      y[(int64_t)v * ncols + j] = sum;
    }
    return;
  }
  if (lane < nq) {
    s_col[wb][lane] = col[beg + lane];
    s_sgn[wb][lane] = sgn[beg + lane] > 0 ? 1.0 : -1.0;
  }
  __syncwarp();
  const int* cq = s_col[wb];
  const double* sq = s_sgn[wb];
  const int n2 = ncols >> 1;
  const double2* r2 = reinterpret_cast<const double2*>(r);
  double2* y2 = reinterpret_cast<double2*>(y + (int64_t)v * ncols);
  // blockIdx.y: a chunk of GT_CHUNK column pairs (more warps in flight on long rows)
  const int j1 = min(n2, (int)(blockIdx.y + 1) * GT_CHUNK);
  for (int j = (int)blockIdx.y * GT_CHUNK + lane; j < j1; j += 32) {
    double2 sum = make_double2(0.0, 0.0);
    int q = 0;
    for (; q + 4 <= nq; q += 4) {
      double2 rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) rv[u] = r2[(int64_t)cq[q + u] * n2 + j];
      // sum +- r as one FMA with the sign +-1 (the product is exact: the same rounding as
      // the add or subtract, one FP64 operation; this kernel is bound by the FP64 pipe)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sum.x = fma(sq[q + u], rv[u].x, sum.x);
        sum.y = fma(sq[q + u], rv[u].y, sum.y);
      }
    }
    for (; q < nq; ++q) {
      const double2 rv = r2[(int64_t)cq[q] * n2 + j];
      sum.x = fma(sq[q], rv.x, sum.x);
      sum.y = fma(sq[q], rv.y, sum.y);
    }
    y2[j] = sum;
  }
}
// x += G w: one block per interior edge, double2 column pairs.
__global__ void k_grad_add(const int32_t* __restrict__ tail, const int32_t* __restrict__ head,
                           const double* __restrict__ w, double* __restrict__ x, int ncols) {
  pdl_entry();
  const int e = blockIdx.x;
  const int t = tail[e], h = head[e];
  double* xr = x + (int64_t)e * ncols;
  if (ncols & 1) {
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
      double d = 0.0;
      if (h >= 0) d += w[(int64_t)h * ncols + j];
      if (t >= 0) d -= w[(int64_t)t * ncols + j];
      xr[j] += d;
    }
    return;
  }
  const int n2 = ncols >> 1;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* x2 = reinterpret_cast<double2*>(xr);
  for (int j = threadIdx.x; j < n2; j += blockDim.x) {   // (one or two iterations at 256 slabs)
    double2 d = make_double2(0.0, 0.0);
    if (h >= 0) {
      const double2 a = w2[(int64_t)h * n2 + j];
      d.x += a.x;
      d.y += a.y;
    }
    if (t >= 0) {
      const double2 b = w2[(int64_t)t * n2 + j];
      d.x -= b.x;
      d.y -= b.y;
    }
    double2 xv = x2[j];
    xv.x += d.x;
    xv.y += d.y;
    x2[j] = xv;
  }
}
// The same update with one warp per edge (GA_WARPS edges per block) and the loads of
// GA_UNROLL column pairs per lane issued before their sums: the x row and the two w rows
// of an edge are in flight together.  The same values up to the sign of an exact zero.
constexpr int GA_WARPS = 8;
constexpr int GA_UNROLL = 4;
__global__ void __launch_bounds__(GA_WARPS * 32) k_grad_add_w(const int32_t* __restrict__ tail,
                                                              const int32_t* __restrict__ head,
                                                              const double* __restrict__ w, double* __restrict__ x,
                                                              int nedges, int ncols) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * GA_WARPS + (threadIdx.x >> 5);
  if (e >= nedges) return;
  const int t = tail[e], h = head[e];
  const int n2 = ncols >> 1;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* x2 = reinterpret_cast<double2*>(x + (int64_t)e * ncols);
  const double2 zero = make_double2(0.0, 0.0);
  for (int j0 = 0; j0 < n2; j0 += 32 * GA_UNROLL) {
    double2 xv[GA_UNROLL], a[GA_UNROLL], b[GA_UNROLL];
#pragma unroll
    for (int u = 0; u < GA_UNROLL; ++u) {
      const int j = j0 + u * 32 + lane;
      const bool in = j < n2;
      xv[u] = in ? x2[j] : zero;
      a[u] = (in && h >= 0) ? w2[(int64_t)h * n2 + j] : zero;
      b[u] = (in && t >= 0) ? w2[(int64_t)t * n2 + j] : zero;
    }
#pragma unroll
    for (int u = 0; u < GA_UNROLL; ++u) {
      const int j = j0 + u * 32 + lane;
      if (j >= n2) continue;
      // w_head - w_tail once, then x += it: two FP64 operations per entry (the FP64 pipe
      // bounds this kernel); a boundary endpoint contributes nothing
      double2 d;
      if (h >= 0 && t >= 0) {
        d.x = a[u].x - b[u].x;
        d.y = a[u].y - b[u].y;
      } else if (h >= 0) {
        d = a[u];
      } else if (t >= 0) {
        d.x = -b[u].x;
        d.y = -b[u].y;
      } else {
        d = zero;
      }
      xv[u].x += d.x;
      xv[u].y += d.y;
      x2[j] = xv[u];
    }
  }
}

// CARRY: the time grid continues an earlier one whose last slab held w_{-1} = carry[v]
// (q values per node), the state a time-slab shard receives from the shard before it.
// The recurrence's homogeneous part is T = -K_t^{-1} N_t: 1 for DG(0), [[1,1],[0,0]]
// for DG(1), both idempotent (T^k = T), so w_n gains T carry for every n: the running
// sum starts at carry (DG(0)) or at carry_0 + carry_1 (DG(1)).
template <bool CARRY>
__global__ void k_time_integrate(const double* __restrict__ z, double* __restrict__ w, int nrows, int N_t,
                                 int degree, const double* __restrict__ carry) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= nrows) return;
  const int q = degree + 1;
  const int C = (N_t + 31) / 32;
  const int n0 = lane * C, n1 = min(N_t, n0 + C);
  const double* zr = z + (int64_t)v * N_t * q;
  double* wr = w + (int64_t)v * N_t * q;
  double s = 0.0;
  for (int n = n0; n < n1; ++n) s += zr[n * q];
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  double e = incl - s;   // exclusive carry
  if (CARRY) e += degree == 0 ? carry[v] : carry[2 * v] + carry[2 * v + 1];
  for (int n = n0; n < n1; ++n) {
    if (degree == 0) {
      e += zr[n];
      wr[n] = e;
    } else {
      const double z0 = zr[2 * n], z1 = zr[2 * n + 1];
      wr[2 * n] = 0.5 * (z0 - z1) + e;
      wr[2 * n + 1] = 0.5 * (z0 + z1);
      e += z0;
    }
  }
}

// The same scan with the row staged in shared memory: the row is read and written with
// coalesced warp-wide accesses (a lane's own chunk of C consecutive slabs is strided by
// C slabs across the warp in global memory), and the chunks sit Cp >= C + 1 entries
// apart in shared memory (Cp odd) so that the lanes' chunk reads hit distinct banks.
// Same chunks, same operations in the same order as k_time_integrate: bit-identical.
// smem per warp: 32 Cp values of q doubles; rows of up to TI_MAX_SLABS slabs.
constexpr int TI_MAX_SLABS = 2048;
template <int Q, bool CARRY>
__global__ void k_time_integrate_s(const double* __restrict__ z, double* __restrict__ w, int nrows, int N_t,
                                   const double* __restrict__ carry) {
  pdl_entry();
  extern __shared__ __align__(16) double ti_smem[];
  using V = typename std::conditional<Q == 2, double2, double>::type;
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int C = (N_t + 31) / 32;
  const int Cp = (C + 1) | 1;
  V* sv = reinterpret_cast<V*>(ti_smem) + (int64_t)wb * 32 * Cp;
  const int v = blockIdx.x * (blockDim.x >> 5) + wb;
  if (v >= nrows) return;
  const V* zr = reinterpret_cast<const V*>(z + (int64_t)v * N_t * Q);
  V* wr = reinterpret_cast<V*>(w + (int64_t)v * N_t * Q);
  for (int i = lane; i < N_t; i += 32) sv[(i / C) * Cp + i % C] = zr[i];
  __syncwarp();
  const int n0 = lane * C, n1 = min(N_t, n0 + C);
  V* my = sv + lane * Cp - n0;   // my[n] = slab n of this lane's chunk
  double s = 0.0;
  for (int n = n0; n < n1; ++n) {
    if constexpr (Q == 2) s += my[n].x;
    else s += my[n];
  }
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  double e = incl - s;   // exclusive carry
  if (CARRY) {
    if constexpr (Q == 1) e += carry[v];
    else e += carry[2 * v] + carry[2 * v + 1];
  }
  for (int n = n0; n < n1; ++n) {
    if constexpr (Q == 1) {
      e += my[n];
      my[n] = e;
    } else {
      const double z0 = my[n].x, z1 = my[n].y;
      my[n] = make_double2(0.5 * (z0 - z1) + e, 0.5 * (z0 + z1));
      e += z0;
    }
  }
  __syncwarp();
  for (int i = lane; i < N_t; i += 32) wr[i] = sv[(i / C) * Cp + i % C];
}

// ---- per-column power-of-two scaling of complex FP32 columns (FP16 slab solve).
// Thread t of block (bx, by) owns column bx * 128 + t and rows by * COL_ROWS ...: loads
// of consecutive threads are consecutive columns of one row (coalesced).
constexpr int COL_THREADS = 128;
constexpr int COL_ROWS = 256;

__device__ __forceinline__ float col_factor(unsigned bits) {
  // s = 2^(1 - e) for max = m 2^e, m in [0.5, 1): max * s in [1, 2); 1 for a zero column
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f)) return 1.f;
  int e;
  frexpf(mx, &e);
  return ldexpf(1.f, 1 - e);
}

__global__ void k_col_absmax(const float2* __restrict__ Q, int nrows, int cnt, int ld, unsigned* __restrict__ colmax) {
  pdl_entry();
  const int c = blockIdx.x * COL_THREADS + threadIdx.x;
  if (c >= cnt) return;
  const int r0 = blockIdx.y * COL_ROWS, r1 = min(nrows, r0 + COL_ROWS);
  float m = 0.f;
  for (int r = r0; r < r1; ++r) {
    const float2 v = Q[(int64_t)r * ld + c];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  atomicMax(colmax + c, __float_as_uint(m));   // non-negative floats order as their bit patterns
}

template <bool UNSCALE>
__global__ void k_col_scale(float2* __restrict__ Q, int nrows, int cnt, int ld, const unsigned* __restrict__ colmax) {
  pdl_entry();
  const int c = blockIdx.x * COL_THREADS + threadIdx.x;
  if (c >= cnt) return;
  const float s0 = col_factor(colmax[c]);
  const float s = UNSCALE ? 1.f / s0 : s0;   // exact: a power of two
  const int r0 = blockIdx.y * COL_ROWS, r1 = min(nrows, r0 + COL_ROWS);
  for (int r = r0; r < r1; ++r) {
    float2 v = Q[(int64_t)r * ld + c];
    v.x *= s;
    v.y *= s;
    Q[(int64_t)r * ld + c] = v;
  }
}

__global__ void k_fill_u32(unsigned* v, int n, unsigned value) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = value;
}

// ---- time-slab sharding (the time axis split into contiguous slab ranges, one per
// rank, Section 2.1's time-parallel groups): the two couplings between ranges.
// out[row q + i] = v[row ld + off + i]: one slab of every row (the halo a range sends on).
__global__ void k_slab_copy(const double* __restrict__ v, int64_t ld, int64_t off, int q, int nrows,
                            double* __restrict__ out) {
  pdl_entry();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrows * q) return;
  out[t] = v[(t / q) * ld + off + t % q];
}

// r_0 -= (N_t (x) M) xh: the history term of a range's first slab, xh = the last slab of
// the range before it (DG(0): N_t = -1; DG(1): N_t = [[-1,-1],[1,1]]).
__global__ void k_halo_history(int nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ m, const double* __restrict__ xh, double* __restrict__ r,
                               int64_t ld, int degree) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nrows) return;
  double mx0 = 0.0, mx1 = 0.0;
  for (int64_t p = rowptr[e]; p < rowptr[e + 1]; ++p) {
    if (degree == 0) {
      mx0 = fma(m[p], xh[col[p]], mx0);
    } else {
      mx0 = fma(m[p], xh[2 * (int64_t)col[p]], mx0);
      mx1 = fma(m[p], xh[2 * (int64_t)col[p] + 1], mx1);
    }
  }
  if (degree == 0) {
    r[e * ld] += mx0;
  } else {
    const double s = mx0 + mx1;
    r[e * ld] += s;
    r[e * ld + 1] -= s;
  }
}

// Carry into range n_prev from the local end states of the ranges before it (exclusive
// scan over ranges): c_0 = 0, c_{k+1} = e_k + T c_k, T as in k_time_integrate (every
// range holds at least one slab, so T^{len} = T).  ends[k][v q + i].
__global__ void k_time_carry(const double* __restrict__ ends, int n_prev, int nrows, int degree,
                             double* __restrict__ carry) {
  pdl_entry();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nrows) return;
  const int q = degree + 1;
  double c0 = 0.0, c1 = 0.0;
  for (int k = 0; k < n_prev; ++k) {
    const double* ek = ends + ((int64_t)k * nrows + v) * q;
    if (degree == 0) {
      c0 = ek[0] + c0;
    } else {
      c0 = ek[0] + (c0 + c1);
      c1 = ek[1];
    }
  }
  carry[(int64_t)v * q] = c0;
  if (degree == 1) carry[(int64_t)v * q + 1] = c1;
}

__global__ void k_nodal_jacobi(int nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ kv, const double* __restrict__ dinv,
                               const double* __restrict__ y, const double* __restrict__ zi, double* __restrict__ zo,
                               int ncols, double wgt) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= nrows) return;
  const int64_t beg = rowptr[v], end = rowptr[v + 1];
  const double dv = dinv[v] * wgt;
  for (int j = lane; j < ncols; j += 32) {
    double s = 0.0;
    for (int64_t q = beg; q < end; ++q) s = fma(kv[q], zi[(int64_t)col[q] * ncols + j], s);
    const int64_t o = (int64_t)v * ncols + j;
    zo[o] = zi[o] + dv * (y[o] - s);
  }
}

// Time restriction r_c = P_t^T r and prolongation x += P_t e_c between 2 Nc fine and
// Nc coarse slabs.  DG(0): a coarse slab is the two fine slabs (P_t = [1; 1]).  DG(1),
// Legendre basis: coarse (1, 2s-1) restricted to the first fine half is
// (1, -1/2 + phi_1/2), to the second (1, 1/2 + phi_1/2), i.e. the blocks
// P0 = [[1, -1/2], [0, 1/2]] and P1 = [[1, 1/2], [0, 1/2]].
// Row blockIdx.x = (edge e, problem p) of the fine level, Bf problems per edge row; the
// coarse level holds Bc >= Bf problems per edge row (a ragged batch adds the problems
// whose own finest level it is after the fine level's ones), so row (e, p) lands at
// e Bc + p.  Bf = Bc: contiguous rows.
__global__ void k_time_restrict(const double* __restrict__ r, double* __restrict__ rc, int Nc, int degree, int Bf,
                                int Bc) {
  pdl_entry();
  const int ef = blockIdx.x;
  const int e = (Bf == Bc) ? ef : (ef / Bf) * Bc + ef % Bf;
  if (degree == 0) {
    const double* src = r + (int64_t)ef * 2 * Nc;
    double* dst = rc + (int64_t)e * Nc;
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) dst[k] = src[2 * k] + src[2 * k + 1];
  } else {
    const double2* src = reinterpret_cast<const double2*>(r + (int64_t)ef * 4 * Nc);
    double2* dst = reinterpret_cast<double2*>(rc + (int64_t)e * 2 * Nc);
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
      const double2 a = src[2 * k], b = src[2 * k + 1];   // fine slab 2k and 2k+1, (i=0, i=1)
      dst[k] = make_double2(a.x + b.x, 0.5 * (a.y - a.x + b.x + b.y));
    }
  }
}

// Row blockIdx.x = (edge e, problem p) of the fine level; its coarse row is e Bc + p (see
// k_time_restrict).
__global__ void k_time_prolong_add(const double* __restrict__ ec, double* __restrict__ x, int Nc, int degree, int Bf,
                                   int Bc) {
  pdl_entry();
  const int ef = blockIdx.x;
  const int e = (Bf == Bc) ? ef : (ef / Bf) * Bc + ef % Bf;
  if (degree == 0) {
    const double* src = ec + (int64_t)e * Nc;
    double* dst = x + (int64_t)ef * 2 * Nc;
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
      const double v = src[k];
      dst[2 * k] += v;
      dst[2 * k + 1] += v;
    }
  } else {
    const double2* src = reinterpret_cast<const double2*>(ec + (int64_t)e * 2 * Nc);
    double2* dst = reinterpret_cast<double2*>(x + (int64_t)ef * 4 * Nc);
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
      const double2 v = src[k];
      double2 a = dst[2 * k], b = dst[2 * k + 1];
      a.x += v.x - 0.5 * v.y;
      a.y += 0.5 * v.y;
      b.x += v.x + 0.5 * v.y;
      b.y += 0.5 * v.y;
      dst[2 * k] = a;
      dst[2 * k + 1] = b;
    }
  }
}

__global__ void k_csr_spmm(int nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ pv, const double* __restrict__ in, double* __restrict__ out,
                           int ncols, int beta) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int rrow = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (rrow >= nrows) return;
  const int64_t beg = rowptr[rrow], end = rowptr[rrow + 1];
  for (int j = lane; j < ncols; j += 32) {
    double s = 0.0;
    for (int64_t q = beg; q < end; ++q) s = fma(pv[q], in[(int64_t)col[q] * ncols + j], s);
    const int64_t o = (int64_t)rrow * ncols + j;
    out[o] = beta ? out[o] + s : s;
  }
}

__global__ void k_history_rhs(int nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ m, const double* __restrict__ f,
                              const double* __restrict__ x, double* __restrict__ g, int N_t, int n, int degree) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nrows) return;
  const int q = degree + 1;
  const int64_t ld = (int64_t)N_t * q;
  double mx0 = 0.0, mx1 = 0.0;
  if (n > 0) {
    for (int64_t p = rowptr[e]; p < rowptr[e + 1]; ++p) {
      const double* xr = x + (int64_t)col[p] * ld + (int64_t)(n - 1) * q;
      mx0 = fma(m[p], xr[0], mx0);
      if (degree == 1) mx1 = fma(m[p], xr[1], mx1);
    }
  }
  if (degree == 0) {
    g[e] = f[e * ld + n] + mx0;                      // -N_t M x_{n-1} with N_t = -1
  } else {
    const double s = mx0 + mx1;                      // N_t = [[-1,-1],[1,1]]
    g[2 * e] = f[e * ld + 2 * n] + s;
    g[2 * e + 1] = f[e * ld + 2 * n + 1] - s;
  }
}

__global__ void k_fill(double* v, int64_t n, double value) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = value;
}
__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
__global__ void k_outer_load(const double* __restrict__ b, const double* __restrict__ c, double* __restrict__ f,
                             int ncols, int row_stride) {
  pdl_entry();
  const int e = blockIdx.x;
  const double be = b[e];
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) f[(int64_t)e * row_stride + j] = c[j] * be;
}

// Per-problem sums of squares of a batched vector v[e][b * seg + j]: block (x, b)
// sums rows x, x + gridDim.x, ... of problem b in a fixed order.
__global__ void k_batch_norm_partial(const double* __restrict__ v, int nrows, int nb, int seg,
                                     double* __restrict__ partial) {
  pdl_entry();
  const int b = blockIdx.y;
  double s = 0.0;
  for (int e = blockIdx.x; e < nrows; e += gridDim.x) {
    const double* row = v + ((int64_t)e * nb + b) * seg;
    for (int j = threadIdx.x; j < seg; j += blockDim.x) s = fma(row[j], row[j], s);
  }
  block_sum_store<256>(s, partial + (int64_t)b * gridDim.x + blockIdx.x);
}

__global__ void k_batch_norm_final(const double* __restrict__ partial, int g, double* __restrict__ out) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < g; i += blockDim.x) s += partial[(int64_t)blockIdx.x * g + i];
  block_sum_store<256>(s, out + blockIdx.x);
}

// v[e * stride + offset + j] = 0 for j < count (one problem's columns of a batched vector)
__global__ void k_zero_cols(double* __restrict__ v, int nrows, int stride, int offset, int count) {
  pdl_entry();
  for (int e = blockIdx.x; e < nrows; e += gridDim.x)
    for (int j = threadIdx.x; j < count; j += blockDim.x) v[(int64_t)e * stride + offset + j] = 0.0;
}

// FP64 pipe throughput probe: eight independent FMA chains per thread.
__global__ void k_fp64_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = warp_sum(x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7);
  if ((threadIdx.x & 31) == 0 && s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live
}

unsigned grid1(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

std::atomic<int64_t> g_launches{0};

}  // namespace

int64_t launch_count() { return g_launches.load(); }
void count_launches(int64_t n) { g_launches += n; }
std::atomic<bool> g_overlap{false};
bool launch_overlap() { return g_overlap.load(std::memory_order_relaxed); }
void set_launch_overlap(bool on) { g_overlap.store(on); }

int residual_blocks(int nrows) { return (nrows + RES_WARPS - 1) / RES_WARPS; }

// lanes per row: the smallest power of two whose SPL-slab passes cover N_t (<= 32)
int lanes_per_row(int N_t) {
  int l = 1;
  while (l < 32 && l * SPL < N_t) l <<= 1;
  return l;
}

#define STMG_RES_DISPATCH_T(KERNEL, T, ...)                                                              \
  do {                                                                                              \
    const int lpr = lanes_per_row(N_t);                                                             \
    const int rows_per_block = RES_WARPS * (32 / lpr);                                              \
    const int nb = (A.nrows + rows_per_block - 1) / rows_per_block;                                 \
    if (nblocks) *nblocks = nb;                                                                     \
    if (nb <= 0) break;                                                                             \
    switch (lpr) {                                                                                  \
      case 1: launch_k(KERNEL<1, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
      case 2: launch_k(KERNEL<2, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
      case 4: launch_k(KERNEL<4, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
      case 8: launch_k(KERNEL<8, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
      case 16: launch_k(KERNEL<16, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
      default: launch_k(KERNEL<32, T>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break; \
    }                                                                                               \
    count_launches(1);                                                                              \
  } while (0)

#define STMG_RES_DISPATCH(KERNEL, ...)                                                              \
  do {                                                                                              \
    const int lpr = lanes_per_row(N_t);                                                             \
    const int rows_per_block = RES_WARPS * (32 / lpr);                                              \
    const int nb = (A.nrows + rows_per_block - 1) / rows_per_block;                                 \
    if (nblocks) *nblocks = nb;                                                                     \
    if (nb <= 0) break;                                                                             \
    switch (lpr) {                                                                                  \
      case 1: launch_k(KERNEL<1>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                   \
      case 2: launch_k(KERNEL<2>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                   \
      case 4: launch_k(KERNEL<4>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                   \
      case 8: launch_k(KERNEL<8>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                   \
      case 16: launch_k(KERNEL<16>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                 \
      default: launch_k(KERNEL<32>, nb, RES_WARPS * 32, 0, st, __VA_ARGS__); break;                 \
    }                                                                                               \
    count_launches(1);                                                                              \
  } while (0)

cudaError_t residual_dg0(CsrView A, const double* a, const double* m, const double* f, const double* x, double* r,
                         int N_t, int seg, double* partial, int* nblocks, cudaStream_t st) {
  STMG_RES_DISPATCH_T(k_residual_dg0, double, A.nrows, A.rowptr, A.col, a, m, f, x, r, N_t, partial, seg);
  return cudaGetLastError();
}

cudaError_t residual_dg1(CsrView A, const double* m, const double* k0, const double* k1, const double* f,
                         const double* x, double* r, int N_t, int seg, double* partial, int* nblocks, cudaStream_t st) {
  STMG_RES_DISPATCH_T(k_residual_dg1, double, A.nrows, A.rowptr, A.col, m, k0, k1, f, x, r, N_t, partial, seg);
  return cudaGetLastError();
}

constexpr int BATCH_NORM_BLOCKS = 256;
int batch_norm_scratch(int nb) { return nb * BATCH_NORM_BLOCKS; }

cudaError_t batch_norms_sq(const double* v, int nrows, int nb, int seg, double* partial, double* out,
                           cudaStream_t st) {
  if (nrows <= 0 || nb <= 0) return cudaSuccess;
  { launch_k(k_batch_norm_partial, dim3(BATCH_NORM_BLOCKS, nb), 256, 0, st, v, nrows, nb, seg, partial); count_launches(1); }
  { launch_k(k_batch_norm_final, nb, 256, 0, st, partial, BATCH_NORM_BLOCKS, out); count_launches(1); }
  return cudaGetLastError();
}

cudaError_t zero_cols(double* v, int nrows, int stride, int offset, int count, cudaStream_t st) {
  if (nrows > 0 && count > 0) {
    launch_k(k_zero_cols, (unsigned)std::min(nrows, 4096), 128, 0, st, v, nrows, stride, offset, count);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t fp64_probe(double* out, int blocks, int iters, cudaStream_t st) {
  { k_fp64_probe<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7); count_launches(1); }
  return cudaGetLastError();
}

cudaError_t residual_dg0_f32(CsrView A, const float* a, const float* m, const double* f, const float* xf, double* r,
                             int N_t, int seg, double* partial, int* nblocks, cudaStream_t st) {
  STMG_RES_DISPATCH_T(k_residual_dg0, float, A.nrows, A.rowptr, A.col, a, m, f, xf, r, N_t, partial, seg);
  return cudaGetLastError();
}
cudaError_t residual_dg1_f32(CsrView A, const float* m, const float* k0, const float* k1, const double* f,
                             const float* xf, double* r, int N_t, int seg, double* partial, int* nblocks,
                             cudaStream_t st) {
  STMG_RES_DISPATCH_T(k_residual_dg1, float, A.nrows, A.rowptr, A.col, m, k0, k1, f, xf, r, N_t, partial, seg);
  return cudaGetLastError();
}
cudaError_t to_float(const double* x, float* xf, int64_t n, cudaStream_t st) {
  if (n > 0) {
    launch_k(k_to_float, (unsigned)std::min<int64_t>(grid1(n, 256), 8 * 1024), 256, 0, st, x, xf, n);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vec_add(const double* a, double* b, int64_t n, cudaStream_t st) {
  if (n > 0) {
    launch_k(k_vec_add, (unsigned)std::min<int64_t>(grid1(n, 256), 8 * 1024), 256, 0, st, a, b, n);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t split_pairs(const double* x, float2* xs, int64_t n, cudaStream_t st) {
  if (n > 0) { launch_k(k_split_pairs, (unsigned)std::min<int64_t>(grid1(n, 256), 8 * 1024), 256, 0, st, x, xs, n); count_launches(1); }
  return cudaGetLastError();
}

cudaError_t residual_dg0_df(CsrView A, const float2* a, const float2* m, const double* f, const float2* xs, double* r,
                            int N_t, int seg, double* partial, int* nblocks, cudaStream_t st) {
  STMG_RES_DISPATCH(k_residual_dg0_df, A.nrows, A.rowptr, A.col, a, m, f, xs, r, N_t, partial, seg);
  return cudaGetLastError();
}

cudaError_t residual_dg1_df(CsrView A, const float2* m, const float2* k0, const float2* k1, const double* f,
                            const float2* xs, double* r, int N_t, int seg, double* partial, int* nblocks, cudaStream_t st) {
  STMG_RES_DISPATCH(k_residual_dg1_df, A.nrows, A.rowptr, A.col, m, k0, k1, f, xs, r, N_t, partial, seg);
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partial, int n, double* out, cudaStream_t st) {
  { launch_k(k_reduce_partials, 1, 256, 0, st, partial, n, out); count_launches(1); }
  return cudaGetLastError();
}

cudaError_t norm2_sq(const double* v, int64_t n, double* partial, double* out, cudaStream_t st) {
  { launch_k(k_norm_partial, NORM_BLOCKS, 256, 0, st, v, n, partial); count_launches(1); }
  { launch_k(k_reduce_partials, 1, 256, 0, st, partial, NORM_BLOCKS, out); count_launches(1); }
  return cudaGetLastError();
}

cudaError_t slab_pre_dg0(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                         double* Q, int ld, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_pre_dg0, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, r, src_ld, slab0, cnt, iperm, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_pre_dg1(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                         double2 c0, double2 c1, double2* Q, int ld, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_pre_dg1, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, r, src_ld, slab0, cnt, iperm, c0, c1, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_post_dg0(const double* X, int ld, const int32_t* iperm, int nrows, double* x, int dst_ld,
                          int slab0, int cnt, double omega, int mode, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_post_dg0, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, x, dst_ld, slab0, cnt, omega, mode); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_post_dg1(const double2* X, int ld, const int32_t* iperm, int nrows, double2 s1, double* x,
                          int dst_ld, int slab0, int cnt, double omega, int mode, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_post_dg1, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, s1, x, dst_ld, slab0, cnt, omega, mode); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_pre_dg0f(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                          float* Q, int ld, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_pre_dg0f, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, r, src_ld, slab0, cnt, iperm, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_pre_dg1f(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                          double2 c0, double2 c1, float2* Q, int ld, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_pre_dg1f, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, r, src_ld, slab0, cnt, iperm, c0, c1, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_post_dg0f(const float* X, int ld, const int32_t* iperm, int nrows, double* x, int dst_ld,
                           int slab0, int cnt, double omega, int mode, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_post_dg0f, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, x, dst_ld, slab0, cnt, omega, mode); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t slab_post_dg1f(const float2* X, int ld, const int32_t* iperm, int nrows, double2 s1, double* x,
                           int dst_ld, int slab0, int cnt, double omega, int mode, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_slab_post_dg1f, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, s1, x, dst_ld, slab0, cnt, omega, mode); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t gather_perm(const double* y, int ncols, const int32_t* iperm, int nrows, double* Q, int ld,
                        cudaStream_t st) {
  if (nrows > 0) { launch_k(k_gather_perm<double>, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, y, ncols, iperm, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t scatter_perm(const double* X, int ld, const int32_t* iperm, int nrows, double* z, int ncols,
                         cudaStream_t st) {
  if (nrows > 0) { launch_k(k_scatter_perm<double>, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, z, ncols); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t gather_perm_f(const double* y, int ncols, const int32_t* iperm, int nrows, float* Q, int ld,
                          cudaStream_t st) {
  if (nrows > 0) { launch_k(k_gather_perm<float>, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, y, ncols, iperm, Q, ld); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t scatter_perm_f(const float* X, int ld, const int32_t* iperm, int nrows, double* z, int ncols,
                           cudaStream_t st) {
  if (nrows > 0) { launch_k(k_scatter_perm<float>, grid1(nrows, SLAB_ROWS), SLAB_ROWS * 32, 0, st, nrows, X, ld, iperm, z, ncols); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t grad_T(CsrView GT, const int8_t* gt_sign, const double* r, double* y, int ncols, cudaStream_t st) {
  if (GT.nrows > 0) { launch_k(k_grad_T, dim3(grid1(GT.nrows, GT_WARPS), (unsigned)std::max<int64_t>(1, grid1(ncols / 2, GT_CHUNK))), GT_WARPS * 32, 0, st, GT.nrows, GT.rowptr, GT.col, gt_sign, r, y, ncols); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t grad_add(const int32_t* tail, const int32_t* head, int nedges, const double* w, double* x, int ncols,
                     cudaStream_t st) {
  if (nedges <= 0) return cudaSuccess;
  if (ncols & 1)
    launch_k(k_grad_add, nedges, 128, 0, st, tail, head, w, x, ncols);
  else
    launch_k(k_grad_add_w, grid1(nedges, GA_WARPS), GA_WARPS * 32, 0, st, tail, head, w, x, nedges, ncols);
  count_launches(1);
  return cudaGetLastError();
}
// Shared-memory scan when the rows fit (warps per block so that a block holds <= 48 KiB),
// the register scan otherwise.
template <bool CARRY>
void time_integrate_launch(const double* z, const double* carry, double* w, int nrows, int N_t, int degree,
                           cudaStream_t st) {
  if (nrows <= 0) return;
  const int q = degree + 1;
  const int C = (N_t + 31) / 32;
  const size_t warp_bytes = (size_t)32 * ((C + 1) | 1) * q * sizeof(double);
  if (N_t > TI_MAX_SLABS) {
    launch_k(k_time_integrate<CARRY>, grid1(nrows, 8), 256, 0, st, z, w, nrows, N_t, degree, carry);
  } else {
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / warp_bytes));
    const size_t smem = warp_bytes * wpb;
    if (degree == 0)
      launch_k(k_time_integrate_s<1, CARRY>, grid1(nrows, wpb), wpb * 32, smem, st, z, w, nrows, N_t, carry);
    else
      launch_k(k_time_integrate_s<2, CARRY>, grid1(nrows, wpb), wpb * 32, smem, st, z, w, nrows, N_t, carry);
  }
  count_launches(1);
}

cudaError_t time_integrate(const double* z, double* w, int nrows, int N_t, int degree, cudaStream_t st) {
  time_integrate_launch<false>(z, nullptr, w, nrows, N_t, degree, st);
  return cudaGetLastError();
}
cudaError_t col_scale(float2* Q, int nrows, int cnt, int ld, unsigned* colmax, cudaStream_t st) {
  if (nrows <= 0 || cnt <= 0) return cudaSuccess;
  const dim3 g(grid1(cnt, COL_THREADS), grid1(nrows, COL_ROWS));
  launch_k(k_fill_u32, grid1(cnt, 256), 256, 0, st, colmax, cnt, 0u);
  launch_k(k_col_absmax, g, COL_THREADS, 0, st, Q, nrows, cnt, ld, colmax);
  launch_k(k_col_scale<false>, g, COL_THREADS, 0, st, Q, nrows, cnt, ld, colmax);
  count_launches(3);
  return cudaGetLastError();
}
cudaError_t col_unscale(float2* Q, int nrows, int cnt, int ld, const unsigned* colmax, cudaStream_t st) {
  if (nrows <= 0 || cnt <= 0) return cudaSuccess;
  const dim3 g(grid1(cnt, COL_THREADS), grid1(nrows, COL_ROWS));
  launch_k(k_col_scale<true>, g, COL_THREADS, 0, st, Q, nrows, cnt, ld, colmax);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t time_integrate_carry(const double* z, const double* carry, double* w, int nrows, int N_t, int degree,
                                 cudaStream_t st) {
  time_integrate_launch<true>(z, carry, w, nrows, N_t, degree, st);
  return cudaGetLastError();
}
cudaError_t slab_copy(const double* v, int64_t ld, int64_t off, int q, int nrows, double* out, cudaStream_t st) {
  const int64_t n = (int64_t)nrows * q;
  if (n > 0) { launch_k(k_slab_copy, (unsigned)grid1(n, 256), 256, 0, st, v, ld, off, q, nrows, out); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t halo_history(CsrView A, const double* m, const double* xh, double* r, int64_t ld, int degree,
                         cudaStream_t st) {
  if (A.nrows > 0) { launch_k(k_halo_history, grid1(A.nrows, 128), 128, 0, st, A.nrows, A.rowptr, A.col, m, xh, r, ld, degree); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t time_carry(const double* ends, int n_prev, int nrows, int degree, double* carry, cudaStream_t st) {
  if (nrows > 0) { launch_k(k_time_carry, grid1(nrows, 128), 128, 0, st, ends, n_prev, nrows, degree, carry); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t nodal_jacobi(CsrView Kn, const double* kval, const double* dinv, const double* y, const double* zi,
                         double* zo, int ncols, double wgt, cudaStream_t st) {
  if (Kn.nrows > 0)
    { launch_k(k_nodal_jacobi, grid1(Kn.nrows, 8), 256, 0, st, Kn.nrows, Kn.rowptr, Kn.col, kval, dinv, y, zi, zo, ncols,
                                                       wgt); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t time_restrict(const double* r, double* rc, int nrows, int Nc, int degree, cudaStream_t st, int Bf,
                          int Bc) {
  if (nrows > 0) { launch_k(k_time_restrict, nrows, 128, 0, st, r, rc, Nc, degree, Bf, Bc); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t time_prolong_add(const double* ec, double* x, int nrows, int Nc, int degree, cudaStream_t st, int Bf,
                             int Bc) {
  if (nrows > 0) { launch_k(k_time_prolong_add, nrows, 128, 0, st, ec, x, Nc, degree, Bf, Bc); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t csr_spmm(CsrView P, const double* pval, const double* in, double* out, int ncols, int beta,
                     cudaStream_t st) {
  if (P.nrows > 0) { launch_k(k_csr_spmm, grid1(P.nrows, 8), 256, 0, st, P.nrows, P.rowptr, P.col, pval, in, out, ncols, beta); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t history_rhs(CsrView A, const double* m, const double* f, const double* x, double* g, int N_t, int n,
                        int degree, cudaStream_t st) {
  if (A.nrows > 0) { launch_k(k_history_rhs, grid1(A.nrows, 128), 128, 0, st, A.nrows, A.rowptr, A.col, m, f, x, g, N_t, n, degree); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t vec_fill(double* v, int64_t n, double value, cudaStream_t st) {
  if (n > 0) { launch_k(k_fill, (unsigned)std::min<int64_t>(grid1(n, 256), 4096), 256, 0, st, v, n, value); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t vec_copy(const double* a, double* b, int64_t n, cudaStream_t st) {
  if (n > 0) { launch_k(k_copy, (unsigned)std::min<int64_t>(grid1(n, 256), 4096), 256, 0, st, a, b, n); count_launches(1); }
  return cudaGetLastError();
}
cudaError_t outer_load(const double* b, const double* c, double* f, int nrows, int ncols, int row_stride,
                       cudaStream_t st) {
  if (nrows > 0) { launch_k(k_outer_load, nrows, 128, 0, st, b, c, f, ncols, row_stride); count_launches(1); }
  return cudaGetLastError();
}

}  // namespace stmg
