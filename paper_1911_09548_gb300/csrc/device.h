// Launch interface between the host runtime and the CUDA kernels.  Plain
// pointers and sizes only; every launcher queues work on `st` and returns the
// launch status (cudaGetLastError) without synchronising.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace stmg {

// One supernode of a nested-dissection factor as the GPU sees it.
struct DevNode {
  int32_t col0, nc, nr, pad;
  int64_t w_off, row_off, u_off, g_off;
};

// Row tile height of the supernodal products (tiles are built on the host with it).
constexpr int kSnBM = 64;
constexpr int kSnBmFP64 = 16;   // tile rows of the FP64 factors' tiled path (DevFactor::bm)

// Factor of one matrix (slab matrix of a time level, or K_n of a space level).
// T = memory type of right-hand sides and pivots: double (real symmetric), double2
// (complex symmetric, x = re, y = im), or float / float2 (mixed precision);
// WT = memory type of the blocks W: T, or FP32 (hi, lo) pairs for the double-float
// path (float2 real, float4 complex).
template <typename T, typename WT = T>
struct DevFactor {
  int32_t n = 0, nnodes = 0, max_depth = 0;
  DevNode* nodes = nullptr;
  WT* W = nullptr;                // per-node blocks W_s = [L11^-1; -L21 L11^-1], row-major
  T* Dinv = nullptr;              // [n], permuted order
  int32_t* rows = nullptr;        // struct(s) lists, permuted indices
  int32_t* gsrc = nullptr;        // forward gather table, 2 per front position
  int32_t* iperm = nullptr;       // original index -> permuted position
  // per depth d: tiles [tile_off[d], tile_off[d+1]) as (node, row tile)
  int2* fwd_tiles = nullptr;
  int2* bwd_tiles = nullptr;
  int32_t bm = kSnBM;             // rows per tile of fwd_tiles / bwd_tiles
  int64_t* h_fwd_off = nullptr;   // host arrays, size max_depth + 2
  int64_t* h_bwd_off = nullptr;
  int64_t u_rows = 0;
  double macs_per_rhs = 0;        // complex/real multiply-adds of one solve per right-hand side
  // split-K path for few right-hand sides: per depth, work items (node, row0, k0, k1)
  // of kSkRows rows and units (node, row0, item_begin, item_end) that reduce them
  int4* fs_items = nullptr;
  int4* fs_units = nullptr;
  int4* bs_items = nullptr;
  int4* bs_units = nullptr;
  const int64_t* d_fs_item_off = nullptr;   // the four offset arrays below, on the device
  const int64_t* d_fs_unit_off = nullptr;   // (persistent split-K solve)
  const int64_t* d_bs_item_off = nullptr;
  const int64_t* d_bs_unit_off = nullptr;
  int64_t* h_fs_item_off = nullptr;   // host, size max_depth + 2
  int64_t* h_fs_unit_off = nullptr;
  int64_t* h_bs_item_off = nullptr;
  int64_t* h_bs_unit_off = nullptr;
  int64_t max_items = 0;              // largest item count of one depth (partial buffer rows / kSkRows)
  // dataflow split-K solve: tasks (0, item) / (1, unit) in topological order per sweep,
  // the unit of every item, units per node, and per node the nodes it waits for
  // (forward: children; backward: (parent, -1))
  int2* df_tasks_f = nullptr;
  int2* df_tasks_b = nullptr;
  int32_t* df_item_unit_f = nullptr;
  int32_t* df_item_unit_b = nullptr;
  int32_t* df_node_units_f = nullptr;
  int32_t* df_node_units_b = nullptr;
  int2* df_children = nullptr;
  int2* df_parent = nullptr;
  int64_t n_df_tasks_f = 0, n_df_tasks_b = 0;
  int64_t n_fs_items = 0, n_bs_items = 0, n_fs_units = 0, n_bs_units = 0;   // totals over all depths
  int32_t n_sm = 152;                 // multiprocessors of the device (wave size of the tiled path)
  // tensor-core split-K: per depth, items (node, row tile, k0, k1) of kTcSplitK complex
  // columns and units (node, row tile, item_begin, item_end)
  int4* tcf_items = nullptr;
  int4* tcf_units = nullptr;
  int4* tcb_items = nullptr;
  int4* tcb_units = nullptr;
  int64_t* h_tcf_item_off = nullptr;
  int64_t* h_tcf_unit_off = nullptr;
  int64_t* h_tcb_item_off = nullptr;
  int64_t* h_tcb_unit_off = nullptr;
  int64_t max_tc_items = 0;
  // pipelined tensor-core path: the factor blocks pre-laid-out as 16 KiB tiles in the
  // shared-memory operand format (forward and transposed), per-node tile metadata and,
  // per depth, the (node, k stage) list of right-hand-side tiles to assemble
  uint8_t* tw_f = nullptr;            // forward A tiles
  uint8_t* tw_b = nullptr;            // backward A tiles
  int4* tnode = nullptr;              // per node: (fwd tile base, fwd k stages, bwd tile base, bwd k stages)
  int2* tpre = nullptr;               // per node: prefix of k stages over its depth (fwd, bwd)
  int2* tas_f = nullptr;              // per depth: (node, k stage) pairs
  int2* tas_b = nullptr;
  int64_t* h_tas_f_off = nullptr;
  int64_t* h_tas_b_off = nullptr;
  int64_t max_stage_tiles = 0;        // largest per-depth sum of k stages (fwd or bwd)
};
constexpr int kTcTileBytes = 16384;   // one operand tile: 128 real rows x 64 real K of BF16
constexpr int kTcSplitK = 256;      // complex K columns per tensor-core split-K item

// Split-K path: rows per item, columns per item, and the largest right-hand-side
// count it serves (complex: kSkMaxRhsC, real: kSkMaxRhsR).
constexpr int kSkRows = 32;
constexpr int kSkK = 32;     // default K columns per item (st_mg_options.split_k)
constexpr int kSkMaxRhsC = 16;
constexpr int kSkMaxRhsR = 32;

// Number of kernels launched by this library since load (all launchers add to it).
int64_t launch_count();
void count_launches(int64_t n);
// Programmatic dependent launch of the library's kernels (process-wide, default off: it
// measured slower on GB300): a kernel may be scheduled while the previous one on its
// stream drains (launch.cuh).
bool launch_overlap();
void set_launch_overlap(bool on);


// ---- supernodal solve: X = A^{-1} Q on `nrhs` columns, leading dimension ld.
// Q (in) is overwritten by X (out); Z and U are workspaces ([n*ld], [u_rows*ld]).
// P is the split-K partial buffer: max_items * kSkRows * (max right-hand sides per
// solve, rounded up to the column block) elements.  Null disables the split-K path.
// Per-handle solve state: grid-barrier words of the persistent split-K solve
// (arrivals, generation; zero at allocation; bar == nullptr disables the persistent
// launch), the flag a bounded wait sets, and the tiled/split-K threshold.
struct SkSync {
  unsigned* bar = nullptr;
  int* err = nullptr;
  int split_waves = 2;   // a tree depth runs split-K when its tiles fill fewer than this many
                         // waves of the SMs (setup may tune it per level)
  unsigned* df = nullptr;    // dataflow split-K solve: counter words (null: per-depth launches)
  bool tc_persist = false;   // tiled tensor-core depths: one persistent CTA per SM walking the
                            // depth's tiles (true) or one CTA per tile (false)
};

cudaError_t sn_solve_real(const DevFactor<double>& F, double* Q, double* Z, double* U, double* P, int nrhs, int ld,
                          const SkSync& sy, cudaStream_t st);
cudaError_t sn_solve_cplx(const DevFactor<double2>& F, double2* Q, double2* Z, double2* U, double2* P, int nrhs,
                          int ld, const SkSync& sy, cudaStream_t st);

// Mixed precision: the same solve with the factor and the right-hand sides in FP32
// (factor computed in FP64 and rounded once at setup).
cudaError_t sn_solve_realf(const DevFactor<float>& F, float* Q, float* Z, float* U, float* P, int nrhs, int ld,
                           const SkSync& sy, cudaStream_t st);
cudaError_t sn_solve_cplxf(const DevFactor<float2>& F, float2* Q, float2* Z, float2* U, float2* P, int nrhs, int ld,
                           const SkSync& sy, cudaStream_t st);

// BF16 factor on the tensor cores (DG(1)): W as complex BF16, right-hand sides and
// accumulation in FP32.  Depths with enough tiles run the tcgen05 kernels on tasks of 64
// complex rows x kTcCols right-hand sides (sy.tc_persist: one persistent CTA per SM
// walking the depth's tasks, else one CTA per task), the others split K into chunks
// (Ptc: max_tc_items * ceil(nrhs / kTcCols) * kSnBM * kTcCols float2); small nrhs takes
// the CUDA-core split-K path.  sy.err: set to 1 if a bounded wait timed out.
constexpr int kTcCols = 128;
cudaError_t sn_solve_cplx_bf16(const DevFactor<float2, __nv_bfloat162>& F, float2* Q, float2* Z, float2* U,
                               float2* P, float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy,
                               cudaStream_t st);
// The same BF16 factor applied on the CUDA cores with the tensor-core kernels'
// operand rounding (right-hand sides rounded to BF16 as they enter each product, FP32
// accumulation), tiled at every depth: the element-wise reference of those kernels.
cudaError_t sn_solve_cplx_bf16_cc(const DevFactor<float2, __nv_bfloat162>& F, float2* Q, float2* Z, float2* U,
                                  int nrhs, int ld, cudaStream_t st);
// FP16 factor on the tensor cores (slab_prec 4): the same kernels with FP16 operands.
// FP16 keeps 3 more significant bits than BF16 but only 5 exponent bits, so the
// caller scales every right-hand-side column by a power of two first (col_scale).
cudaError_t sn_solve_cplx_f16(const DevFactor<float2, __half2>& F, float2* Q, float2* Z, float2* U, float2* P,
                              float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy, cudaStream_t st);
cudaError_t sn_solve_cplx_f16_cc(const DevFactor<float2, __half2>& F, float2* Q, float2* Z, float2* U, int nrhs,
                                 int ld, cudaStream_t st);
// Pipelined tensor-core depth: assemble the right-hand-side tiles of the depth into
// Bst (gy * max_stage_tiles tiles), then the products with bulk-copied operand tiles.
// WT = __nv_bfloat162 (BF16 operands) or __half2 (FP16 operands).
template <typename WT>
cudaError_t sn_tc2_depth(const DevFactor<float2, WT>& F, int d, bool fwd, bool split, float2* Q, float2* Z,
                         float2* U, float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy, cudaStream_t st);
// Per-column power-of-two scaling of cnt complex columns of Q (rows x ld): colmax
// (ld unsigned, the bits of max(|re|, |im|) per column) is cleared and filled, then
// every column is multiplied by s_j = 2^(1 - e_j), e_j the binary exponent of its
// maximum, so that its largest entry lies in [1, 2) (s_j = 1 for a zero column);
// col_unscale divides by the same s_j (exact: powers of two).
cudaError_t col_scale(float2* Q, int nrows, int cnt, int ld, unsigned* colmax, cudaStream_t st);
cudaError_t col_unscale(float2* Q, int nrows, int cnt, int ld, const unsigned* colmax, cudaStream_t st);

// FP64-accurate double-float path (W as FP32 pairs, FP64 right-hand sides).
cudaError_t sn_solve_real_df(const DevFactor<double, float2>& F, double* Q, double* Z, double* U, double* P, int nrhs,
                             int ld, const SkSync& sy, cudaStream_t st);
cudaError_t sn_solve_cplx_df(const DevFactor<double2, float4>& F, double2* Q, double2* Z, double2* U, double2* P,
                             int nrhs, int ld, const SkSync& sy, cudaStream_t st);

// ---- space-time kernels.  Edge-major layout v[e*ncols + n*q + i], ncols = N_t*q.
struct CsrView {
  int32_t nrows;
  const int64_t* rowptr;
  const int32_t* col;
};

// r = f - L x.  DG(0): a = M + tau K, m = M.  DG(1): m = M, k0 = tau K, k1 = tau K / 3.
// partial (nullable): one double per block with the block's sum of r^2 (deterministic
// second stage by reduce_partials).  Returns the number of blocks via *nblocks.
// N_t = slab columns of the call (all problems of a batch), seg = slabs per problem:
// the history coupling is cut where a new problem starts (slab index % seg == 0).
cudaError_t residual_dg0(CsrView A, const double* a, const double* m, const double* f, const double* x,
                         double* r, int N_t, int seg, double* partial, int* nblocks, cudaStream_t st);
cudaError_t residual_dg1(CsrView A, const double* m, const double* k0, const double* k1, const double* f,
                         const double* x, double* r, int N_t, int seg, double* partial, int* nblocks, cudaStream_t st);
int residual_blocks(int nrows);
// Double-float residual (FP64-accurate on the FP32 pipes): xs = x split into (hi, lo)
// FP32 pairs by split_pairs, coefficient arrays as pairs; f, r and norms in FP64.
cudaError_t split_pairs(const double* x, float2* xs, int64_t n, cudaStream_t st);
cudaError_t residual_dg0_df(CsrView A, const float2* a, const float2* m, const double* f, const float2* xs, double* r,
                            int N_t, int seg, double* partial, int* nblocks, cudaStream_t st);
cudaError_t residual_dg1_df(CsrView A, const float2* m, const float2* k0, const float2* k1, const double* f,
                            const float2* xs, double* r, int N_t, int seg, double* partial, int* nblocks, cudaStream_t st);
// FP32 residual (the correction-form V-cycle of residual_prec 1): x as FP32 (to_float),
// FP32 coefficients and sums, f and r in FP64.
cudaError_t to_float(const double* x, float* xf, int64_t n, cudaStream_t st);
cudaError_t residual_dg0_f32(CsrView A, const float* a, const float* m, const double* f, const float* xf, double* r,
                             int N_t, int seg, double* partial, int* nblocks, cudaStream_t st);
cudaError_t residual_dg1_f32(CsrView A, const float* m, const float* k0, const float* k1, const double* f,
                             const float* xf, double* r, int N_t, int seg, double* partial, int* nblocks,
                             cudaStream_t st);
// b += a
cudaError_t vec_add(const double* a, double* b, int64_t n, cudaStream_t st);
// out[0] = sum of partial[0..n) in a fixed order.
cudaError_t reduce_partials(const double* partial, int n, double* out, cudaStream_t st);
// out[0] = sum v^2 over n values (deterministic two-stage); partial has >= 1024 entries.
cudaError_t norm2_sq(const double* v, int64_t n, double* partial, double* out, cudaStream_t st);

// Slab right-hand sides -> permuted solve columns (slabs slab0 .. slab0+cnt-1 of a
// source with row length src_ld).  DG(1) maps the pair (r0, r1) to c0 r0 + c1 r1.
cudaError_t slab_pre_dg0(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                         double* Q, int ld, cudaStream_t st);
cudaError_t slab_pre_dg1(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                         double2 c0, double2 c1, double2* Q, int ld, cudaStream_t st);
// Solution columns -> slabs.  mode 0: x = v;  mode 1: x += omega * v.
// DG(1): u_i = 2 Re(s_i v) with s = (1, s1).
cudaError_t slab_post_dg0(const double* X, int ld, const int32_t* iperm, int nrows, double* x, int dst_ld,
                          int slab0, int cnt, double omega, int mode, cudaStream_t st);
cudaError_t slab_post_dg1(const double2* X, int ld, const int32_t* iperm, int nrows, double2 s1, double* x,
                          int dst_ld, int slab0, int cnt, double omega, int mode, cudaStream_t st);
// FP32 variants for the mixed-precision slab solve (FP64 in, FP32 solve, FP64 out).
cudaError_t slab_pre_dg0f(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                          float* Q, int ld, cudaStream_t st);
cudaError_t slab_pre_dg1f(const double* r, int src_ld, int slab0, int cnt, const int32_t* iperm, int nrows,
                          double2 c0, double2 c1, float2* Q, int ld, cudaStream_t st);
cudaError_t slab_post_dg0f(const float* X, int ld, const int32_t* iperm, int nrows, double* x, int dst_ld,
                           int slab0, int cnt, double omega, int mode, cudaStream_t st);
cudaError_t slab_post_dg1f(const float2* X, int ld, const int32_t* iperm, int nrows, double2 s1, double* x,
                           int dst_ld, int slab0, int cnt, double omega, int mode, cudaStream_t st);
// Nodal solve columns: Q[iperm[v]][j] = y[v][j];  z[v][j] = X[iperm[v]][j].
cudaError_t gather_perm(const double* y, int ncols, const int32_t* iperm, int nrows, double* Q, int ld,
                        cudaStream_t st);
cudaError_t scatter_perm(const double* X, int ld, const int32_t* iperm, int nrows, double* z, int ncols,
                         cudaStream_t st);
// the same with an FP32 workspace (FP32 nodal solve)
cudaError_t gather_perm_f(const double* y, int ncols, const int32_t* iperm, int nrows, float* Q, int ld,
                          cudaStream_t st);
cudaError_t scatter_perm_f(const float* X, int ld, const int32_t* iperm, int nrows, double* z, int ncols,
                           cudaStream_t st);

// y[v][j] = sum over incident interior edges of G[e][v] r[e][j]  (G^T, node-major CSR,
// gt_sign = +1 head / -1 tail).
cudaError_t grad_T(CsrView GT, const int8_t* gt_sign, const double* r, double* y, int ncols, cudaStream_t st);
// x[e][j] += w[head][j] - w[tail][j]  (G w), -1 = boundary vertex.
cudaError_t grad_add(const int32_t* tail, const int32_t* head, int nedges, const double* w, double* x,
                     int ncols, cudaStream_t st);
// w = L_t^{-1} z per node row (DG(0): running sum; DG(1): upwind recurrence).
cudaError_t time_integrate(const double* z, double* w, int nrows, int N_t, int degree, cudaStream_t st);
// Time-slab sharding: the scan continued from w_{-1} = carry (q values per node row);
// one slab of every row, out[row q + i] = v[row ld + off + i]; the history term of a
// range's first slab, r_0 -= (N_t (x) M) xh; the carry into range n_prev from the end
// states ends[k][row q + i] of the ranges before it.
cudaError_t time_integrate_carry(const double* z, const double* carry, double* w, int nrows, int N_t, int degree,
                                 cudaStream_t st);
cudaError_t slab_copy(const double* v, int64_t ld, int64_t off, int q, int nrows, double* out, cudaStream_t st);
cudaError_t halo_history(CsrView A, const double* m, const double* xh, double* r, int64_t ld, int degree,
                         cudaStream_t st);
cudaError_t time_carry(const double* ends, int n_prev, int nrows, int degree, double* carry, cudaStream_t st);
// One damped Jacobi sweep on K_n: zo = zi + wgt * D^{-1} (y - K_n zi).
cudaError_t nodal_jacobi(CsrView Kn, const double* kval, const double* dinv, const double* y, const double* zi,
                         double* zo, int ncols, double wgt, cudaStream_t st);

// Time transfers between N_t (fine) and N_t/2 (coarse) slabs, same space level; nrows =
// edges x Bf rows of one problem each, the coarse level has Bc >= Bf problems per edge row
// (a ragged batch; Bf = Bc = 1 by default: contiguous rows).
cudaError_t time_restrict(const double* r, double* rc, int nrows, int Nc, int degree, cudaStream_t st, int Bf = 1,
                          int Bc = 1);
cudaError_t time_prolong_add(const double* ec, double* x, int nrows, int Nc, int degree, cudaStream_t st, int Bf = 1,
                             int Bc = 1);
// Space transfers per time column: out = P in (P given as CSR rows), beta 0 overwrite / 1 add.
cudaError_t csr_spmm(CsrView P, const double* pval, const double* in, double* out, int ncols, int beta,
                     cudaStream_t st);
// Coarse forward substitution: g[e][i] = f[e][n q + i] - sum_j N_t[i][j] (M x_{n-1})_j.
cudaError_t history_rhs(CsrView A, const double* m, const double* f, const double* x, double* g, int N_t,
                        int n, int degree, cudaStream_t st);
// Per-problem sums of squares of a batched finest-level vector (v[e][b * seg + j]);
// partial: batch_norm_scratch(nb) doubles; out: nb doubles (device).
int batch_norm_scratch(int nb);
cudaError_t batch_norms_sq(const double* v, int nrows, int nb, int seg, double* partial, double* out,
                           cudaStream_t st);
// Zero columns [offset, offset + count) of every row (row length stride).
cudaError_t zero_cols(double* v, int nrows, int stride, int offset, int count, cudaStream_t st);
// FP64 FMA throughput probe: blocks x 256 threads x iters x 8 FMAs (out: >= blocks doubles).
cudaError_t fp64_probe(double* out, int blocks, int iters, cudaStream_t st);
// Elementwise helpers.
cudaError_t vec_fill(double* v, int64_t n, double value, cudaStream_t st);
cudaError_t vec_copy(const double* a, double* b, int64_t n, cudaStream_t st);
// Outer-product load f[e * row_stride + j] = c[j] * b[e], j < ncols.
cudaError_t outer_load(const double* b, const double* c, double* f, int nrows, int ncols, int row_stride,
                       cudaStream_t st);

}  // namespace stmg
