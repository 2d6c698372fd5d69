// Tensor-core (tcgen05) supernodal products for the BF16 slab solve of DG(1):
// the dense contraction of the method (the slab inverse applied to all slabs,
// eq. StandardSmoother) on the 5th-generation tensor cores, BF16 operands and
// FP32 accumulators in tensor memory.
//
// A block computes 64 complex rows x 128 right-hand sides of one supernode's
// product.  Complex arithmetic is real-ified: each complex factor entry
// w = a + ib becomes the 2x2 block [[a, -b], [b, a]] of a 128 x 2K real tile, and
// each complex right-hand side entry g becomes the pair (Re g, Im g) along K, so
// row 2i of the FP32 accumulator holds Re y_i and row 2i+1 holds Im y_i.
// Operands live in the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes
// per core matrix; 128 bytes between K-adjacent cores, 1024 bytes between 8-row
// groups): the factor tiles are laid out so at setup, the right-hand-side tiles by
// k_tc_assemble once per tree depth.  k_sn_tc2 moves (factor, right-hand side) tile
// pairs into a 3-stage shared-memory ring with cp.async.bulk, one thread issues
// tcgen05.mma kind::f16 (M = 128, N = 128, K = 16 per instruction) and frees each
// stage with tcgen05.commit.  Every wait is bounded: on timeout the block records an
// error in *err, waits (bounded) for its copies and MMAs in flight and skips its
// epilogue.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "device.h"
#include "launch.cuh"

namespace stmg {
namespace {

constexpr int TC_ROWS = kSnBM;            // complex rows per block (128 real MMA rows)
constexpr int TC_M = 2 * TC_ROWS;         // 128
constexpr int TC_N = kTcCols;             // right-hand sides per block (MMA N)
constexpr int TC_KC = 32;                 // complex K per stage (64 real = 4 MMAs of K = 16)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = TC_N;   // FP32 accumulator columns
constexpr uint32_t CORE_K = 128;          // bytes between K-adjacent core matrices
constexpr uint32_t CORE_MN = 1024;        // bytes between 8-row groups (8 cores along K)
constexpr int WAIT_LIMIT = 1 << 20;       // try_wait rounds before a wait gives up (well under a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major tile
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)(row >> 3) * CORE_MN + (uint32_t)(k >> 3) * CORE_K + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// shared-memory matrix descriptor: start >> 4, leading (K) byte offset >> 4,
// stride (8-row group) byte offset >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(CORE_K >> 4) << 16;
  d |= (uint64_t)(CORE_MN >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B both BF16
// (bits 7-9 and 10-12 = 1) or both FP16 (0), both K-major, N >> 3 and M >> 4
template <bool F16>
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (F16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(TC_N >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < WAIT_LIMIT; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(TC_TMEM_COLS));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// complex K rows k (even) and k + 1 of column c: four adjacent 16-bit values, one 8-byte store
template <bool F16>
__device__ __forceinline__ void put_g2(uint8_t* Bs, int c, int k, float2 g0, float2 g1) {
  uint2 w;
  if (F16) {
    const __half2 a = __floats2half2_rn(g0.x, g0.y), b = __floats2half2_rn(g1.x, g1.y);
    w = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  } else {
    const __nv_bfloat162 a = __floats2bfloat162_rn(g0.x, g0.y), b = __floats2bfloat162_rn(g1.x, g1.y);
    w = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
  *reinterpret_cast<uint2*>(Bs + core_off(c, 2 * k)) = w;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// one rounded product and one fused multiply-add per part, spelled out so that every
// kernel here rounds the same way (left to the compiler, the contraction may differ
// between kernels)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// One block per (unit = node row tile, column tile, group of TC_RED_ROWS rows): sums
// the unit's K-chunk partials in item order, then the forward or backward epilogue.
constexpr int TC_RED_ROWS = 8;
template <bool FWD>
__global__ void __launch_bounds__(256) k_sn_tc_reduce(const DevNode* __restrict__ nodes,
                                                      const float2* __restrict__ Dinv,
                                                      const int32_t* __restrict__ gsrc,
                                                      const int4* __restrict__ units, int64_t item_base,
                                                      int64_t n_items, const float2* __restrict__ P,
                                                      float2* __restrict__ Z, float2* __restrict__ U,
                                                      float2* __restrict__ X, int nrhs, int ld) {
  pdl_entry();
  const int4 un = units[blockIdx.x];
  const DevNode nd = nodes[un.x];
  const int nc = nd.nc, m = nd.nc + nd.nr;
  const int row0 = un.y * TC_ROWS, c0 = blockIdx.y * TC_N;
  const int rows_out = FWD ? m : nc;
  // block z: rows TC_RED_ROWS z .. TC_RED_ROWS (z + 1) - 1 of the unit's row tile
  for (int t = threadIdx.x; t < TC_RED_ROWS * TC_N; t += blockDim.x) {
    const int il = blockIdx.z * TC_RED_ROWS + t / TC_N, cl = t % TC_N;
    const int i = row0 + il, c = c0 + cl;
    if (i >= rows_out || c >= nrhs) continue;
    float2 y = make_float2(0.f, 0.f);
    for (int q = un.z; q < un.w; ++q)
      y = cadd(y, P[(((int64_t)blockIdx.y * n_items + (q - item_base)) * TC_ROWS + il) * TC_N + cl]);
    if (FWD) {
      if (i < nc) {
        Z[(int64_t)(nd.col0 + i) * ld + c] = cmul(Dinv[nd.col0 + i], y);
      } else {
        const int32_t* gs = gsrc + nd.g_off * 2;
        const int s0 = gs[2 * i], s1 = gs[2 * i + 1];
        if (s0 >= 0) y = cadd(y, U[(int64_t)s0 * ld + c]);
        if (s1 >= 0) y = cadd(y, U[(int64_t)s1 * ld + c]);
        U[(int64_t)(nd.u_off + i - nc) * ld + c] = y;
      }
    } else {
      X[(int64_t)(nd.col0 + i) * ld + c] = y;
    }
  }
}

// ---------------------------------------------------------------- pipelined path
// The factor's operand tiles are stored in global memory already in the shared-memory
// layout above (16 KiB per 64 complex rows x 32 complex K), so a stage is two 16 KiB
// cp.async.bulk copies (factor tile and right-hand-side tile) completing on an
// mbarrier; TC2_STAGES stages are in flight.  Thread 0 produces (bulk copies),
// thread 32 issues the MMAs and frees a stage by tcgen05.commit on its "empty"
// barrier; all four warps run the epilogue.

constexpr int TC2_STAGES = 3;
constexpr int TC2_SMEM = TC2_STAGES * 2 * kTcTileBytes + 1024;   // + alignment slack
constexpr int TC2_OS = 2 * TC_N + 2;   // floats per staged output row (epilogue)
static_assert(TC_ROWS * TC2_OS * 4 <= TC2_STAGES * 2 * kTcTileBytes, "epilogue tile must fit the stage buffers");
static_assert(TC_THREADS == TC_N, "epilogue maps one column per thread");

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes));
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Right-hand-side tiles of one depth: item (node, k stage) x column tile ->
// tile gy * pre(node) + ct * kstages(node) + ks of Bst, the (Re, Im) pairs of the
// gathered right-hand side (forward: Q + children's update rows; backward: z of the
// node's columns, x of its below-structure rows) rounded to BF16 in operand layout.
template <bool FWD, bool F16>
__global__ void __launch_bounds__(256) k_tc_assemble(const DevNode* __restrict__ nodes,
                                                     const int32_t* __restrict__ gsrc,
                                                     const int32_t* __restrict__ rows,
                                                     const int4* __restrict__ tnode, const int2* __restrict__ tpre,
                                                     const int2* __restrict__ items, const float2* __restrict__ Q,
                                                     const float2* __restrict__ Z, const float2* __restrict__ U,
                                                     const float2* __restrict__ X, uint8_t* __restrict__ Bst, int nrhs,
                                                     int ld) {
  pdl_entry();
  const int2 it = items[blockIdx.x];
  const int s = it.x, ks = it.y, ct = blockIdx.y, gy = gridDim.y;
  const DevNode nd = nodes[s];
  const int nc = nd.nc, m = nc + nd.nr;
  const int4 tn = tnode[s];
  const int nks = FWD ? tn.y : tn.w;
  const int pre = FWD ? tpre[s].x : tpre[s].y;
  __shared__ __align__(16) uint8_t tile[kTcTileBytes];
  uint8_t* out = Bst + ((int64_t)gy * pre + (int64_t)ct * nks + ks) * kTcTileBytes;
  const int32_t* gs = gsrc + nd.g_off * 2;
  const int32_t* rw = rows + nd.row_off;
  const int kend = FWD ? nc : m;
  // thread: column cl, rows kk = 4 j + 2 kp + h (kp = thread / TC_N, h = 0, 1), eight rows
  // per batch.  A batch first loads the rows' gather indices, then every value, then sums
  // (in the order Q + U_s0 + U_s1), so a block waits for a few memory round trips
  // instead of two per row
  const int cl = threadIdx.x % TC_N, kp = threadIdx.x / TC_N;
  const int c = ct * TC_N + cl;
  const bool col_ok = c < nrhs;
  constexpr int RB = 8;   // rows per batch
  static_assert(TC_KC == 2 * 2 * RB, "two batches of eight rows per thread");
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    int s0[RB], s1[RB];
    bool ok[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int kk = 4 * (b * (RB / 2) + r / 2) + 2 * kp + (r & 1);
      const int k = ks * TC_KC + kk;
      ok[r] = col_ok && k < kend;
      s0[r] = s1[r] = -1;
      if (FWD) {
        if (ok[r]) {
          s0[r] = gs[2 * k];
          s1[r] = gs[2 * k + 1];
        }
      } else if (ok[r] && k >= nc) {
        s0[r] = rw[k - nc];
      }
    }
    float2 v[RB], u0[RB], u1[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int kk = 4 * (b * (RB / 2) + r / 2) + 2 * kp + (r & 1);
      const int k = ks * TC_KC + kk;
      v[r] = u0[r] = u1[r] = make_float2(0.f, 0.f);
      if (FWD) {
        if (ok[r]) v[r] = Q[(int64_t)(nd.col0 + k) * ld + c];
        if (s0[r] >= 0) u0[r] = U[(int64_t)s0[r] * ld + c];
        if (s1[r] >= 0) u1[r] = U[(int64_t)s1[r] * ld + c];
      } else if (ok[r]) {
        v[r] = (k < nc) ? Z[(int64_t)(nd.col0 + k) * ld + c] : X[(int64_t)s0[r] * ld + c];
      }
    }
#pragma unroll
    for (int r = 0; r < RB; r += 2) {
      const int kk = 4 * (b * (RB / 2) + r / 2) + 2 * kp;
      float2 g0 = v[r], g1 = v[r + 1];
      if (FWD) {
        if (s0[r] >= 0) g0 = cadd(g0, u0[r]);
        if (s1[r] >= 0) g0 = cadd(g0, u1[r]);
        if (s0[r + 1] >= 0) g1 = cadd(g1, u0[r + 1]);
        if (s1[r + 1] >= 0) g1 = cadd(g1, u1[r + 1]);
      }
      put_g2<F16>(tile, cl, kk, g0, g1);
    }
  }
  __syncthreads();
  // the finished tile leaves in 16-byte pieces, consecutive threads consecutive pieces
  const uint4* src = reinterpret_cast<const uint4*>(tile);
  uint4* dst = reinterpret_cast<uint4*>(out);
  for (int t = threadIdx.x; t < kTcTileBytes / 16; t += blockDim.x) dst[t] = src[t];
}

// SPLIT = false: grid over (node, row tile) tiles, whole K range; SPLIT = true: grid
// over (node, row tile, k0, k1) items (k0, k1 multiples of 32 complex), partial
// products to P for k_sn_tc_reduce.
template <bool FWD, bool SPLIT, bool F16>
__global__ void __launch_bounds__(TC_THREADS) k_sn_tc2(const DevNode* __restrict__ nodes,
                                                       const uint8_t* __restrict__ TW,
                                                       const int4* __restrict__ tnode, const int2* __restrict__ tpre,
                                                       const uint8_t* __restrict__ Bst,
                                                       const float2* __restrict__ Dinv,
                                                       const int32_t* __restrict__ gsrc,
                                                       const int2* __restrict__ tiles, const int4* __restrict__ items,
                                                       float2* __restrict__ Z, float2* __restrict__ U,
                                                       float2* __restrict__ X, float2* __restrict__ P, int nrhs, int ld,
                                                       int* __restrict__ err) {
  pdl_entry();
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full[TC2_STAGES], empty[TC2_STAGES], done;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  int node, rtile, ik0 = 0, ik1 = 0;
  if (SPLIT) {
    const int4 it = items[blockIdx.x];
    node = it.x; rtile = it.y; ik0 = it.z; ik1 = it.w;
  } else {
    const int2 tl = tiles[blockIdx.x];
    node = tl.x; rtile = tl.y;
  }
  const DevNode nd = nodes[node];
  const int nc = nd.nc, m = nc + nd.nr;
  const int row0 = rtile * TC_ROWS, c0 = blockIdx.y * TC_N, ct = blockIdx.y, gy = gridDim.y;
  const int4 tn = tnode[node];
  const int nks = FWD ? tn.y : tn.w;
  const int pre = FWD ? tpre[node].x : tpre[node].y;
  const uint8_t* atiles = TW + ((int64_t)(FWD ? tn.x : tn.z) + (int64_t)rtile * nks) * kTcTileBytes;
  const uint8_t* btiles = Bst + ((int64_t)gy * pre + (int64_t)ct * nks) * kTcTileBytes;
  // k stages: forward rows inside L11^{-1} stop at the tile's last row; backward
  // rows start at the first nonzero of L11^{-1} (stage 2 rtile)
  int ks0, ks1;
  if (SPLIT) {
    ks0 = ik0 / TC_KC;
    ks1 = (ik1 + TC_KC - 1) / TC_KC;
  } else if (FWD) {
    ks0 = 0;
    ks1 = ((row0 + TC_ROWS <= nc ? row0 + TC_ROWS : nc) + TC_KC - 1) / TC_KC;
  } else {
    ks0 = row0 / TC_KC;
    ks1 = nks;
  }
  if (tid == 0) {
    for (int i = 0; i < TC2_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncwarp();
  if (warp == 0) tmem_alloc(&tmem_slot);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const int nst = ks1 - ks0;
  bool ok = true;
  int issued = 0;   // stages whose bulk copies thread 0 has started
  if (tid == 0) {
    // producer: stage i waits until the MMAs that used its buffers have completed
    for (int i = 0; i < nst && ok; ++i) {
      const int slot = i % TC2_STAGES;
      const uint32_t ph = (uint32_t)((i / TC2_STAGES) & 1);
      if (!mbar_wait(&empty[slot], ph ^ 1u)) { ok = false; break; }
      uint8_t* a = base + slot * 2 * kTcTileBytes;
      mbar_arrive_tx(&full[slot], 2 * kTcTileBytes);
      bulk_g2s(smem_u32(a), atiles + (int64_t)(ks0 + i) * kTcTileBytes, kTcTileBytes, &full[slot]);
      bulk_g2s(smem_u32(a + kTcTileBytes), btiles + (int64_t)(ks0 + i) * kTcTileBytes, kTcTileBytes, &full[slot]);
      issued = i + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int i = 0; i < nst && ok; ++i) {
      const int slot = i % TC2_STAGES;
      const uint32_t ph = (uint32_t)((i / TC2_STAGES) & 1);
      if (!mbar_wait(&full[slot], ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint8_t* a = base + slot * 2 * kTcTileBytes;
#pragma unroll
      for (int s4 = 0; s4 < (2 * TC_KC) / 16; ++s4) {
        const uint64_t ad = smem_desc(smem_u32(a) + s4 * 2 * CORE_K);
        const uint64_t bd = smem_desc(smem_u32(a + kTcTileBytes) + s4 * 2 * CORE_K);
        const uint32_t acc = (i == 0 && s4 == 0) ? 0u : 1u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(tc_idesc<F16>()), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty[slot])));
    }
    // also after a failed wait: `done` then tracks the MMAs already issued, so that
    // no thread frees TMEM or leaves while they run
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&done)));
  }
  // everyone waits for the last MMA; the result is used only if no wait failed
  if (!ok) atomicExch(err, 1);
  const bool mine = (nst > 0) && mbar_wait(&done, 0);
  const bool fin = __syncthreads_and(mine && ok) != 0;   // block-uniform: the TMEM loads are warp-collective
  if (!fin && nst > 0 && tid == 0) {
    atomicExch(err, 1);
    // bulk copies still in flight land in this block's shared memory: wait for them
    // (bounded) before the block can exit
    for (int i = issued > TC2_STAGES ? issued - TC2_STAGES : 0; i < issued; ++i)
      mbar_wait(&full[i % TC2_STAGES], (uint32_t)((i / TC2_STAGES) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (fin) {
    // accumulator -> shared memory (the pipeline buffers are idle now): complex row
    // il = R / 2 (R = TMEM lane), real part from even lanes, imaginary from odd ones;
    // rows padded to 2 * TC_N + 2 floats so that a warp's 32 lanes hit 32 banks
    float* Os = reinterpret_cast<float*>(base);
    const int R = warp * 32 + lane;
    for (int cb = 0; cb < TC_N; cb += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) Os[(R >> 1) * TC2_OS + 2 * (cb + j) + (R & 1)] = __uint_as_float(v[j]);
    }
  }
  __syncthreads();
  if (fin) {
    // one column per thread, row by row: coalesced stores and update-row reads
    const float* Os = reinterpret_cast<const float*>(base);
    const int rows_out = FWD ? m : nc;
    const int c = c0 + tid;
    const int32_t* gs = gsrc + nd.g_off * 2;
    for (int il = 0; il < TC_ROWS; ++il) {
      const int i = row0 + il;
      const float2 y = *reinterpret_cast<const float2*>(Os + il * TC2_OS + 2 * tid);
      if (SPLIT) {
        P[(((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * TC_ROWS + il) * TC_N + tid] = y;
        continue;
      }
      if (i >= rows_out || c >= nrhs) continue;
      if (FWD) {
        if (i < nc) {
          Z[(int64_t)(nd.col0 + i) * ld + c] = cmul(Dinv[nd.col0 + i], y);
        } else {
          float2 u = y;
          const int s0 = gs[2 * i], s1 = gs[2 * i + 1];
          if (s0 >= 0) u = cadd(u, U[(int64_t)s0 * ld + c]);
          if (s1 >= 0) u = cadd(u, U[(int64_t)s1 * ld + c]);
          U[(int64_t)(nd.u_off + i - nc) * ld + c] = u;
        }
      } else {
        X[(int64_t)(nd.col0 + i) * ld + c] = y;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem);
}

// ---------------------------------------------------------------- persistent tiled path
// One CTA per SM walks the depth's (row tile, column block) tasks t = blockIdx.x,
// blockIdx.x + gridDim.x, ... with three roles: warp 0 (lane 0) streams the operand tiles
// of all its tasks through a TC3_STAGES-deep ring of shared-memory stages, warp 1 (lane 0)
// issues the MMAs of a task into one of two TMEM accumulators (columns 0..127 or
// 128..255), and warps 2..9 read a finished accumulator from TMEM (warp w reads TMEM
// lanes 32 (w % 4) .., two warps per lane quarter splitting the columns), apply the
// epilogue and store, while the next task's MMAs run into the other accumulator.  The
// ring never drains between tasks, so a CTA's short K loops no longer pay the pipeline
// fill each.  Products and epilogue are those of k_sn_tc2 (same stage order, FP32
// accumulation, same complex multiply), so the results are the same bit for bit.
// Barriers: full/empty per stage (producer <-> MMA), accf/acce per accumulator (MMA <->
// epilogue); every wait is bounded; a role whose wait gives up sets *err and stops, the
// others then stop at their own bounded waits, and the CTA waits (bounded) for its MMAs
// and copies in flight before it frees TMEM.
constexpr int TC3_STAGES = 4;
constexpr int TC3_THREADS = 320;   // producer warp, MMA warp, eight epilogue warps
constexpr uint32_t TC3_TMEM_COLS = 2 * TC_N;

// A task's descriptor, computed once per kernel for each of the CTA's tasks (all threads
// together, before the roles start) and kept in shared memory, so that no role waits on
// a chain of dependent index loads between tasks.  Task t of a depth: tile t / gy (node,
// row tile), column block t % gy; K stages ks0 .. ks1 - 1 (forward: up to the tile's last
// row inside L11^{-1}; backward: from the tile's first row).
struct Tc3Task {
  int32_t ks0, ks1;   // K stages
  int32_t a0, b0;     // operand tile index of stage 0: factor (TW), right-hand side (Bst)
  int32_t col0, nc, m, row0, c0, pad;
  int64_t u_off, g_off;
};
constexpr int TC3_MAX_TASKS = 160;   // tasks per CTA (the host takes the per-tile kernel beyond)
constexpr int TC3_EPI_ROWS = 16;     // complex rows of an epilogue warp
constexpr int TC3_EPI_LD = 66;       // floats per staged row: 32 complex columns + 2 (conflict-free)
constexpr int TC3_SMEM = TC3_STAGES * 2 * kTcTileBytes + 1024 + TC3_MAX_TASKS * (int)sizeof(Tc3Task) +
                         8 * TC3_EPI_ROWS * TC3_EPI_LD * 4;

template <bool FWD, bool F16>
__global__ void __launch_bounds__(TC3_THREADS, 1) k_sn_tc3(const DevNode* __restrict__ nodes,
                                                           const uint8_t* __restrict__ TW,
                                                           const int4* __restrict__ tnode,
                                                           const int2* __restrict__ tpre,
                                                           const uint8_t* __restrict__ Bst,
                                                           const float2* __restrict__ Dinv,
                                                           const int32_t* __restrict__ gsrc,
                                                           const int2* __restrict__ tiles, int ntiles, int gy,
                                                           float2* __restrict__ Z, float2* __restrict__ U,
                                                           float2* __restrict__ X, int nrhs, int ld,
                                                           int* __restrict__ err) {
  // launched with programmatic stream serialisation: the prologue below (task descriptors
  // from the factor's static lists, barriers, TMEM) may overlap the end of the kernel
  // before (the depth's right-hand-side assembly); nothing written by a kernel is read
  // before griddepcontrol.wait
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full[TC3_STAGES], empty[TC3_STAGES], accf[2], acce[2], done;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  Tc3Task* task = reinterpret_cast<Tc3Task*>(base + TC3_STAGES * 2 * kTcTileBytes);
  const int ntasks = ntiles * gy;
  // this CTA's tasks: t = blockIdx.x + k gridDim.x, k < nmine (<= TC3_MAX_TASKS, host-checked)
  const int nmine = blockIdx.x < ntasks ? (ntasks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  for (int k = tid; k < nmine && k < TC3_MAX_TASKS; k += blockDim.x) {
    const int t = blockIdx.x + k * gridDim.x;
    const int2 tl = tiles[t / gy];
    const int ct = t % gy, node = tl.x, rtile = tl.y;
    const DevNode nd = nodes[node];
    const int4 tn = tnode[node];
    const int nks = FWD ? tn.y : tn.w;
    const int pre = FWD ? tpre[node].x : tpre[node].y;
    const int row0 = rtile * TC_ROWS;
    Tc3Task d;
    if (FWD) {
      d.ks0 = 0;
      d.ks1 = ((row0 + TC_ROWS <= nd.nc ? row0 + TC_ROWS : nd.nc) + TC_KC - 1) / TC_KC;
    } else {
      d.ks0 = row0 / TC_KC;
      d.ks1 = nks;
    }
    d.a0 = (FWD ? tn.x : tn.z) + rtile * nks;
    d.b0 = gy * pre + ct * nks;
    d.col0 = nd.col0;
    d.nc = nd.nc;
    d.m = nd.nc + nd.nr;
    d.row0 = row0;
    d.c0 = ct * TC_N;
    d.pad = 0;
    d.u_off = nd.u_off;
    d.g_off = nd.g_off;
    task[k] = d;
  }
  if (tid == 0) {
    for (int i = 0; i < TC3_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&acce[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TC3_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  pdl_entry();
  const uint32_t tmem = tmem_slot;
  const int ntask = nmine < TC3_MAX_TASKS ? nmine : TC3_MAX_TASKS;
  int issued = 0;   // producer: stages whose copies it started
  bool pfail = false;
  if (warp == 0 && lane == 0) {
    // ---- producer
    int g = 0;
    for (int k = 0; k < ntask && !pfail; ++k) {
      const Tc3Task& d = task[k];
      const uint8_t* atiles = TW + (int64_t)d.a0 * kTcTileBytes;
      const uint8_t* btiles = Bst + (int64_t)d.b0 * kTcTileBytes;
      for (int ks = d.ks0; ks < d.ks1; ++ks, ++g) {
        const int slot = g % TC3_STAGES;
        const uint32_t ph = (uint32_t)((g / TC3_STAGES) & 1);
        if (!mbar_wait(&empty[slot], ph ^ 1u)) { pfail = true; break; }
        uint8_t* a = base + slot * 2 * kTcTileBytes;
        mbar_arrive_tx(&full[slot], 2 * kTcTileBytes);
        bulk_g2s(smem_u32(a), atiles + (int64_t)ks * kTcTileBytes, kTcTileBytes, &full[slot]);
        bulk_g2s(smem_u32(a + kTcTileBytes), btiles + (int64_t)ks * kTcTileBytes, kTcTileBytes, &full[slot]);
        issued = g + 1;
      }
    }
    if (pfail) atomicExch(err, 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool fail = false;
    int g = 0;
    for (int k = 0; k < ntask && !fail; ++k) {
      const Tc3Task& d = task[k];
      const int abuf = k & 1;
      const uint32_t aph = (uint32_t)((k >> 1) & 1);
      if (!mbar_wait(&acce[abuf], aph ^ 1u)) { fail = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t acc_addr = tmem + (uint32_t)(abuf * TC_N);
      for (int i = 0; i < d.ks1 - d.ks0; ++i, ++g) {
        const int slot = g % TC3_STAGES;
        const uint32_t ph = (uint32_t)((g / TC3_STAGES) & 1);
        if (!mbar_wait(&full[slot], ph)) { fail = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint8_t* a = base + slot * 2 * kTcTileBytes;
#pragma unroll
        for (int s4 = 0; s4 < (2 * TC_KC) / 16; ++s4) {
          const uint64_t ad = smem_desc(smem_u32(a) + s4 * 2 * CORE_K);
          const uint64_t bd = smem_desc(smem_u32(a + kTcTileBytes) + s4 * 2 * CORE_K);
          const uint32_t accum = (i == 0 && s4 == 0) ? 0u : 1u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(tc_idesc<F16>()), "r"(accum));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[slot])));
      }
      if (fail) break;
      // the accumulator is complete once every MMA issued so far has finished
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&accf[abuf])));
    }
    if (fail) atomicExch(err, 1);
    // tracks every MMA issued: nobody frees TMEM or leaves before they finish
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&done)));
  } else if (warp >= 2) {
    // ---- epilogue.  Warp w owns TMEM lanes 32 (w % 4) .. (real accumulator rows; complex
    // row R / 2, real part on even lanes) and columns 64 hc .. 64 hc + 63 (hc = (w - 2) / 4),
    // read as two 32-column chunks.  A chunk goes through the warp's shared-memory stage
    // (16 complex rows x 32 columns) so that afterwards lane = column: every global load
    // and store of the epilogue is one row's 32 consecutive complex values per
    // instruction.  D^{-1} and the children's update rows do not depend on the product;
    // they are loaded before the accumulator is waited for (first chunk) or while the
    // previous chunk is stored (second chunk).
    bool fail = false;
    const uint32_t lq = (uint32_t)(warp & 3) * 32u;   // first TMEM lane of this warp
    const int hc = (warp - 2) >> 2;
    float* stg = reinterpret_cast<float*>(base + TC3_STAGES * 2 * kTcTileBytes + TC3_MAX_TASKS * sizeof(Tc3Task)) +
                 (warp - 2) * (TC3_EPI_ROWS * TC3_EPI_LD);
    for (int k = 0; k < ntask && !fail; ++k) {
      const Tc3Task& d = task[k];
      const int abuf = k & 1;
      const uint32_t aph = (uint32_t)((k >> 1) & 1);
      const int nc = d.nc;
      const int rows_out = FWD ? d.m : nc;
      const int i0 = d.row0 + (int)(lq >> 1);   // first complex row of this warp
      // a task without K stages has no product (the per-tile kernel writes nothing either)
      const bool any = d.ks1 > d.ks0;
      const int cw = d.c0 + hc * 64 + lane;     // this lane's column in chunk 0
      float2 dv[TC3_EPI_ROWS], ua[TC3_EPI_ROWS], ub[TC3_EPI_ROWS];
      const int32_t* gs = gsrc + d.g_off * 2;
#pragma unroll
      for (int r = 0; r < TC3_EPI_ROWS; ++r) {
        const int i = i0 + r;
        dv[r] = (FWD && any && i < nc) ? Dinv[d.col0 + i] : make_float2(0.f, 0.f);
      }
      // children's update rows (zero where a row has no such child: adding +0 changes no
      // value but the sign of a zero)
      auto prefetch = [&](int c) {
#pragma unroll
        for (int r = 0; r < TC3_EPI_ROWS; ++r) {
          const int i = i0 + r;
          ua[r] = ub[r] = make_float2(0.f, 0.f);
          if (FWD && any && i >= nc && i < rows_out && c < nrhs) {
            const int s0 = gs[2 * i], s1 = gs[2 * i + 1];
            if (s0 >= 0) ua[r] = U[(int64_t)s0 * ld + c];
            if (s1 >= 0) ub[r] = U[(int64_t)s1 * ld + c];
          }
        }
      };
      if (FWD) prefetch(cw);
      // warp-uniform outcome: the TMEM loads below are warp-collective
      if (!__all_sync(0xffffffffu, mbar_wait(&accf[abuf], aph))) { fail = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + (lq << 16) + (uint32_t)(abuf * TC_N + hc * 64 + h * 32), v);
        // lane = real row: complex row lane / 2, real part on even lanes
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[(lane >> 1) * TC3_EPI_LD + 2 * j + (lane & 1)] = __uint_as_float(v[j]);
        __syncwarp();
        const int c = cw + h * 32;
#pragma unroll
        for (int r = 0; r < TC3_EPI_ROWS; ++r) {
          const int i = i0 + r;
          if (!any || i >= rows_out || c >= nrhs) continue;
          const float2 y = *reinterpret_cast<const float2*>(stg + r * TC3_EPI_LD + 2 * lane);
          if (FWD && i < nc) {
            Z[(int64_t)(d.col0 + i) * ld + c] = cmul(dv[r], y);
          } else if (FWD) {
            U[(int64_t)(d.u_off + i - nc) * ld + c] = cadd(cadd(y, ua[r]), ub[r]);
          } else {
            X[(int64_t)(d.col0 + i) * ld + c] = y;
          }
        }
        __syncwarp();
        if (FWD && h == 0) prefetch(cw + 32);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[abuf])));
    }
    if (fail && lane == 0) atomicExch(err, 1);
  }
  // ---- teardown: every MMA finished, every bulk copy landed, then TMEM is freed
  __syncthreads();
  if (tid == 0 && !mbar_wait(&done, 0)) atomicExch(err, 1);
  if (warp == 0 && lane == 0 && pfail) {
    // copies issued but never consumed land in this CTA's shared memory: wait (bounded)
    for (int g = issued > TC3_STAGES ? issued - TC3_STAGES : 0; g < issued; ++g)
      mbar_wait(&full[g % TC3_STAGES], (uint32_t)((g / TC3_STAGES) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC3_TMEM_COLS));
}

}  // namespace

template <typename WT>
cudaError_t sn_tc2_depth(const DevFactor<float2, WT>& F, int d, bool fwd, bool split, float2* Q, float2* Z,
                         float2* U, float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  constexpr bool H = std::is_same<WT, __half2>::value;
  int* err = sy.err;
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaFuncSetAttribute(k_sn_tc2<true, false, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC2_SMEM);
    cudaFuncSetAttribute(k_sn_tc2<false, false, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC2_SMEM);
    cudaFuncSetAttribute(k_sn_tc2<true, true, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC2_SMEM);
    cudaFuncSetAttribute(k_sn_tc2<false, true, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC2_SMEM);
    cudaFuncSetAttribute(k_sn_tc3<true, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC3_SMEM);
    cudaFuncSetAttribute(k_sn_tc3<false, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC3_SMEM);
    attr_set = true;
  }
  const unsigned gy = (unsigned)((nrhs + TC_N - 1) / TC_N);
  const int64_t* ao = fwd ? F.h_tas_f_off : F.h_tas_b_off;
  const int64_t aa = ao[d], ab = ao[d + 1];
  if (ab <= aa) return cudaSuccess;
  if (fwd)
    launch_k(k_tc_assemble<true, H>, dim3((unsigned)(ab - aa), gy), 256, 0, st, F.nodes, F.gsrc, F.rows, F.tnode, F.tpre,
                                                                        F.tas_f + aa, Q, Z, U, Q, Bst, nrhs, ld);
  else
    launch_k(k_tc_assemble<false, H>, dim3((unsigned)(ab - aa), gy), 256, 0, st, F.nodes, F.gsrc, F.rows, F.tnode, F.tpre,
                                                                         F.tas_b + aa, Q, Z, U, Q, Bst, nrhs, ld);
  count_launches(1);
  const uint8_t* TW = fwd ? F.tw_f : F.tw_b;
  const int64_t* tof = fwd ? F.h_fwd_off : F.h_bwd_off;
  const int64_t ntasks = (tof[d + 1] - tof[d]) * (int64_t)gy;
  const int64_t grid3 = ntasks < F.n_sm ? ntasks : F.n_sm;
  if (!split && sy.tc_persist && grid3 > 0 && (ntasks + grid3 - 1) / grid3 <= TC3_MAX_TASKS) {
    const int64_t a = tof[d], b = tof[d + 1];
    const int2* tl = (fwd ? F.fwd_tiles : F.bwd_tiles) + a;
    const unsigned grid = (unsigned)grid3;
    if (fwd)
      launch_k_overlap(k_sn_tc3<true, H>, dim3(grid), TC3_THREADS, TC3_SMEM, st, F.nodes, TW, F.tnode, F.tpre, Bst,
                       F.Dinv, F.gsrc, tl, (int)(b - a), (int)gy, Z, U, Q, nrhs, ld, err);
    else
      launch_k_overlap(k_sn_tc3<false, H>, dim3(grid), TC3_THREADS, TC3_SMEM, st, F.nodes, TW, F.tnode, F.tpre, Bst,
                       F.Dinv, F.gsrc, tl, (int)(b - a), (int)gy, Z, U, Q, nrhs, ld, err);
    count_launches(1);
  } else if (!split) {
    const int64_t* to = fwd ? F.h_fwd_off : F.h_bwd_off;
    const int64_t a = to[d], b = to[d + 1];
    const int2* tl = (fwd ? F.fwd_tiles : F.bwd_tiles) + a;
    if (fwd)
      launch_k(k_sn_tc2<true, false, H>, dim3((unsigned)(b - a), gy), TC_THREADS, TC2_SMEM, st, F.nodes, TW, F.tnode,
               F.tpre, Bst, F.Dinv, F.gsrc, tl, nullptr, Z, U, Q, nullptr, nrhs, ld, err);
    else
      launch_k(k_sn_tc2<false, false, H>, dim3((unsigned)(b - a), gy), TC_THREADS, TC2_SMEM, st, F.nodes, TW, F.tnode,
               F.tpre, Bst, F.Dinv, F.gsrc, tl, nullptr, Z, U, Q, nullptr, nrhs, ld, err);
    count_launches(1);
  } else {
    const int64_t* io = fwd ? F.h_tcf_item_off : F.h_tcb_item_off;
    const int64_t* uo = fwd ? F.h_tcf_unit_off : F.h_tcb_unit_off;
    const int64_t ia = io[d], ib = io[d + 1], ua = uo[d], ub = uo[d + 1];
    const int4* its = (fwd ? F.tcf_items : F.tcb_items) + ia;
    const int4* uns = (fwd ? F.tcf_units : F.tcb_units) + ua;
    if (fwd) {
      launch_k(k_sn_tc2<true, true, H>, dim3((unsigned)(ib - ia), gy), TC_THREADS, TC2_SMEM, st, F.nodes, TW, F.tnode,
               F.tpre, Bst, F.Dinv, F.gsrc, nullptr, its, Z, U, Q, Ptc, nrhs, ld, err);
      launch_k(k_sn_tc_reduce<true>, dim3((unsigned)(ub - ua), gy, TC_ROWS / TC_RED_ROWS), 256, 0, st, F.nodes,
               F.Dinv, F.gsrc, uns, ia, ib - ia, Ptc, Z, U, Q, nrhs, ld);
    } else {
      launch_k(k_sn_tc2<false, true, H>, dim3((unsigned)(ib - ia), gy), TC_THREADS, TC2_SMEM, st, F.nodes, TW,
               F.tnode, F.tpre, Bst, F.Dinv, F.gsrc, nullptr, its, Z, U, Q, Ptc, nrhs, ld, err);
      launch_k(k_sn_tc_reduce<false>, dim3((unsigned)(ub - ua), gy, TC_ROWS / TC_RED_ROWS), 256, 0, st, F.nodes,
               F.Dinv, F.gsrc, uns, ia, ib - ia, Ptc, Z, U, Q, nrhs, ld);
    }
    count_launches(2);
  }
  return cudaGetLastError();
}

template cudaError_t sn_tc2_depth<__nv_bfloat162>(const DevFactor<float2, __nv_bfloat162>&, int, bool, bool, float2*,
                                                   float2*, float2*, float2*, uint8_t*, int, int, const SkSync&,
                                                   cudaStream_t);
template cudaError_t sn_tc2_depth<__half2>(const DevFactor<float2, __half2>&, int, bool, bool, float2*, float2*,
                                           float2*, float2*, uint8_t*, int, int, const SkSync&, cudaStream_t);

}  // namespace stmg
