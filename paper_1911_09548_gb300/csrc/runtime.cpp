// Host runtime and C ABI of the space-time multigrid library (see include/st_mg.h).
//
// Setup builds, per space level s (finest first), the Kuhn mesh, M_sigma and K_nu
// (assembled on the finest mesh, Galerkin products P_x^T A P_x below it), G, K_n
// and P_x; per time level l the coarsening decision of eq. CoarseningRule, the
// residual coefficient arrays and the factor of the shared slab matrix; then it
// uploads everything and sizes one workspace.  The V-cycle (Section 2.1) with the
// hybrid smoother S^nu A S^nu (Section 4) is a fixed sequence of kernel launches
// on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/st_mg.h"
#include "device.h"
#include "host.h"

using namespace stmg;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

struct CudaError {
  cudaError_t e;
  const char* where;
};

// A factor that the requested arithmetic cannot hold (reported as ST_MG_ERR_NUMERIC).
struct NumericError {
  const char* what;
};


// Host-side tile and item lists of one factor (kept alive: the device view points at them).
struct FactorLists {
  std::vector<int64_t> fo, bo, fsi, fsu, bsi, bsu, tfi, tfu, tbi, tbu, asf, asb;
  int64_t df_items = 0;   // split-K items of the larger sweep (partial blocks of a dataflow solve)
  int64_t df_words = 0;   // counter words of a dataflow sweep: 1 + units + nodes
};

#define CK(call)                                                    \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) throw CudaError{e_, #call};              \
  } while (0)

}  // namespace

namespace stmg {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace stmg

namespace {
// Device allocations freed together: a handle's own buffers, or one cached factor.
struct DevArena {
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int n_sm = 152;
  DevArena() = default;
  DevArena(const DevArena&) = delete;
  DevArena& operator=(const DevArena&) = delete;
  ~DevArena() {
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  T* dalloc(int64_t count) {
    void* p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) throw CudaError{e, "cudaMalloc"};
    allocs.push_back(p);
    bytes += count * (int64_t)sizeof(T);
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* d = dalloc<T>((int64_t)v.size());
    if (!v.empty()) CK(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
};

// Device factor of one time level's slab matrix (every slab of a level shares it,
// Section 2.1) in that level's precision.  Read-only once built, so handles with the
// same mesh, materials, DG degree, tau and precision can share one.
struct SlabFactor {
  DevArena mem;
  DevFactor<double> dr;
  DevFactor<double2> dc;
  DevFactor<float> drf;                                   // mixed precision (FP32 apply)
  DevFactor<float2> dcf;
  DevFactor<double, float2> drd;                          // double-float (FP64-accurate) apply
  DevFactor<double2, float4> dcd;
  DevFactor<float2, __nv_bfloat162> dcb;                  // BF16 factor on the tensor cores
  DevFactor<float2, __half2> dch;                         // FP16 factor on the tensor cores
  FactorLists lists;
  int64_t w_bytes = 0;                                   // device bytes of the factor blocks
  int64_t u_rows = 0, max_items = 0, max_tc_items = 0, max_stage_tiles = 0;
};

// Device factor of one space level's nodal matrix K_n (exact auxiliary solve, Section 4).
struct NodalFactor {
  DevArena mem;
  DevFactor<double> kn;
  DevFactor<double, float2> kn_df;                        // the same factor as FP32 pairs
  DevFactor<float> kn_f;                                  // the same factor rounded to FP32
  FactorLists kn_lists, kn_df_lists, kn_f_lists;
  int64_t u_rows = 0, max_items = 0;
};

// Process-wide cache of device factors, keyed by everything that determines them
// (device, mesh, space level, materials, DG degree, tau, precision).  Entries stay
// resident until st_mg_cache_trim evicts them; a handle holds a reference to each
// entry it uses, so an entry in use is never evicted.
struct FactorCache {
  struct Entry {
    std::shared_ptr<SlabFactor> slab;
    std::shared_ptr<NodalFactor> nodal;
    int64_t last_use = 0;
    int64_t bytes() const { return slab ? slab->mem.bytes : nodal ? nodal->mem.bytes : 0; }
    long refs() const { return slab ? slab.use_count() : nodal ? nodal.use_count() : 0; }
  };
  std::mutex mu;
  std::map<std::string, Entry> map;
  int64_t tick = 0, hits = 0, misses = 0;
};
// never destroyed: at process exit the device memory goes with the context
FactorCache& factor_cache() {
  static FactorCache* c = new FactorCache();
  return *c;
}

void cache_put(const std::string& key, std::shared_ptr<SlabFactor> sf, std::shared_ptr<NodalFactor> nf) {
  auto& C = factor_cache();
  std::lock_guard<std::mutex> g(C.mu);
  auto& e = C.map[key];
  if (sf) e.slab = sf;
  if (nf) e.nodal = nf;
  e.last_use = ++C.tick;
}

// Second look at the device phase: an entry some other handle left since this handle's
// host phase looked counts as a hit; otherwise this handle builds it (a miss).  Every
// factor a handle uses is thus counted once, as a hit or as a miss.
template <typename T>
std::shared_ptr<T> cache_recheck(const std::string& key) {
  auto& C = factor_cache();
  std::lock_guard<std::mutex> g(C.mu);
  auto it = C.map.find(key);
  std::shared_ptr<T> p;
  if (it != C.map.end()) {
    if constexpr (std::is_same<T, SlabFactor>::value) p = it->second.slab;
    else p = it->second.nodal;
  }
  if (p) {
    it->second.last_use = ++C.tick;
    ++C.hits;
  } else {
    ++C.misses;
  }
  return p;
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}
}  // namespace

struct st_mg_s {
  st_mg_problem prob{};
  st_mg_options opt{};
  std::vector<double> nu, sigma;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool host_only = false;              // built by st_mg_setup_host: no device state
  int n_sm = 152;
  double* stage_f = nullptr;           // host-buffer solve staging (allocated on first use)
  double* stage_x = nullptr;
  int q = 1;
  int B = 1;                            // problems solved together (batch)
  // ragged batch (st_mg_problem.batch_nt): problem b has pnt[b] slabs of its own step T / pnt[b];
  // it enters the time hierarchy at level pent[b] (whose step equals its own) in slot pslot[b],
  // and the caller's vectors hold its columns at poff[b] .. poff[b] + pnt[b] q of rows of prow
  bool ragged = false;
  std::vector<int> pnt, pent, pslot;
  std::vector<int64_t> poff;
  int64_t prow = 0;
  int64_t user_len = 0;                 // length of the caller's f and x (edges x prow)
  DevArena mem;                         // the handle's own device buffers
  uint64_t mat_hash = 0;                // of (n_cube, nu, sigma): the factor cache's material key
  bool use_cache = false;               // factors from / into the process-wide cache
  bool pending_upload = false;          // host phase done (st_mg_setup_begin), device phase not yet
  std::vector<std::string> lkey, skey;  // cache keys per time level / space level

  template <typename T>
  T* dalloc(int64_t count) { return mem.dalloc<T>(count); }
  template <typename T>
  T* upload(const std::vector<T>& v) { return mem.upload(v); }

  struct Space {
    TetMesh mesh;
    Csr M, K, Kn, Px, PxT, GT;            // Px: prolongation from space level s+1 to s
    std::vector<int32_t> gtail, ghead;
    std::vector<int8_t> gt_sign;
    int32_t ne = 0, nn = 0;
    // device
    int64_t* rowptr = nullptr; int32_t* col = nullptr; double* Mv = nullptr;
    int32_t* gtail_d = nullptr; int32_t* ghead_d = nullptr;
    int64_t* gt_rowptr = nullptr; int32_t* gt_col = nullptr; int8_t* gt_sign_d = nullptr;
    int64_t* kn_rowptr = nullptr; int32_t* kn_col = nullptr; double* kn_val = nullptr; double* kn_dinv = nullptr;
    int64_t* px_rowptr = nullptr; int32_t* px_col = nullptr; double* px_val = nullptr;
    int64_t* pxt_rowptr = nullptr; int32_t* pxt_col = nullptr; double* pxt_val = nullptr;
    SupernodalFactor<double> knF;         // host factor (released after upload)
    std::shared_ptr<NodalFactor> nf;      // device factor (own, or shared through the cache)
    NDCoords ecoord, ncoord;
  };
  std::vector<Space> space;

  struct Level {
    int s = 0, N_t = 1;
    int B = 1;                                              // problems on this level (ragged: fewer on finer levels)
    double tau = 1.0;
    double *v0 = nullptr, *v1 = nullptr, *v2 = nullptr;   // residual coefficients per nnz
    float2 *p0 = nullptr, *p1 = nullptr, *p2 = nullptr;   // the same as (hi, lo) FP32 pairs
    float *q0 = nullptr, *q1 = nullptr, *q2 = nullptr;    // ... rounded to FP32 (residual_prec 1)
    SupernodalFactor<double> fr;                            // host factors (released after upload)
    SupernodalFactor<cplx> fc;
    std::shared_ptr<SlabFactor> fac;                        // device factor (own, or from the cache)
    int prec = 0;                                           // 0 FP64, 1 FP32, 2 double-float, 3 BF16
    int split_waves = 2;                                    // tiled / split-K threshold (autotuned)
    int tc_mode = 0;                                        // 16-bit factor: 0 tensor cores (persistent tiled depths),
                                                            // 1 CUDA-core reference, 2 tensor cores one CTA per tile
    double *f = nullptr, *x = nullptr, *r = nullptr;      // level vectors (levels >= 1)
    int64_t len = 0;
  };
  std::vector<Level> lv;

  // workspaces
  void *sQ = nullptr, *sZ = nullptr, *sU = nullptr, *sP = nullptr;   // sP: split-K partials
  int ld_slab = 1;
  double *nQ = nullptr, *nZ = nullptr, *nU = nullptr, *nP = nullptr;
  int ld_nod = 1;
  double *ny = nullptr, *nz = nullptr, *nw = nullptr;
  double* tmp_fine = nullptr;
  double* g1 = nullptr;                 // one-slab right-hand side of the forward substitution
  double* r0 = nullptr;                 // finest residual
  double* partial = nullptr;
  double* scalar = nullptr;
  double* zero_f = nullptr;             // finest-level zero load of the rate harness (allocated on first use)
  int sk_k = kSkK;                      // K columns of a split-K work item (st_mg_options.split_k)
  int tc_k = kTcSplitK;                 // ... of a tensor-core split-K item (st_mg_options.tc_split_k)
  float2* xsplit = nullptr;             // x as FP32 pairs for the double-float residual
  bool res32 = false;                   // residual_prec 1: FP32 residuals inside a correction-form V-cycle
  float* xf32 = nullptr;                // x as FP32 for those residuals
  double* corr_r = nullptr;             // correction form: outer residual r = f - L x (finest level)
  double* corr_e = nullptr;             //   and the correction e = V(r), x += e
  int nodal_prec = 0;                   // nodal K_n solve: 0 FP64, 1 FP32 (slab_prec 1, 3), 2 double-float
  int* tc_err = nullptr;                // flags[0]: set by a block whose bounded wait timed out
  int* flags = nullptr;                 // [0] wait error, [1] spare, [2..3] grid-barrier words
  SkSync sk;                            // persistent split-K solve: barrier words + error flag
  float2* tcP = nullptr;                // tensor-core split-K partials
  uint8_t* tcB = nullptr;               // tensor-core right-hand-side tiles of one depth
  unsigned* colmax = nullptr;           // FP16 slab solve: per-column maxima (scaling)
  double* load_b = nullptr;             // load assembly staging: space part [n_edge], time part [N_t q]
  double* load_c = nullptr;
  double* bn_partial = nullptr;         // per-problem norm scratch
  double* bn_out = nullptr;
  // captured V-cycle (replayed while f and x stay the same buffers)
  cudaGraphExec_t graph_exec = nullptr;
  const double* graph_f = nullptr;
  double* graph_x = nullptr;
  int64_t graph_launches = 0;
  bool df_residual = false;
  double2 c0{}, c1{}, s1{};             // DG(1) complex slab transformation

  ~st_mg_s() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
  }
};

namespace {

using Handle = st_mg_s;

CsrView view(const Handle::Space& S) { return CsrView{S.ne, S.rowptr, S.col}; }

// Element conversion of factor blocks to the device type (FP64 as is, or rounded to FP32).
inline void to_dev(double a, double& b) { b = a; }
inline void to_dev(const cplx& a, double2& b) { b = make_double2(a.re, a.im); }
inline void to_dev(double a, float& b) { b = (float)a; }
inline void to_dev(const cplx& a, float2& b) { b = make_float2((float)a.re, (float)a.im); }
inline void to_dev(const cplx& a, __nv_bfloat162& b) { b = __floats2bfloat162_rn((float)a.re, (float)a.im); }
inline void to_dev(const cplx& a, __half2& b) { b = __floats2half2_rn((float)a.re, (float)a.im); }
// double-float pairs: hi = FP32 rounding, lo = FP32 rounding of the remainder
inline void to_dev(double a, float2& b, int) {
  const float h = (float)a;
  b = make_float2(h, (float)(a - (double)h));
}
inline void to_dev(const cplx& a, float4& b) {
  const float rh = (float)a.re, ih = (float)a.im;
  b = make_float4(rh, (float)(a.re - (double)rh), ih, (float)(a.im - (double)ih));
}
template <typename DT, typename T>
std::vector<DT> convert(const std::vector<T>& v) {
  std::vector<DT> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) to_dev(v[i], out[i]);
  return out;
}
template <typename DT, typename T>
std::vector<DT> convert_pairs(const std::vector<T>& v);
template <>
std::vector<float2> convert_pairs<float2, double>(const std::vector<double>& v) {
  std::vector<float2> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) to_dev(v[i], out[i], 0);
  return out;
}
template <>
std::vector<float4> convert_pairs<float4, cplx>(const std::vector<cplx>& v) {
  std::vector<float4> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) to_dev(v[i], out[i]);
  return out;
}
template <typename WT, typename T>
std::vector<WT> convert_w(const std::vector<T>& v) {
  if constexpr (std::is_same<WT, float2>::value && std::is_same<T, double>::value) return convert_pairs<float2>(v);
  else if constexpr (std::is_same<WT, float4>::value) return convert_pairs<float4>(v);
  else return convert<WT>(v);
}

// byte offset of element (row, k) in a 128 x 64 BF16 operand tile, K-major core
// matrices of 8 rows x 16 bytes (128 B between K-adjacent cores, 1024 B between
// 8-row groups) -- the layout the tensor-core kernels read with one descriptor
inline size_t tile_off(int row, int k) {
  return (size_t)(row >> 3) * 1024 + (size_t)(k >> 3) * 128 + (size_t)(row & 7) * 16 + (size_t)(k & 7) * 2;
}

inline uint16_t bf16_bits(float v) {
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  uint16_t u;
  std::memcpy(&u, &b, 2);
  return u;
}

inline uint16_t f16_bits(float v) {
  __half b = __float2half_rn(v);
  uint16_t u;
  std::memcpy(&u, &b, 2);
  return u;
}

// Largest |Re| or |Im| of a factor's blocks W_s; an FP16 factor needs it well inside
// FP16's range (65504), the BF16 one has FP32's exponent range.
double max_abs_entry(const SupernodalFactor<cplx>& F) {
  double m = 0.0;
  for (const cplx& w : F.W) m = std::max(m, std::max(std::fabs(w.re), std::fabs(w.im)));
  return m;
}

// Tensor-core operand tiles of a complex factor: for node s, forward tile (rt, ks)
// holds W rows 64 rt .. 64 rt + 63 and columns 32 ks .. 32 ks + 31, each complex
// entry a + ib as the real block [[a, -b], [b, a]]; backward tile (rt, ks) holds the
// same for W^T (rows of W^T = columns of W).  Zero outside the node's block.
template <typename WT>
void build_tc_tiles(DevArena& h, const SupernodalFactor<cplx>& F, DevFactor<float2, WT>& D, FactorLists& Lh) {
  const auto bits = [](float v) { return std::is_same<WT, __half2>::value ? f16_bits(v) : bf16_bits(v); };
  const size_t TB = kTcTileBytes;
  std::vector<int4> tnode(F.nodes.size());
  std::vector<int2> tpre(F.nodes.size());
  int64_t nf = 0, nb = 0;
  for (size_t s = 0; s < F.nodes.size(); ++s) {
    const auto& a = F.nodes[s];
    const int m = a.nc + a.nr;
    const int rtf = (m + 63) / 64, ksf = (a.nc + 31) / 32, rtb = (a.nc + 63) / 64, ksb = (m + 31) / 32;
    tnode[s] = make_int4((int)nf, ksf, (int)nb, ksb);
    nf += (int64_t)rtf * ksf;
    nb += (int64_t)rtb * ksb;
  }
  std::vector<uint8_t> tf((size_t)nf * TB, 0), tb((size_t)nb * TB, 0);
  auto put = [&](uint8_t* tile, int i, int k, cplx w) {
    const uint16_t re = bits((float)w.re), im = bits((float)w.im), nim = bits(-(float)w.im);
    std::memcpy(tile + tile_off(2 * i, 2 * k), &re, 2);
    std::memcpy(tile + tile_off(2 * i, 2 * k + 1), &nim, 2);
    std::memcpy(tile + tile_off(2 * i + 1, 2 * k), &im, 2);
    std::memcpy(tile + tile_off(2 * i + 1, 2 * k + 1), &re, 2);
  };
  for (size_t s = 0; s < F.nodes.size(); ++s) {
    const auto& a = F.nodes[s];
    const int nc = a.nc, m = nc + a.nr;
    const cplx* W = F.W.data() + a.w_off;
    const int4 tn = tnode[s];
    for (int r = 0; r < m; ++r)
      for (int k = 0; k < nc; ++k) {
        const cplx w = W[(int64_t)r * nc + k];
        if (w.re == 0.0 && w.im == 0.0) continue;
        uint8_t* t = tf.data() + ((size_t)tn.x + (size_t)(r / 64) * tn.y + (k / 32)) * TB;
        put(t, r % 64, k % 32, w);
        // backward: row k of W^T (k < nc), column r
        uint8_t* u = tb.data() + ((size_t)tn.z + (size_t)(k / 64) * tn.w + (r / 32)) * TB;
        put(u, k % 64, r % 32, w);
      }
  }
  // per depth: prefix of k stages and the (node, k stage) assembly lists
  std::vector<int2> asf, asb;
  Lh.asf.assign(F.max_depth + 2, 0);
  Lh.asb.assign(F.max_depth + 2, 0);
  int64_t max_stage = 0;
  for (int d = 0; d <= F.max_depth; ++d) {
    Lh.asf[d] = (int64_t)asf.size();
    Lh.asb[d] = (int64_t)asb.size();
    int pf = 0, pb = 0;
    for (size_t s = 0; s < F.nodes.size(); ++s) {
      if (F.nodes[s].depth != d) continue;
      tpre[s] = make_int2(pf, pb);
      for (int ks = 0; ks < tnode[s].y; ++ks) asf.push_back(make_int2((int)s, ks));
      for (int ks = 0; ks < tnode[s].w; ++ks) asb.push_back(make_int2((int)s, ks));
      pf += tnode[s].y;
      pb += tnode[s].w;
    }
    max_stage = std::max<int64_t>(max_stage, std::max(pf, pb));
  }
  Lh.asf[F.max_depth + 1] = (int64_t)asf.size();
  Lh.asb[F.max_depth + 1] = (int64_t)asb.size();
  D.tw_f = h.upload(tf);
  D.tw_b = h.upload(tb);
  D.tnode = h.upload(tnode);
  D.tpre = h.upload(tpre);
  D.tas_f = h.upload(asf);
  D.tas_b = h.upload(asb);
  D.h_tas_f_off = Lh.asf.data();
  D.h_tas_b_off = Lh.asb.data();
  D.max_stage_tiles = max_stage;
}

template <typename T, typename DT, typename WT>
void make_dev_factor(DevArena& h, const SupernodalFactor<T>& F, DevFactor<DT, WT>& D, FactorLists& Lh, int sk_k,
                     int tc_k, int bm = kSnBM) {
  std::vector<int64_t>& fo = Lh.fo;
  std::vector<int64_t>& bo = Lh.bo;
  D.n = F.n;
  D.nnodes = (int32_t)F.nodes.size();
  D.max_depth = F.max_depth;
  std::vector<DevNode> nodes(F.nodes.size());
  for (size_t s = 0; s < F.nodes.size(); ++s) {
    const auto& a = F.nodes[s];
    nodes[s] = DevNode{a.col0, a.nc, a.nr, 0, a.w_off, a.row_off, a.u_off, F.gather_off[s]};
  }
  std::vector<int2> ft, bt;
  D.bm = bm;
  fo.assign(F.max_depth + 2, 0);
  bo.assign(F.max_depth + 2, 0);
  for (int d = 0; d <= F.max_depth; ++d) {
    fo[d] = (int64_t)ft.size();
    bo[d] = (int64_t)bt.size();
    for (size_t s = 0; s < F.nodes.size(); ++s) {
      const auto& a = F.nodes[s];
      if (a.depth != d) continue;
      const int mf = (a.nc + a.nr + bm - 1) / bm, mb = (a.nc + bm - 1) / bm;
      for (int t = 0; t < mf; ++t) ft.push_back(make_int2((int)s, t));
      for (int t = 0; t < mb; ++t) bt.push_back(make_int2((int)s, t));
    }
    // longest K range first (stable): blocks, and the tasks a persistent kernel deals out
    // round robin, then start with the long tiles and the depth ends with short ones
    auto kf = [&](const int2& t) { return std::min((t.y + 1) * bm, F.nodes[t.x].nc); };
    auto kb = [&](const int2& t) {
      const auto& a = F.nodes[t.x];
      return a.nc + a.nr - (t.y * bm / 32) * 32;
    };
    std::stable_sort(ft.begin() + fo[d], ft.end(), [&](const int2& x, const int2& y) { return kf(x) > kf(y); });
    std::stable_sort(bt.begin() + bo[d], bt.end(), [&](const int2& x, const int2& y) { return kb(x) > kb(y); });
  }
  fo[F.max_depth + 1] = (int64_t)ft.size();
  bo[F.max_depth + 1] = (int64_t)bt.size();
  // split-K items: forward rows [0, nc+nr) against K [0, nc) (rows inside L11^{-1}
  // stop at their last row); backward rows [0, nc) against K [row0, nc+nr)
  std::vector<int4> fsi, fsu, bsi, bsu;
  Lh.fsi.assign(F.max_depth + 2, 0);
  Lh.fsu.assign(F.max_depth + 2, 0);
  Lh.bsi.assign(F.max_depth + 2, 0);
  Lh.bsu.assign(F.max_depth + 2, 0);
  int64_t max_items = 0;
  for (int d = 0; d <= F.max_depth; ++d) {
    Lh.fsi[d] = (int64_t)fsi.size();
    Lh.fsu[d] = (int64_t)fsu.size();
    Lh.bsi[d] = (int64_t)bsi.size();
    Lh.bsu[d] = (int64_t)bsu.size();
    for (size_t s = 0; s < F.nodes.size(); ++s) {
      const auto& a = F.nodes[s];
      if (a.depth != d) continue;
      const int m = a.nc + a.nr;
      for (int r0 = 0; r0 < m; r0 += kSkRows) {
        const int kend = (r0 + kSkRows <= a.nc) ? r0 + kSkRows : a.nc;
        const int first = (int)fsi.size();
        for (int k0 = 0; k0 < kend; k0 += sk_k) fsi.push_back(make_int4((int)s, r0, k0, std::min(k0 + sk_k, kend)));
        fsu.push_back(make_int4((int)s, r0, first, (int)fsi.size()));
      }
      for (int r0 = 0; r0 < a.nc; r0 += kSkRows) {
        const int first = (int)bsi.size();
        for (int k0 = r0; k0 < m; k0 += sk_k) bsi.push_back(make_int4((int)s, r0, k0, std::min(k0 + sk_k, m)));
        bsu.push_back(make_int4((int)s, r0, first, (int)bsi.size()));
      }
    }
    max_items = std::max<int64_t>(max_items, (int64_t)fsi.size() - Lh.fsi[d]);
    max_items = std::max<int64_t>(max_items, (int64_t)bsi.size() - Lh.bsi[d]);
  }
  Lh.fsi[F.max_depth + 1] = (int64_t)fsi.size();
  Lh.fsu[F.max_depth + 1] = (int64_t)fsu.size();
  Lh.bsi[F.max_depth + 1] = (int64_t)bsi.size();
  Lh.bsu[F.max_depth + 1] = (int64_t)bsu.size();
  D.fs_items = h.upload(fsi);
  D.fs_units = h.upload(fsu);
  D.bs_items = h.upload(bsi);
  D.bs_units = h.upload(bsu);
  D.h_fs_item_off = Lh.fsi.data();
  D.h_fs_unit_off = Lh.fsu.data();
  D.h_bs_item_off = Lh.bsi.data();
  D.h_bs_unit_off = Lh.bsu.data();
  D.d_fs_item_off = h.upload(Lh.fsi);
  D.d_fs_unit_off = h.upload(Lh.fsu);
  D.d_bs_item_off = h.upload(Lh.bsi);
  D.d_bs_unit_off = h.upload(Lh.bsu);
  D.max_items = max_items;
  D.n_sm = h.n_sm;
  // dataflow split-K solve: one task list per sweep in topological order (forward:
  // deepest depth first; backward: root first; each depth's items before its units)
  {
    const size_t nn = F.nodes.size();
    std::vector<int2> tf, tb, ch(nn), par(nn);
    std::vector<int32_t> iuf(fsi.size(), 0), iub(bsi.size(), 0), nuf(nn, 0), nub(nn, 0);
    for (size_t u = 0; u < fsu.size(); ++u) {
      for (int q = fsu[u].z; q < fsu[u].w; ++q) iuf[q] = (int32_t)u;
      ++nuf[fsu[u].x];
    }
    for (size_t u = 0; u < bsu.size(); ++u) {
      for (int q = bsu[u].z; q < bsu[u].w; ++q) iub[q] = (int32_t)u;
      ++nub[bsu[u].x];
    }
    for (int d = F.max_depth; d >= 0; --d) {
      for (int64_t q = Lh.fsi[d]; q < Lh.fsi[d + 1]; ++q) tf.push_back(make_int2(0, (int)q));
      for (int64_t u = Lh.fsu[d]; u < Lh.fsu[d + 1]; ++u) tf.push_back(make_int2(1, (int)u));
    }
    for (int d = 0; d <= F.max_depth; ++d) {
      for (int64_t q = Lh.bsi[d]; q < Lh.bsi[d + 1]; ++q) tb.push_back(make_int2(0, (int)q));
      for (int64_t u = Lh.bsu[d]; u < Lh.bsu[d + 1]; ++u) tb.push_back(make_int2(1, (int)u));
    }
    for (size_t t = 0; t < nn; ++t) {
      ch[t] = make_int2(F.nodes[t].child[0], F.nodes[t].child[1]);
      par[t] = make_int2(F.nodes[t].parent, -1);
    }
    D.df_tasks_f = h.upload(tf);
    D.df_tasks_b = h.upload(tb);
    D.df_item_unit_f = h.upload(iuf);
    D.df_item_unit_b = h.upload(iub);
    D.df_node_units_f = h.upload(nuf);
    D.df_node_units_b = h.upload(nub);
    D.df_children = h.upload(ch);
    D.df_parent = h.upload(par);
    D.n_df_tasks_f = (int64_t)tf.size();
    D.n_df_tasks_b = (int64_t)tb.size();
    D.n_fs_items = (int64_t)fsi.size();
    D.n_bs_items = (int64_t)bsi.size();
    D.n_fs_units = (int64_t)fsu.size();
    D.n_bs_units = (int64_t)bsu.size();
    Lh.df_items = std::max<int64_t>(D.n_fs_items, D.n_bs_items);
    Lh.df_words = 1 + std::max<int64_t>(D.n_fs_units, D.n_bs_units) + (int64_t)nn;
  }
  // tensor-core split-K items: the tiles above, each cut into tc_k-wide K chunks (a multiple
  // of the 32-column stage)
  std::vector<int4> tfi, tfu, tbi, tbu;
  Lh.tfi.assign(F.max_depth + 2, 0);
  Lh.tfu.assign(F.max_depth + 2, 0);
  Lh.tbi.assign(F.max_depth + 2, 0);
  Lh.tbu.assign(F.max_depth + 2, 0);
  int64_t max_tc = 0;
  for (int d = 0; d <= F.max_depth; ++d) {
    Lh.tfi[d] = (int64_t)tfi.size();
    Lh.tfu[d] = (int64_t)tfu.size();
    Lh.tbi[d] = (int64_t)tbi.size();
    Lh.tbu[d] = (int64_t)tbu.size();
    for (size_t s = 0; s < F.nodes.size(); ++s) {
      const auto& a = F.nodes[s];
      if (a.depth != d) continue;
      const int m = a.nc + a.nr;
      for (int rt = 0; rt * kSnBM < m; ++rt) {
        const int r0 = rt * kSnBM;
        const int kend = (r0 + kSnBM <= a.nc) ? r0 + kSnBM : a.nc;
        const int first = (int)tfi.size();
        for (int k0 = 0; k0 < kend; k0 += tc_k)
          tfi.push_back(make_int4((int)s, rt, k0, std::min(k0 + tc_k, kend)));
        tfu.push_back(make_int4((int)s, rt, first, (int)tfi.size()));
      }
      for (int rt = 0; rt * kSnBM < a.nc; ++rt) {
        const int r0 = rt * kSnBM;
        const int kbeg = (r0 / 32) * 32;   // the tensor-core stage width
        const int first = (int)tbi.size();
        for (int k0 = kbeg; k0 < m; k0 += tc_k) tbi.push_back(make_int4((int)s, rt, k0, std::min(k0 + tc_k, m)));
        tbu.push_back(make_int4((int)s, rt, first, (int)tbi.size()));
      }
    }
    max_tc = std::max<int64_t>(max_tc, (int64_t)tfi.size() - Lh.tfi[d]);
    max_tc = std::max<int64_t>(max_tc, (int64_t)tbi.size() - Lh.tbi[d]);
  }
  Lh.tfi[F.max_depth + 1] = (int64_t)tfi.size();
  Lh.tfu[F.max_depth + 1] = (int64_t)tfu.size();
  Lh.tbi[F.max_depth + 1] = (int64_t)tbi.size();
  Lh.tbu[F.max_depth + 1] = (int64_t)tbu.size();
  D.tcf_items = h.upload(tfi);
  D.tcf_units = h.upload(tfu);
  D.tcb_items = h.upload(tbi);
  D.tcb_units = h.upload(tbu);
  D.h_tcf_item_off = Lh.tfi.data();
  D.h_tcf_unit_off = Lh.tfu.data();
  D.h_tcb_item_off = Lh.tbi.data();
  D.h_tcb_unit_off = Lh.tbu.data();
  D.max_tc_items = max_tc;
  D.nodes = h.upload(nodes);
  D.W = h.upload(convert_w<WT>(F.W));
  D.Dinv = h.upload(convert<DT>(F.Dinv));
  D.rows = h.upload(F.rows);
  D.gsrc = h.upload(F.gsrc);
  D.iperm = h.upload(F.iperm);
  D.fwd_tiles = h.upload(ft);
  D.bwd_tiles = h.upload(bt);
  D.h_fwd_off = fo.data();
  D.h_bwd_off = bo.data();
  D.u_rows = F.u_rows;
  D.macs_per_rhs = F.flops_apply_per_rhs;
}

int hw_threads(int req) {
  if (req > 0) return req;
  unsigned n = std::thread::hardware_concurrency();
  return n ? (int)n : 1;
}

// ---------------------------------------------------------------- operations
// outer: a residual whose accuracy decides the fixed point (the solve's stopping test, the
// public entry points, the correction form's residual); inner: the smoothers' and the
// restriction's residuals inside a V-cycle, FP32 with residual_prec 1.
void op_residual(Handle& h, int l, const double* f, const double* x, double* r, double* norm_sq_host,
                 bool outer = false) {
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  int nb = 0;
  double* part = norm_sq_host ? h.partial : nullptr;
  if (h.res32 && !outer) {
    CK(to_float(x, h.xf32, L.len, h.stream));
    if (h.prob.degree == 0)
      CK(residual_dg0_f32(view(S), L.q0, L.q1, f, h.xf32, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
    else
      CK(residual_dg1_f32(view(S), L.q0, L.q1, L.q2, f, h.xf32, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
  } else if (h.df_residual) {
    CK(split_pairs(x, h.xsplit, L.len, h.stream));
    if (h.prob.degree == 0)
      CK(residual_dg0_df(view(S), L.p0, L.p1, f, h.xsplit, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
    else
      CK(residual_dg1_df(view(S), L.p0, L.p1, L.p2, f, h.xsplit, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
  } else if (h.prob.degree == 0) {
    CK(residual_dg0(view(S), L.v0, L.v1, f, x, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
  } else {
    CK(residual_dg1(view(S), L.v0, L.v1, L.v2, f, x, r, L.N_t * L.B, L.N_t, part, &nb, h.stream));
  }
  if (norm_sq_host) {
    CK(reduce_partials(h.partial, nb, h.scalar, h.stream));
    CK(cudaMemcpyAsync(norm_sq_host, h.scalar, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
  }
}

// The slab factor of level l applied to cnt permuted columns of the workspace Q
// (in place), in the level's arithmetic.
void level_solve(Handle& h, int l, int cnt) {
  auto& L = h.lv[l];
  SkSync sk = h.sk;
  sk.split_waves = L.split_waves;
  sk.tc_persist = L.tc_mode != 2;
  if (L.prec == 4) {
    if (L.tc_mode == 1)
      CK(sn_solve_cplx_f16_cc(L.fac->dch, static_cast<float2*>(h.sQ), static_cast<float2*>(h.sZ),
                              static_cast<float2*>(h.sU), cnt, h.ld_slab, h.stream));
    else
      CK(sn_solve_cplx_f16(L.fac->dch, static_cast<float2*>(h.sQ), static_cast<float2*>(h.sZ),
                           static_cast<float2*>(h.sU), static_cast<float2*>(h.sP), h.tcP, h.tcB, cnt, h.ld_slab, sk,
                           h.stream));
  } else if (L.prec == 3 && L.tc_mode == 1) {
    CK(sn_solve_cplx_bf16_cc(L.fac->dcb, static_cast<float2*>(h.sQ), static_cast<float2*>(h.sZ),
                             static_cast<float2*>(h.sU), cnt, h.ld_slab, h.stream));
  } else if (L.prec == 3) {
    CK(sn_solve_cplx_bf16(L.fac->dcb, static_cast<float2*>(h.sQ), static_cast<float2*>(h.sZ),
                          static_cast<float2*>(h.sU), static_cast<float2*>(h.sP), h.tcP, h.tcB, cnt, h.ld_slab, sk,
                          h.stream));
  } else if (L.prec == 1) {
    if (h.prob.degree == 0)
      CK(sn_solve_realf(L.fac->drf, static_cast<float*>(h.sQ), static_cast<float*>(h.sZ), static_cast<float*>(h.sU),
                        static_cast<float*>(h.sP), cnt, h.ld_slab, sk, h.stream));
    else
      CK(sn_solve_cplxf(L.fac->dcf, static_cast<float2*>(h.sQ), static_cast<float2*>(h.sZ),
                        static_cast<float2*>(h.sU), static_cast<float2*>(h.sP), cnt, h.ld_slab, sk, h.stream));
  } else if (h.prob.degree == 0) {
    if (L.prec == 2)
      CK(sn_solve_real_df(L.fac->drd, static_cast<double*>(h.sQ), static_cast<double*>(h.sZ),
                          static_cast<double*>(h.sU), static_cast<double*>(h.sP), cnt, h.ld_slab, sk, h.stream));
    else
      CK(sn_solve_real(L.fac->dr, static_cast<double*>(h.sQ), static_cast<double*>(h.sZ), static_cast<double*>(h.sU),
                       static_cast<double*>(h.sP), cnt, h.ld_slab, sk, h.stream));
  } else {
    if (L.prec == 2)
      CK(sn_solve_cplx_df(L.fac->dcd, static_cast<double2*>(h.sQ), static_cast<double2*>(h.sZ),
                          static_cast<double2*>(h.sU), static_cast<double2*>(h.sP), cnt, h.ld_slab, sk, h.stream));
    else
      CK(sn_solve_cplx(L.fac->dc, static_cast<double2*>(h.sQ), static_cast<double2*>(h.sZ),
                       static_cast<double2*>(h.sU), static_cast<double2*>(h.sP), cnt, h.ld_slab, sk, h.stream));
  }
}

// Slab solve on slabs [slab0, slab0+cnt) of src (row length src_ld doubles) into dst
// (row length dst_ld) at slab dst0: mode 0 assign, mode 1 dst += omega * A^{-1} src.
void op_slab_cols(Handle& h, int l, const double* src, int src_ld, int slab0, int cnt, double* dst, int dst_ld,
                  int dst0, double omega, int mode) {
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  const double inv_tau = 1.0 / L.tau;
  const double2 c0 = make_double2(h.c0.x * inv_tau, h.c0.y * inv_tau);
  const double2 c1 = make_double2(h.c1.x * inv_tau, h.c1.y * inv_tau);
  if (L.prec == 1 || L.prec == 3 || L.prec == 4) {   // FP32 workspace
    if (h.prob.degree == 0) {
      float* Q = static_cast<float*>(h.sQ);
      CK(slab_pre_dg0f(src, src_ld, slab0, cnt, L.fac->drf.iperm, S.ne, Q, h.ld_slab, h.stream));
      level_solve(h, l, cnt);
      CK(slab_post_dg0f(Q, h.ld_slab, L.fac->drf.iperm, S.ne, dst, dst_ld, dst0, cnt, omega, mode, h.stream));
    } else {
      const int32_t* ip = L.prec == 3 ? L.fac->dcb.iperm : L.prec == 4 ? L.fac->dch.iperm : L.fac->dcf.iperm;
      float2* Q = static_cast<float2*>(h.sQ);
      CK(slab_pre_dg1f(src, src_ld, slab0, cnt, ip, S.ne, c0, c1, Q, h.ld_slab, h.stream));
      // FP16 operands: every column scaled into [1, 2) first (the solve is linear per column)
      if (L.prec == 4) CK(col_scale(Q, S.ne, cnt, h.ld_slab, h.colmax, h.stream));
      level_solve(h, l, cnt);
      if (L.prec == 4) CK(col_unscale(Q, S.ne, cnt, h.ld_slab, h.colmax, h.stream));
      CK(slab_post_dg1f(Q, h.ld_slab, ip, S.ne, h.s1, dst, dst_ld, dst0, cnt, omega, mode, h.stream));
    }
    return;
  }
  if (h.prob.degree == 0) {
    double* Q = static_cast<double*>(h.sQ);
    const int32_t* ip = L.prec == 2 ? L.fac->drd.iperm : L.fac->dr.iperm;
    CK(slab_pre_dg0(src, src_ld, slab0, cnt, ip, S.ne, Q, h.ld_slab, h.stream));
    level_solve(h, l, cnt);
    CK(slab_post_dg0(Q, h.ld_slab, ip, S.ne, dst, dst_ld, dst0, cnt, omega, mode, h.stream));
  } else {
    double2* Q = static_cast<double2*>(h.sQ);
    const int32_t* ip = L.prec == 2 ? L.fac->dcd.iperm : L.fac->dc.iperm;
    CK(slab_pre_dg1(src, src_ld, slab0, cnt, ip, S.ne, c0, c1, Q, h.ld_slab, h.stream));
    level_solve(h, l, cnt);
    CK(slab_post_dg1(Q, h.ld_slab, ip, S.ne, h.s1, dst, dst_ld, dst0, cnt, omega, mode, h.stream));
  }
}

double* level_r(Handle& h, int l) { return l == 0 ? h.r0 : h.lv[l].r; }

void op_smooth_S(Handle& h, int l, const double* f, double* x) {
  auto& L = h.lv[l];
  double* r = level_r(h, l);
  op_residual(h, l, f, x, r, nullptr);
  const int ld = L.N_t * L.B * h.q;
  op_slab_cols(h, l, r, ld, 0, L.N_t * L.B, x, ld, 0, h.opt.omega, 1);
}

void op_grad_T(Handle& h, int l, const double* r, double* y) {
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  CK(grad_T(CsrView{S.nn, S.gt_rowptr, S.gt_col}, S.gt_sign_d, r, y, L.N_t * L.B * h.q, h.stream));
}

void op_nodal_solve(Handle& h, int l, const double* y, double* z) {
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  const int ncols = L.N_t * L.B * h.q;
  if (h.opt.nodal_solve == 0) {
    CK(gather_perm(y, ncols, S.nf->kn.iperm, S.nn, h.nQ, h.ld_nod, h.stream));
    if (h.nodal_prec == 1) {
      // FP32 (a preconditioner step of the mixed-precision modes): float views of the
      // double workspaces
      float* Qf = reinterpret_cast<float*>(h.nQ);
      CK(gather_perm_f(y, ncols, S.nf->kn.iperm, S.nn, Qf, h.ld_nod, h.stream));
      CK(sn_solve_realf(S.nf->kn_f, Qf, reinterpret_cast<float*>(h.nZ), reinterpret_cast<float*>(h.nU),
                        reinterpret_cast<float*>(h.nP), ncols, h.ld_nod, h.sk, h.stream));
      CK(scatter_perm_f(Qf, h.ld_nod, S.nf->kn.iperm, S.nn, z, ncols, h.stream));
      return;
    }
    if (h.nodal_prec == 2)
      CK(sn_solve_real_df(S.nf->kn_df, h.nQ, h.nZ, h.nU, h.nP, ncols, h.ld_nod, h.sk, h.stream));
    else
      CK(sn_solve_real(S.nf->kn, h.nQ, h.nZ, h.nU, h.nP, ncols, h.ld_nod, h.sk, h.stream));
    CK(scatter_perm(h.nQ, h.ld_nod, S.nf->kn.iperm, S.nn, z, ncols, h.stream));
  } else {
    // damped Jacobi from z = 0, ping-pong through the nodal workspace
    const int64_t n = (int64_t)S.nn * ncols;
    CK(vec_fill(z, n, 0.0, h.stream));
    CsrView kv{S.nn, S.kn_rowptr, S.kn_col};
    for (int it = 0; it < h.opt.nodal_jacobi_sweeps; ++it) {
      CK(nodal_jacobi(kv, S.kn_val, S.kn_dinv, y, z, h.nQ, ncols, 2.0 / 3.0, h.stream));
      CK(vec_copy(h.nQ, z, n, h.stream));
    }
  }
}

void op_time_integrate(Handle& h, int l, const double* z, double* w) {
  auto& L = h.lv[l];
  // each problem's slabs of a node are one contiguous segment: nn * B independent scans
  CK(time_integrate(z, w, h.space[L.s].nn * L.B, L.N_t, h.prob.degree, h.stream));
}

void op_grad_add(Handle& h, int l, const double* w, double* x) {
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  CK(grad_add(S.gtail_d, S.ghead_d, S.ne, w, x, L.N_t * L.B * h.q, h.stream));
}

void op_correct_A(Handle& h, int l, const double* f, double* x) {
  double* r = level_r(h, l);
  op_residual(h, l, f, x, r, nullptr);
  op_grad_T(h, l, r, h.ny);
  op_nodal_solve(h, l, h.ny, h.nz);
  op_time_integrate(h, l, h.nz, h.nw);
  op_grad_add(h, l, h.nw, x);
}

bool space_coarsened(Handle& h, int l) { return h.lv[l + 1].s != h.lv[l].s; }

void op_restrict(Handle& h, int l, const double* r, double* rc) {
  auto& L = h.lv[l];
  auto& Sf = h.space[L.s];
  const int Nc = h.lv[l + 1].N_t;
  if (space_coarsened(h, l)) {   // (never on a ragged batch: checked at setup)
    CK(time_restrict(r, h.tmp_fine, Sf.ne * L.B, Nc, h.prob.degree, h.stream));
    CK(csr_spmm(CsrView{Sf.PxT.nrows, Sf.pxt_rowptr, Sf.pxt_col}, Sf.pxt_val, h.tmp_fine, rc, Nc * L.B * h.q, 0,
                h.stream));
  } else {
    // the coarse level's first L.B problems of every edge row are this level's problems
    CK(time_restrict(r, rc, Sf.ne * L.B, Nc, h.prob.degree, h.stream, L.B, h.lv[l + 1].B));
  }
}

void op_prolong_add(Handle& h, int l, const double* ec, double* x) {
  auto& L = h.lv[l];
  auto& Sf = h.space[L.s];
  const int Nc = h.lv[l + 1].N_t;
  if (space_coarsened(h, l)) {
    CK(csr_spmm(CsrView{Sf.Px.nrows, Sf.px_rowptr, Sf.px_col}, Sf.px_val, ec, h.tmp_fine, Nc * L.B * h.q, 0,
                h.stream));
    CK(time_prolong_add(h.tmp_fine, x, Sf.ne * L.B, Nc, h.prob.degree, h.stream));
  } else {
    CK(time_prolong_add(ec, x, Sf.ne * L.B, Nc, h.prob.degree, h.stream, L.B, h.lv[l + 1].B));
  }
}

void op_coarse_solve(Handle& h, const double* f, double* x) {
  const int l = (int)h.lv.size() - 1;
  auto& L = h.lv[l];
  auto& S = h.space[L.s];
  const int ld = L.N_t * L.B * h.q;
  if (L.N_t == 1) {   // one slab per problem: one solve over the batch
    op_slab_cols(h, l, f, ld, 0, L.B, x, ld, 0, 1.0, 0);
    return;
  }
  for (int n = 0; n < L.N_t; ++n) {
    CK(history_rhs(view(S), S.Mv, f, x, h.g1, L.N_t, n, h.prob.degree, h.stream));
    op_slab_cols(h, l, h.g1, h.q, 0, 1, x, ld, n, 1.0, 0);
  }
}

// Hybrid smoother of Section 4 on level l: the option's S/A product (pre-smoother:
// right to left as a matrix product, post-smoother: the same factors in reverse), or
// S^nu A S^nu.
void op_smooth(Handle& h, int l, const double* f, double* x, int nu, bool post) {
  const char* pat = h.opt.smoother;
  const int np = (int)strnlen(pat, sizeof(h.opt.smoother));
  if (np > 0) {
    for (int i = 0; i < np; ++i) {
      const char op = pat[post ? i : np - 1 - i];
      if (op == 'S') op_smooth_S(h, l, f, x);
      else op_correct_A(h, l, f, x);
    }
    return;
  }
  for (int k = 0; k < nu; ++k) op_smooth_S(h, l, f, x);
  if (h.opt.use_A) op_correct_A(h, l, f, x);
  for (int k = 0; k < nu; ++k) op_smooth_S(h, l, f, x);
}

void op_vcycle(Handle& h, int l, const double* f, double* x) {
  if (l == (int)h.lv.size() - 1) {
    op_coarse_solve(h, f, x);
    return;
  }
  op_smooth(h, l, f, x, h.opt.nu_pre, false);
  double* r = level_r(h, l);
  op_residual(h, l, f, x, r, nullptr);
  auto& C = h.lv[l + 1];
  op_restrict(h, l, r, C.f);
  if (C.B == h.lv[l].B) {
    CK(vec_fill(C.x, C.len, 0.0, h.stream));
  } else {   // ragged: the coarse level's own problems keep their iterates
    const int cq = C.N_t * h.q;
    CK(zero_cols(C.x, h.space[C.s].ne, cq * C.B, 0, cq * h.lv[l].B, h.stream));
  }
  op_vcycle(h, l + 1, C.f, C.x);
  op_prolong_add(h, l, C.x, x);
  op_smooth(h, l, f, x, h.opt.nu_post, true);
}

// ---- ragged batches: the caller's rows hold problem b at columns poff[b] .. poff[b] +
// pnt[b] q; its finest level is level pent[b], where it has slot pslot[b] (the level's rows
// hold B problems of N_t q columns each).  Runs of problems with consecutive columns on both
// sides move as one strided copy.
template <typename Fn>
void ragged_runs(const Handle& h, Fn fn) {
  int b = 0;
  while (b < h.B) {
    int e = b + 1;
    while (e < h.B && h.pent[e] == h.pent[b] && h.pslot[e] == h.pslot[e - 1] + 1 &&
           h.poff[e] == h.poff[e - 1] + (int64_t)h.pnt[e - 1] * h.q)
      ++e;
    fn(b, e);
    b = e;
  }
}

// caller's vector -> the level vectors (which = 0: f, 1: x)
void ragged_in(Handle& h, const double* user, int which) {
  ragged_runs(h, [&](int b, int e) {
    auto& L = h.lv[h.pent[b]];
    const int64_t seg = (int64_t)L.N_t * h.q;
    double* dst = (which ? L.x : L.f) + h.pslot[b] * seg;
    CK(cudaMemcpy2DAsync(dst, L.B * seg * sizeof(double), user + h.poff[b], h.prow * sizeof(double),
                         (e - b) * seg * sizeof(double), h.space[0].ne, cudaMemcpyDeviceToDevice, h.stream));
  });
}

// the level vectors' x -> caller's vector
void ragged_out(Handle& h, double* user) {
  ragged_runs(h, [&](int b, int e) {
    auto& L = h.lv[h.pent[b]];
    const int64_t seg = (int64_t)L.N_t * h.q;
    CK(cudaMemcpy2DAsync(user + h.poff[b], h.prow * sizeof(double), L.x + h.pslot[b] * seg,
                         L.B * seg * sizeof(double), (e - b) * seg * sizeof(double), h.space[0].ne,
                         cudaMemcpyDeviceToDevice, h.stream));
  });
}

// Sum of the squared residuals of every problem on its own finest level (f and x already
// in the level vectors): the level's residual over all its slots, the sums of squares of
// the slots of the problems that start there (blocking).
double ragged_res_norm_sq(Handle& h) {
  double total = 0.0;
  std::vector<double> sq(h.B);
  for (size_t l = 0; l < h.lv.size(); ++l) {
    auto& L = h.lv[l];
    const int first = l > 0 ? h.lv[l - 1].B : 0;
    if (L.B == first) continue;
    double* r = level_r(h, (int)l);
    op_residual(h, (int)l, L.f, L.x, r, nullptr, true);
    CK(batch_norms_sq(r, h.space[L.s].ne, L.B, L.N_t * h.q, h.bn_partial, h.bn_out, h.stream));
    CK(cudaMemcpyAsync(sq.data(), h.bn_out, L.B * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
    for (int b = first; b < L.B; ++b) total += sq[b];
  }
  return total;
}

// One V-cycle of every problem of a ragged batch: each problem's load and iterate are
// copied into its slot on its own finest level, the V-cycle runs from level 0 (a level's
// smoothing covers every problem on it, the restriction fills the descending problems'
// slots of the coarser level, whose own problems keep their load and iterate), and the
// iterates are copied back.  In correction form (residual_prec 1) every problem's slot
// first receives its residual in place of its load and a zero iterate, and the caller's x
// gains the correction.
void ragged_vcycle(Handle& h, const double* f, double* x) {
  ragged_in(h, f, 0);
  ragged_in(h, x, 1);
  if (h.res32) {
    for (size_t l = 0; l < h.lv.size(); ++l) {
      auto& L = h.lv[l];
      const int first = l > 0 ? h.lv[l - 1].B : 0;
      if (L.B == first) continue;
      double* r = level_r(h, (int)l);
      op_residual(h, (int)l, L.f, L.x, r, nullptr, true);
      const int64_t seg = (int64_t)L.N_t * h.q;
      const int64_t pitch = L.B * seg * sizeof(double);
      CK(cudaMemcpy2DAsync(L.f + first * seg, pitch, r + first * seg, pitch, (L.B - first) * seg * sizeof(double),
                           h.space[L.s].ne, cudaMemcpyDeviceToDevice, h.stream));
      CK(zero_cols(L.x, h.space[L.s].ne, (int)(L.B * seg), (int)(first * seg), (int)((L.B - first) * seg), h.stream));
    }
    op_vcycle(h, 0, h.lv[0].f, h.lv[0].x);
    ragged_out(h, h.corr_e);
    CK(vec_add(h.corr_e, x, h.user_len, h.stream));
    return;
  }
  op_vcycle(h, 0, h.lv[0].f, h.lv[0].x);
  ragged_out(h, x);
}

// The finest-level V-cycle x <- x + V(f - L x).  With residual_prec 1 it runs in
// correction form: r = f - L x (outer, double-float), e = V(r) from e = 0 with FP32
// residuals inside (their rounding is relative to r, which shrinks as x converges),
// x += e; the same iteration in exact arithmetic, since a V-cycle is affine in (f, x).
void op_vcycle_top(Handle& h, const double* f, double* x) {
  if (h.ragged) {
    ragged_vcycle(h, f, x);
    return;
  }
  if (!h.res32) {
    op_vcycle(h, 0, f, x);
    return;
  }
  const int64_t len = h.lv[0].len;
  op_residual(h, 0, f, x, h.corr_r, nullptr, true);
  CK(vec_fill(h.corr_e, len, 0.0, h.stream));
  op_vcycle(h, 0, h.corr_r, h.corr_e);
  CK(vec_add(h.corr_e, x, len, h.stream));
}

// One V-cycle on the finest level.  With use_graph and a non-default stream the
// fixed launch sequence is captured once per (f, x) pair and replayed.
void run_vcycle(Handle& h, const double* f, double* x) {
  if (!h.opt.use_graph || h.stream == nullptr) {
    op_vcycle_top(h, f, x);
    return;
  }
  if (!h.graph_exec || h.graph_f != f || h.graph_x != x) {
    if (h.graph_exec) {
      CK(cudaGraphExecDestroy(h.graph_exec));
      h.graph_exec = nullptr;
    }
    const int64_t l0 = launch_count();
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
    try {
      op_vcycle_top(h, f, x);
    } catch (...) {
      cudaStreamEndCapture(h.stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    CK(cudaStreamEndCapture(h.stream, &g));
    h.graph_launches = launch_count() - l0;
    count_launches(-h.graph_launches);     // counted when replayed
    cudaError_t e = cudaGraphInstantiate(&h.graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw CudaError{e, "cudaGraphInstantiate"};
    h.graph_f = f;
    h.graph_x = x;
  }
  CK(cudaGraphLaunch(h.graph_exec, h.stream));
  count_launches(h.graph_launches);
}

// l2 norm of a caller's vector (h.user_len doubles: the finest level, or a ragged batch's
// rows), deterministic, blocking
double f_norm(Handle& h, const double* f) {
  double v = 0.0;
  CK(norm2_sq(f, h.user_len, h.partial, h.scalar, h.stream));
  CK(cudaMemcpyAsync(&v, h.scalar, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  return std::sqrt(v);
}

// ---------------------------------------------------------------- setup
// Leaf size of the slab matrices' nested dissection.  The FP64 / FP32 / double-float
// solves are bound by arithmetic, so small leaves (least fill) win; the BF16 tensor-core
// solve is bound by the latency of its dependent tree depths, so it takes large leaves
// (a shallower tree) at the price of more fill.
int nd_leaf_of(const st_mg_options& o) {
  if (o.nd_leaf > 0) return o.nd_leaf;
  return (o.slab_prec == 3 || o.slab_prec == 4) ? 512 : 64;
}

// smoother pattern: NUL-terminated within the field, letters S and A only
bool valid_pattern(const char (&p)[16]) {
  const size_t n = strnlen(p, sizeof(p));
  if (n >= sizeof(p)) return false;
  for (size_t i = 0; i < n; ++i)
    if (p[i] != 'S' && p[i] != 'A') return false;
  return true;
}

int do_setup(const st_mg_problem* pr, const st_mg_options* op, void* stream, st_mg_t* out, bool host_only) {
  if (!pr || !op || !out) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const st_mg_mesh* gm = pr->mesh;
  const int n = gm ? 0 : pr->n_cube, nsl = pr->n_space_levels;
  if ((!gm && n < 2) || nsl < 1 || pr->N_t < 1 || !(pr->T > 0) || (pr->degree != 0 && pr->degree != 1) || !pr->nu ||
      !pr->sigma)
    return fail(ST_MG_ERR_INVALID_ARG, "invalid problem (n_cube >= 2, n_space_levels >= 1, N_t >= 1, T > 0, degree 0|1)");
  if (pr->bc != 0 && pr->bc != 1) return fail(ST_MG_ERR_INVALID_ARG, "bc must be 0 (Dirichlet) or 1 (Neumann)");
  if (gm) {
    if (gm->n_vert < 4 || gm->n_tet < 1 || !gm->xyz || !gm->tet || gm->n_refine < 0 || gm->n_refine > 8 ||
        nsl > gm->n_refine + 1 || ((int64_t)gm->n_tet << (3 * gm->n_refine)) > ((int64_t)1 << 28))
      return fail(ST_MG_ERR_INVALID_ARG,
                  "invalid mesh (n_vert >= 4, n_tet >= 1, 0 <= n_refine <= 8, n_tet 8^n_refine <= 2^28, "
                  "n_space_levels <= n_refine + 1)");
  } else if ((n >> (nsl - 1)) < 2 || (n % (1 << (nsl - 1))) != 0) {
    return fail(ST_MG_ERR_INVALID_ARG, "n_cube must be divisible by 2^(n_space_levels-1) with coarsest >= 2");
  }
  if (!(op->omega > 0) || op->nu_pre < 0 || op->nu_post < 0 || op->min_coarse_slabs < 1 || op->max_levels < 0 ||
      op->coarsen < 0 || op->coarsen > 2 || (op->nodal_solve != 0 && op->nodal_solve != 1) ||
      op->nodal_jacobi_sweeps < 0 || op->slab_prec < 0 || op->slab_prec > 4 || (op->slab_prec >= 3 && pr->degree != 1) ||
      op->persistent_split < 0 || op->persistent_split > 2 || !valid_pattern(op->smoother) ||
      (op->autotune != 0 && op->autotune != 1) || op->nd_leaf < 0 || op->nd_leaf > 4096 ||
      op->split_k < 0 || op->split_k > 1024 || (op->split_k % 16) != 0 || op->tc_split_k < 0 ||
      op->tc_split_k > 4096 || (op->tc_split_k % 32) != 0 ||
      (op->residual_prec < -1 || op->residual_prec > 2))
    return fail(ST_MG_ERR_INVALID_ARG, "invalid options");
  const int64_t nt = gm ? ((int64_t)gm->n_tet << (3 * gm->n_refine)) : (int64_t)6 * n * n * n;
  for (int64_t t = 0; t < nt; ++t)
    if (!(pr->nu[t] > 0) || !(pr->sigma[t] > 0) || !std::isfinite(pr->nu[t]) || !std::isfinite(pr->sigma[t]))
      return fail(ST_MG_ERR_INVALID_ARG, "nu and sigma must be positive and finite");

  std::unique_ptr<Handle> h(new Handle());
  Handle& H = *h;
  H.prob = *pr;
  H.opt = *op;
  H.nu.assign(pr->nu, pr->nu + nt);
  H.sigma.assign(pr->sigma, pr->sigma + nt);
  H.prob.nu = H.nu.data();
  H.prob.sigma = H.sigma.data();
  H.prob.mesh = nullptr;   // the caller's mesh and batch_nt are read during this call only
  H.prob.batch_nt = nullptr;
  H.stream = static_cast<cudaStream_t>(stream);
  H.q = pr->degree + 1;
  H.B = pr->n_batch > 1 ? pr->n_batch : 1;
  H.host_only = host_only;
  if (!host_only) {
    CK(cudaGetDevice(&H.device));
    CK(cudaDeviceGetAttribute(&H.n_sm, cudaDevAttrMultiProcessorCount, H.device));
  }

  // ---- space hierarchy (level 0 finest)
  H.space.resize(nsl);
  if (gm) {
    std::vector<TetMesh> chain(gm->n_refine + 1);   // start mesh, refined once, ...
    std::string err;
    if (build_general(gm->n_vert, gm->xyz, gm->n_tet, gm->tet, pr->bc, chain[0], err))
      return fail(ST_MG_ERR_INVALID_ARG, err);
    for (int r = 1; r <= gm->n_refine; ++r) refine_red(chain[r - 1], pr->bc, chain[r]);
    for (int s = 0; s < nsl; ++s) H.space[s].mesh = std::move(chain[gm->n_refine - s]);
  }
  for (int s = 0; s < nsl; ++s) {
    auto& S = H.space[s];
    if (!gm) build_kuhn(n >> s, S.mesh, pr->bc);
    S.ne = (int32_t)S.mesh.int_edges.size();
    S.nn = (int32_t)S.mesh.int_verts.size();
    if (S.ne < 1 || S.nn < 1)
      return fail(ST_MG_ERR_INVALID_ARG, "a space level has no interior edge or no interior vertex (refine more)");
    gradient_pairs(S.mesh, S.gtail, S.ghead);
    // positions that guide the nested-dissection orderings: edge midpoints, vertices
    for (int32_t e : S.mesh.int_edges) {
      double a[3], b[3];
      vertex_xyz(S.mesh, S.mesh.edge_lo[e], a);
      vertex_xyz(S.mesh, S.mesh.edge_hi[e], b);
      S.ecoord.rx.push_back(0.5 * (a[0] + b[0]));
      S.ecoord.ry.push_back(0.5 * (a[1] + b[1]));
      S.ecoord.rz.push_back(0.5 * (a[2] + b[2]));
    }
    for (int32_t v : S.mesh.int_verts) {
      double a[3];
      vertex_xyz(S.mesh, v, a);
      S.ncoord.rx.push_back(a[0]); S.ncoord.ry.push_back(a[1]); S.ncoord.rz.push_back(a[2]);
    }
  }
  assemble_edge(H.space[0].mesh, H.nu.data(), H.sigma.data(), H.space[0].M, H.space[0].K);
  assemble_nodal(H.space[0].mesh, H.sigma.data(), H.space[0].Kn);
  for (int s = 0; s + 1 < nsl; ++s) {
    auto& F = H.space[s];
    auto& C = H.space[s + 1];
    edge_prolongation(C.mesh, F.mesh, F.Px);
    F.PxT = csr_transpose(F.Px);
    C.M = csr_galerkin(F.Px, F.M);
    C.K = csr_galerkin(F.Px, F.K);
    C.Kn = nodal_from_gradient(C.M, C.gtail, C.ghead, C.nn);
    if (C.M.col != C.K.col) return fail(ST_MG_ERR_NUMERIC, "coarse M and K patterns differ");
  }
  for (auto& S : H.space) {
    S.GT = csr_transpose(gradient_csr(S.gtail, S.ghead, S.nn));
    S.gt_sign.resize(S.GT.val.size());
    for (size_t q = 0; q < S.GT.val.size(); ++q) S.gt_sign[q] = S.GT.val[q] > 0 ? 1 : -1;
  }

  // ---- time hierarchy (eq. CoarseningRule).  Kuhn: h_T = sqrt(3)/n for every tet;
  // general meshes: h_T = the longest edge of the level-s ancestor of each finest tet
  // (tet t >> 3s), the minimum taken over the finest tets.
  double min_ratio = INFINITY;
  for (int64_t t = 0; t < nt; ++t) min_ratio = std::min(min_ratio, H.nu[t] / H.sigma[t]);
  std::vector<double> min_ratio_h2(nsl, INFINITY);
  if (gm)
    for (int s = 0; s < nsl; ++s) {
      const std::vector<double> h = longest_edges(H.space[s].mesh);
      for (int64_t t = 0; t < nt; ++t)
        min_ratio_h2[s] = std::min(min_ratio_h2[s], H.nu[t] / (H.sigma[t] * h[t >> (3 * s)] * h[t >> (3 * s)]));
    }
  {
    Handle::Level L0;
    L0.s = 0;
    L0.N_t = pr->N_t;
    L0.tau = pr->T / pr->N_t;
    H.lv.push_back(L0);
  }
  const int cap = op->max_levels > 0 ? op->max_levels : 1 << 20;
  while ((int)H.lv.size() < cap) {
    const auto& cur = H.lv.back();
    if (cur.N_t <= op->min_coarse_slabs || (cur.N_t % 2) != 0) break;
    const bool can_space = cur.s + 1 < nsl;
    bool coarsen = false;
    if (op->coarsen == 0) {
      if (gm) {
        coarsen = can_space && (min_ratio_h2[cur.s] * cur.tau >= op->lambda_crit);
      } else {
        const double hT = std::sqrt(3.0) / (double)(n >> cur.s);
        coarsen = can_space && (min_ratio * cur.tau / (hT * hT) >= op->lambda_crit);
      }
    } else if (op->coarsen == 2) {
      coarsen = can_space && H.lv.size() == 1;
    }
    Handle::Level C;
    C.s = cur.s + (coarsen ? 1 : 0);
    C.N_t = cur.N_t / 2;
    C.tau = cur.tau * 2.0;
    H.lv.push_back(C);
  }

  // ---- DG(1) complex transformation: M_t^{-1} K_t = S diag(mu, conj mu) S^{-1},
  // mu tau = 2 + i sqrt2, s_0 = (1, 1 + i sqrt2); row 0 of S^{-1} M_t^{-1} is
  // (1/2 + i/(2 sqrt2), -3i/(2 sqrt2)) / tau.
  const double r2 = std::sqrt(2.0);
  H.c0 = make_double2(0.5, 0.5 / r2);
  H.c1 = make_double2(0.0, -1.5 / r2);
  H.s1 = make_double2(1.0, r2);

  // slab_prec 1 (FP32) and 3 (BF16) leave the coarsest level in FP64; slab_prec 2
  // (double-float, FP64-accurate) applies to every level
  for (size_t l = 0; l < H.lv.size(); ++l)
    H.lv[l].prec = ((op->slab_prec == 1 || op->slab_prec >= 3) && l + 1 == H.lv.size()) ? 0 : op->slab_prec;
  H.res32 = op->residual_prec == 1;
  H.sk_k = op->split_k > 0 ? op->split_k : kSkK;
  H.tc_k = op->tc_split_k > 0 ? op->tc_split_k : kTcSplitK;
  H.df_residual = op->residual_prec == 2 || op->residual_prec == 1 || (op->residual_prec < 0 && op->slab_prec != 0);
  H.nodal_prec = op->slab_prec == 0 ? 0 : op->slab_prec == 2 ? 2 : 1;

  // ---- factor cache: take every factor an earlier handle left resident
  H.use_cache = op->factor_cache != 0 && !host_only;
  auto& lkey = H.lkey;
  auto& skey = H.skey;
  lkey.assign(H.lv.size(), std::string());
  skey.assign(H.space.size(), std::string());
  if (H.use_cache) {
    uint64_t mh = fnv1a(1469598103934665603ull, &n, sizeof(n));
    mh = fnv1a(mh, &pr->bc, sizeof(pr->bc));
    if (gm) {   // the start mesh and its refinement count
      mh = fnv1a(mh, &gm->n_refine, sizeof(gm->n_refine));
      mh = fnv1a(mh, gm->xyz, (size_t)gm->n_vert * 3 * sizeof(double));
      mh = fnv1a(mh, gm->tet, (size_t)gm->n_tet * 4 * sizeof(int32_t));
    }
    mh = fnv1a(mh, H.nu.data(), H.nu.size() * sizeof(double));
    H.mat_hash = fnv1a(mh, H.sigma.data(), H.sigma.size() * sizeof(double));
    char buf[192];
    for (size_t l = 0; l < H.lv.size(); ++l) {
      const auto& L = H.lv[l];
      std::snprintf(buf, sizeof buf, "slab dev%d n%d s%d deg%d prec%d leaf%d sk%d tc%d tau%a mat%016llx",
                    H.device, n, L.s, pr->degree, L.prec, nd_leaf_of(*op), H.sk_k, H.tc_k, L.tau,
                    (unsigned long long)H.mat_hash);
      lkey[l] = buf;
    }
    for (size_t sl = 0; sl < H.space.size(); ++sl) {
      std::snprintf(buf, sizeof buf, "nodal dev%d n%d s%d np%d sk%d mat%016llx", H.device, n, (int)sl, H.nodal_prec, H.sk_k,
                    (unsigned long long)H.mat_hash);
      skey[sl] = buf;
    }
    auto& C = factor_cache();
    std::lock_guard<std::mutex> g(C.mu);
    for (size_t l = 0; l < H.lv.size(); ++l) {
      auto it = C.map.find(lkey[l]);
      if (it != C.map.end() && it->second.slab) {
        H.lv[l].fac = it->second.slab;
        it->second.last_use = ++C.tick;
        ++C.hits;
      }
    }
    for (size_t sl = 0; sl < H.space.size(); ++sl) {
      auto it = C.map.find(skey[sl]);
      if (it != C.map.end() && it->second.nodal) {
        H.space[sl].nf = it->second.nodal;
        it->second.last_use = ++C.tick;
        ++C.hits;
      }
    }
  }
  // ---- factorisations (all levels concurrently; cached ones skipped)
  const int nthr = hw_threads(op->setup_threads);
  const int leaf = nd_leaf_of(*op);
  std::vector<std::string> errs(H.lv.size() + H.space.size());
  std::vector<int> rcs(errs.size(), 0);
  {
    // one factorisation at a time, each with every thread (tree and front parallelism)
    const int njobs = (int)errs.size();
    const int inner = nthr;
    std::vector<std::thread> jobs;
    std::mutex mu;
    int next = 0;
    auto worker = [&]() {
      for (;;) {
        int j;
        {
          std::lock_guard<std::mutex> g(mu);
          j = next++;
        }
        if (j >= njobs) return;
        if (j < (int)H.lv.size()) {
          auto& L = H.lv[j];
          auto& S = H.space[L.s];
          if (L.fac) continue;
          if (pr->degree == 0) {
            std::vector<double> v(S.M.val.size());
            for (size_t q = 0; q < v.size(); ++q) v[q] = S.M.val[q] + L.tau * S.K.val[q];
            rcs[j] = factor_nd_threads(S.M, v, S.ecoord, leaf, L.fr, errs[j], inner);
          } else {
            const double mr = 2.0 / L.tau, mi = r2 / L.tau;   // mu = (2 + i sqrt2) / tau
            std::vector<cplx> v(S.M.val.size());
            for (size_t q = 0; q < v.size(); ++q) v[q] = cplx(S.K.val[q] + mr * S.M.val[q], mi * S.M.val[q]);
            rcs[j] = factor_nd_threads(S.M, v, S.ecoord, leaf, L.fc, errs[j], inner);
          }
        } else {
          auto& S = H.space[j - H.lv.size()];
          if (S.nf) continue;
          rcs[j] = factor_nd_threads(S.Kn, S.Kn.val, S.ncoord, 48, S.knF, errs[j], inner);
        }
      }
    };
    jobs.emplace_back(worker);
    for (auto& t : jobs) t.join();
  }
  for (size_t j = 0; j < rcs.size(); ++j)
    if (rcs[j]) return fail(rcs[j] == 6 ? ST_MG_ERR_NUMERIC : ST_MG_ERR_INVALID_ARG, "factorisation: " + errs[j]);
  if (H.B > 1 && H.lv.back().N_t != 1)
    return fail(ST_MG_ERR_INVALID_ARG, "n_batch > 1 needs a hierarchy that coarsens time to one slab "
                                       "(N_t a power of two, no max_levels cap)");
  for (auto& L : H.lv) L.B = H.B;
  if (H.B > 1 && pr->batch_nt) {
    // ragged batch: problem b enters the time hierarchy at the level whose slab count is
    // its own (the steps agree there: T / pnt[b]); the finer levels do not hold it
    H.pnt.assign(pr->batch_nt, pr->batch_nt + H.B);
    H.ragged = false;
    for (int b = 0; b < H.B; ++b) {
      const int nt = H.pnt[b];
      if (nt < 1 || nt > pr->N_t || (pr->N_t % nt) != 0 || ((pr->N_t / nt) & (pr->N_t / nt - 1)) != 0)
        return fail(ST_MG_ERR_INVALID_ARG, "batch_nt[b] must be N_t divided by a power of two");
      if (nt != pr->N_t) H.ragged = true;
    }
  }
  if (H.ragged) {
    for (const auto& L : H.lv)
      if (L.s != 0)
        return fail(ST_MG_ERR_INVALID_ARG, "a ragged batch needs time-only coarsening (coarsen = 1 or one space "
                                           "level)");
    H.pent.assign(H.B, 0);
    H.pslot.assign(H.B, 0);
    for (size_t l = 0; l < H.lv.size(); ++l) {
      auto& L = H.lv[l];
      int count = l > 0 ? H.lv[l - 1].B : 0;
      for (int b = 0; b < H.B; ++b)
        if (H.pnt[b] == L.N_t) {
          H.pent[b] = (int)l;
          H.pslot[b] = count++;
        }
      L.B = count;
    }
    H.poff.assign(H.B, 0);
    int64_t off = 0;
    for (int b = 0; b < H.B; ++b) {
      H.poff[b] = off;
      off += (int64_t)H.pnt[b] * H.q;
    }
    H.prow = off;
  }
  for (auto& L : H.lv) L.len = (int64_t)H.space[L.s].ne * L.N_t * H.q * L.B;
  H.user_len = H.ragged ? (int64_t)H.space[0].ne * H.prow : H.lv[0].len;
  H.pending_upload = !host_only;
  *out = h.release();
  return ST_MG_OK;
}

// Tiled / split-K threshold per time level: each candidate is timed on two slab solves
// of the level's full column count (after one untimed solve), on the handle's stream,
// with the slab workspace as input (the values do not affect the time).  Levels whose
// solve runs split-K throughout (few right-hand sides) have nothing to choose.
void autotune_split(Handle& H) {
  const int cand[] = {0, 1, 2, 4, 8, 16, 32};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (size_t l = 0; l < H.lv.size(); ++l) {
    auto& L = H.lv[l];
    const int cnt = L.N_t * L.B;
    const int skinny_max = (H.prob.degree == 0) ? kSkMaxRhsR : kSkMaxRhsC;
    if (cnt <= skinny_max) continue;
    float best = 0.f;
    int best_w = L.split_waves;
    for (int w : cand) {
      L.split_waves = w;
      level_solve(H, (int)l, cnt);
      CK(cudaEventRecord(e0, H.stream));
      for (int rep = 0; rep < 2; ++rep) level_solve(H, (int)l, cnt);
      CK(cudaEventRecord(e1, H.stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (best == 0.f || ms < best) {
        best = ms;
        best_w = w;
      }
    }
    L.split_waves = best_w;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timed solves may have left the bounded-wait flag set only through a real timeout
  CK(cudaStreamSynchronize(H.stream));
}

// Device phase of the setup: upload meshes, matrices and factors (taking cache entries
// that appeared since the host phase), size the workspaces.
int setup_device(Handle& H) {
  const st_mg_problem* pr = &H.prob;
  const st_mg_options* op = &H.opt;
  const auto& lkey = H.lkey;
  const auto& skey = H.skey;
  if (H.use_cache) {
    for (size_t l = 0; l < H.lv.size(); ++l)
      if (!H.lv[l].fac)
        if (auto f = cache_recheck<SlabFactor>(lkey[l])) H.lv[l].fac = f;
    for (size_t sl = 0; sl < H.space.size(); ++sl)
      if (!H.space[sl].nf)
        if (auto f = cache_recheck<NodalFactor>(skey[sl])) H.space[sl].nf = f;
  }
  for (auto& S : H.space) {
    S.rowptr = H.upload(S.M.rowptr);
    S.col = H.upload(S.M.col);
    S.Mv = H.upload(S.M.val);
    S.gtail_d = H.upload(S.gtail);
    S.ghead_d = H.upload(S.ghead);
    S.gt_rowptr = H.upload(S.GT.rowptr);
    S.gt_col = H.upload(S.GT.col);
    S.gt_sign_d = H.upload(S.gt_sign);
    S.kn_rowptr = H.upload(S.Kn.rowptr);
    S.kn_col = H.upload(S.Kn.col);
    S.kn_val = H.upload(S.Kn.val);
    std::vector<double> dinv(S.nn);
    for (int32_t v = 0; v < S.nn; ++v)
      for (int64_t q = S.Kn.rowptr[v]; q < S.Kn.rowptr[v + 1]; ++q)
        if (S.Kn.col[q] == v) dinv[v] = 1.0 / S.Kn.val[q];
    S.kn_dinv = H.upload(dinv);
    if (!S.Px.rowptr.empty()) {
      S.px_rowptr = H.upload(S.Px.rowptr);
      S.px_col = H.upload(S.Px.col);
      S.px_val = H.upload(S.Px.val);
      S.pxt_rowptr = H.upload(S.PxT.rowptr);
      S.pxt_col = H.upload(S.PxT.col);
      S.pxt_val = H.upload(S.PxT.val);
    }
    if (!S.nf) {
      auto N = std::make_shared<NodalFactor>();
      N->mem.n_sm = H.n_sm;
      make_dev_factor(N->mem, S.knF, N->kn, N->kn_lists, H.sk_k, H.tc_k, kSnBmFP64);
      if (H.nodal_prec == 2) make_dev_factor(N->mem, S.knF, N->kn_df, N->kn_df_lists, H.sk_k, H.tc_k);
      if (H.nodal_prec == 1) make_dev_factor(N->mem, S.knF, N->kn_f, N->kn_f_lists, H.sk_k, H.tc_k);
      N->u_rows = N->kn.u_rows;
      N->max_items = N->kn.max_items;
      S.nf = N;
      if (H.use_cache) cache_put(skey[&S - H.space.data()], nullptr, N);
    }
    S.knF = SupernodalFactor<double>();   // host copy no longer needed
  }
  int64_t max_ne = 0, max_u = 0, max_nn = 0, max_un = 0, max_len_fine_tmp = 0, max_items = 0, max_kn_items = 0;
  int64_t max_len = 0;
  for (auto& S : H.space) max_kn_items = std::max<int64_t>(max_kn_items, S.nf->kn.max_items);
  int max_nt = 1;
  for (size_t l = 0; l < H.lv.size(); ++l) {
    auto& L = H.lv[l];
    auto& S = H.space[L.s];
    const size_t nnz = S.M.val.size();
    std::vector<double> a(nnz), b(nnz), c(nnz);
    if (pr->degree == 0) {
      for (size_t q = 0; q < nnz; ++q) { a[q] = S.M.val[q] + L.tau * S.K.val[q]; b[q] = S.M.val[q]; }
      L.v0 = H.upload(a);
      L.v1 = H.upload(b);
      if (H.df_residual) {
        L.p0 = H.upload(convert_pairs<float2>(a));
        L.p1 = H.upload(convert_pairs<float2>(b));
      }
      if (H.res32) {
        L.q0 = H.upload(convert<float>(a));
        L.q1 = H.upload(convert<float>(b));
      }
      if (!L.fac) {
        auto F = std::make_shared<SlabFactor>();
        F->mem.n_sm = H.n_sm;
        if (L.prec == 1) {
          make_dev_factor(F->mem, L.fr, F->drf, F->lists, H.sk_k, H.tc_k);
          F->max_items = F->drf.max_items;
          F->w_bytes = (int64_t)L.fr.W.size() * 4;
        } else if (L.prec == 2) {
          make_dev_factor(F->mem, L.fr, F->drd, F->lists, H.sk_k, H.tc_k);
          F->max_items = F->drd.max_items;
          F->w_bytes = (int64_t)L.fr.W.size() * 8;
        } else {
          make_dev_factor(F->mem, L.fr, F->dr, F->lists, H.sk_k, H.tc_k, kSnBmFP64);
          F->max_items = F->dr.max_items;
          F->w_bytes = (int64_t)L.fr.W.size() * 8;
        }
        F->u_rows = L.fr.u_rows;
        L.fac = F;
        if (H.use_cache) cache_put(lkey[l], F, nullptr);
      }
      L.fr = SupernodalFactor<double>();
      max_items = std::max<int64_t>(max_items, L.fac->max_items);
      max_u = std::max<int64_t>(max_u, L.fac->u_rows);
    } else {
      for (size_t q = 0; q < nnz; ++q) {
        a[q] = S.M.val[q];
        b[q] = L.tau * S.K.val[q];
        c[q] = L.tau * S.K.val[q] / 3.0;
      }
      L.v0 = H.upload(a);
      L.v1 = H.upload(b);
      L.v2 = H.upload(c);
      if (H.df_residual) {
        L.p0 = H.upload(convert_pairs<float2>(a));
        L.p1 = H.upload(convert_pairs<float2>(b));
        L.p2 = H.upload(convert_pairs<float2>(c));
      }
      if (H.res32) {
        L.q0 = H.upload(convert<float>(a));
        L.q1 = H.upload(convert<float>(b));
        L.q2 = H.upload(convert<float>(c));
      }
      if (!L.fac) {
        auto F = std::make_shared<SlabFactor>();
        F->mem.n_sm = H.n_sm;
        if (L.prec == 1) {
          make_dev_factor(F->mem, L.fc, F->dcf, F->lists, H.sk_k, H.tc_k);
          F->max_items = F->dcf.max_items;
          F->w_bytes = (int64_t)L.fc.W.size() * 8;
        } else if (L.prec == 3) {
          make_dev_factor(F->mem, L.fc, F->dcb, F->lists, H.sk_k, H.tc_k);
          build_tc_tiles(F->mem, L.fc, F->dcb, F->lists);
          F->max_items = F->dcb.max_items;
          F->max_tc_items = F->dcb.max_tc_items;
          F->max_stage_tiles = F->dcb.max_stage_tiles;
          F->w_bytes = (int64_t)L.fc.W.size() * 4;
        } else if (L.prec == 4) {
          if (max_abs_entry(L.fc) > 16384.0)
            throw NumericError{"a slab factor entry exceeds the FP16 range kept for slab_prec 4 (|w| > 16384)"};
          make_dev_factor(F->mem, L.fc, F->dch, F->lists, H.sk_k, H.tc_k);
          build_tc_tiles(F->mem, L.fc, F->dch, F->lists);
          F->max_items = F->dch.max_items;
          F->max_tc_items = F->dch.max_tc_items;
          F->max_stage_tiles = F->dch.max_stage_tiles;
          F->w_bytes = (int64_t)L.fc.W.size() * 4;
        } else if (L.prec == 2) {
          make_dev_factor(F->mem, L.fc, F->dcd, F->lists, H.sk_k, H.tc_k);
          F->max_items = F->dcd.max_items;
          F->w_bytes = (int64_t)L.fc.W.size() * 16;
        } else {
          make_dev_factor(F->mem, L.fc, F->dc, F->lists, H.sk_k, H.tc_k, kSnBmFP64);
          F->max_items = F->dc.max_items;
          F->w_bytes = (int64_t)L.fc.W.size() * 16;
        }
        F->u_rows = L.fc.u_rows;
        L.fac = F;
        if (H.use_cache) cache_put(lkey[l], F, nullptr);
      }
      L.fc = SupernodalFactor<cplx>();
      max_items = std::max<int64_t>(max_items, L.fac->max_items);
      max_u = std::max<int64_t>(max_u, L.fac->u_rows);
    }
    L.len = (int64_t)S.ne * L.N_t * H.q * L.B;
    max_len = std::max(max_len, L.len);
    if (l > 0 || H.ragged) {
      L.f = H.dalloc<double>(L.len);
      L.x = H.dalloc<double>(L.len);
      if (l > 0) L.r = H.dalloc<double>(L.len);
    }
    if (l + 1 < H.lv.size() && H.lv[l + 1].s != L.s)
      max_len_fine_tmp = std::max<int64_t>(max_len_fine_tmp, (int64_t)S.ne * H.lv[l + 1].N_t * H.q * H.B);
    max_ne = std::max<int64_t>(max_ne, S.ne);
    max_nn = std::max<int64_t>(max_nn, S.nn);
    max_nt = std::max(max_nt, L.N_t * L.B);
    max_un = std::max<int64_t>(max_un, S.nf->kn.u_rows);
  }
  const size_t esz = pr->degree == 0 ? sizeof(double) : sizeof(double2);
  H.ld_slab = max_nt;
  H.sQ = H.dalloc<char>((int64_t)(max_ne * H.ld_slab * esz));
  H.sZ = H.dalloc<char>((int64_t)(max_ne * H.ld_slab * esz));
  H.sU = H.dalloc<char>((int64_t)(std::max<int64_t>(max_u, 1) * H.ld_slab * esz));
  int64_t df_items = 0, df_kn_items = 0, df_words = 1;   // dataflow split-K solves
  if (op->persistent_split == 2) {
    for (auto& L : H.lv) {
      df_items = std::max(df_items, L.fac->lists.df_items);
      df_words = std::max(df_words, L.fac->lists.df_words);
    }
    for (auto& S : H.space) {
      df_kn_items = std::max(df_kn_items, S.nf->kn_lists.df_items);
      df_words = std::max(df_words, S.nf->kn_lists.df_words);
    }
  }
  {
    const int nbk = pr->degree == 0 ? kSkMaxRhsR : kSkMaxRhsC;
    const int64_t cols = (int64_t)((H.ld_slab + nbk - 1) / nbk) * nbk;
    H.sP = H.dalloc<char>((int64_t)(std::max<int64_t>(std::max<int64_t>(max_items, 1) * cols, df_items * nbk) *
                                    kSkRows * esz));
  }
  H.ld_nod = max_nt * H.q;
  H.nQ = H.dalloc<double>(max_nn * H.ld_nod);
  H.nZ = H.dalloc<double>(max_nn * H.ld_nod);
  H.nU = H.dalloc<double>(std::max<int64_t>(max_un, 1) * H.ld_nod);
  H.nP = H.dalloc<double>(std::max<int64_t>(std::max<int64_t>(max_kn_items, 1) *
                                               ((int64_t)((H.ld_nod + kSkMaxRhsR - 1) / kSkMaxRhsR) * kSkMaxRhsR),
                                           df_kn_items * kSkMaxRhsR) *
                          kSkRows);
  H.ny = H.dalloc<double>(max_nn * H.ld_nod);
  H.nz = H.dalloc<double>(max_nn * H.ld_nod);
  H.nw = H.dalloc<double>(max_nn * H.ld_nod);
  H.tmp_fine = H.dalloc<double>(std::max<int64_t>(max_len_fine_tmp, 1));
  H.g1 = H.dalloc<double>(max_ne * H.q * H.B);
  H.r0 = H.dalloc<double>(H.lv[0].len);
  if (H.df_residual) H.xsplit = H.dalloc<float2>(max_len);
  if (H.res32) {
    H.xf32 = H.dalloc<float>(max_len);
    H.corr_r = H.dalloc<double>(H.lv[0].len);
    H.corr_e = H.dalloc<double>(std::max(H.lv[0].len, H.user_len));
  }
  H.flags = H.dalloc<int>(4);
  CK(cudaMemset(H.flags, 0, 4 * sizeof(int)));
  H.tc_err = H.flags;
  H.sk.bar = op->persistent_split == 1 ? reinterpret_cast<unsigned*>(H.flags + 2) : nullptr;
  if (op->persistent_split == 2) H.sk.df = H.dalloc<unsigned>(df_words);
  H.sk.err = H.flags;
  if (op->slab_prec >= 3) {
    H.colmax = H.dalloc<unsigned>(H.ld_slab);
    int64_t mt = 1;
    for (auto& L : H.lv)
      if (L.prec >= 3) mt = std::max<int64_t>(mt, L.fac->max_tc_items);
    const int64_t gy = (H.ld_slab + kTcCols - 1) / kTcCols;
    H.tcP = H.dalloc<float2>(mt * gy * kSnBM * kTcCols);
    int64_t ms = 1;
    for (auto& L : H.lv)
      if (L.prec >= 3) ms = std::max<int64_t>(ms, L.fac->max_stage_tiles);
    H.tcB = H.dalloc<uint8_t>(ms * gy * kTcTileBytes);
  }
  H.load_b = H.dalloc<double>(H.space[0].ne);
  H.load_c = H.dalloc<double>((int64_t)H.lv[0].N_t * H.q);
  H.bn_partial = H.dalloc<double>(batch_norm_scratch(H.B));
  H.bn_out = H.dalloc<double>(H.B);
  H.partial = H.dalloc<double>(std::max(std::max(1024, 8 * H.n_sm), residual_blocks((int)max_ne)));
  H.scalar = H.dalloc<double>(1);
  // the uploads above ran on the legacy default stream
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  H.pending_upload = false;
  if (op->autotune) autotune_split(H);
  return ST_MG_OK;
}

// A tensor-core block that gave up waiting leaves a flag; report it (blocking read).
int check_tc(Handle& H) {
  if (!H.tc_err) return ST_MG_OK;
  int v = 0;
  CK(cudaMemcpyAsync(&v, H.tc_err, sizeof(int), cudaMemcpyDeviceToHost, H.stream));
  CK(cudaStreamSynchronize(H.stream));
  if (v) {
    // clear the flag and the grid-barrier words a timed-out barrier may have left behind
    CK(cudaMemsetAsync(H.flags, 0, 4 * sizeof(int), H.stream));
    CK(cudaStreamSynchronize(H.stream));
    return fail(ST_MG_ERR_TIMEOUT, "a bounded device wait timed out; results of this call are invalid");
  }
  return ST_MG_OK;
}

template <typename Fn>
int guarded(Fn fn) {
  try {
    return fn();
  } catch (const CudaError& e) {
    return fail(e.e == cudaErrorMemoryAllocation ? ST_MG_ERR_OOM : ST_MG_ERR_CUDA,
                std::string(e.where) + ": " + cudaGetErrorString(e.e));
  } catch (const NumericError& e) {
    return fail(ST_MG_ERR_NUMERIC, e.what);
  } catch (const std::bad_alloc&) {
    return fail(ST_MG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ST_MG_ERR_INVALID_ARG, e.what());
  }
}

int check_dev(st_mg_t h) {
  if (!h) return fail(ST_MG_ERR_INVALID_ARG, "null handle");
  if (h->host_only) return fail(ST_MG_ERR_INVALID_ARG, "handle was built by st_mg_setup_host (no device state)");
  if (h->pending_upload) return fail(ST_MG_ERR_INVALID_ARG, "setup not finished (st_mg_setup_finish)");
  return ST_MG_OK;
}

int check_level(st_mg_t h, int32_t level) {
  if (int rc = check_dev(h)) return rc;
  if (level < 0 || level >= (int32_t)h->lv.size()) return fail(ST_MG_ERR_INVALID_ARG, "level out of range");
  return ST_MG_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_ptrs(std::initializer_list<const void*> ps) {
  for (const void* p : ps) {
    if (!p) return fail(ST_MG_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(p)) return fail(ST_MG_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  }
  return ST_MG_OK;
}

// ||f - L x||^2 of a caller's f and x (every problem on its own finest level for a
// ragged batch), FP64-accurate, blocking
double outer_res_norm_sq(Handle& H, const double* f, const double* x) {
  if (H.ragged) {
    ragged_in(H, f, 0);
    ragged_in(H, x, 1);
    return ragged_res_norm_sq(H);
  }
  double nsq = 0.0;
  op_residual(H, 0, f, x, H.r0, &nsq, true);
  return nsq;
}

int solve_loop(Handle& H, const double* f, double* x, double rtol, int32_t maxit, int32_t* iters, double* rel_res,
               double* history) {
  const double fn = f_norm(H, f);
  const double denom = fn > 0 ? fn : 1.0;
  double nsq = outer_res_norm_sq(H, f, x);
  double rel = std::sqrt(nsq) / denom;
  const double rel0 = rel;
  if (history) history[0] = rel;
  int it = 0;
  int status = ST_MG_OK;
  while (rel > rtol && it < maxit) {
    run_vcycle(H, f, x);
    if (int rc = check_tc(H)) return rc;
    nsq = outer_res_norm_sq(H, f, x);
    rel = std::sqrt(nsq) / denom;
    ++it;
    if (history) history[it] = rel;
    if (!std::isfinite(rel) || rel > 1e3 * std::max(rel0, 1e-300)) {
      status = fail(ST_MG_ERR_DIVERGED, "residual diverged");
      break;
    }
  }
  if (status == ST_MG_OK && rel > rtol) status = fail(ST_MG_ERR_NOT_CONVERGED, "maxit reached");
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  return status;
}

}  // namespace

// Host evaluation of one factor on one right-hand side, in the same forward /
// backward order as the device kernels (setup check on host-only handles).
template <typename T>
void host_factor_apply(const SupernodalFactor<T>& F, std::vector<T>& b) {
  const int n = F.n;
  std::vector<T> q(n), z(n), x(n), U(F.u_rows);
  for (int i = 0; i < n; ++i) q[F.iperm[i]] = b[i];
  for (size_t s = 0; s < F.nodes.size(); ++s) {
    const auto& nd = F.nodes[s];
    const int m = nd.nc + nd.nr;
    std::vector<T> f(m);
    for (int p = 0; p < m; ++p) {
      T v = p < nd.nc ? q[nd.col0 + p] : T(0.0);
      for (int c = 0; c < 2; ++c) {
        const int32_t src = F.gsrc[(F.gather_off[s] + p) * 2 + c];
        if (src >= 0) v = v + U[src];
      }
      f[p] = v;
    }
    const T* W = F.W.data() + nd.w_off;
    for (int r = 0; r < m; ++r) {
      T acc(0.0);
      for (int k = 0; k < nd.nc; ++k) acc = acc + W[(int64_t)r * nd.nc + k] * f[k];
      if (r < nd.nc) z[nd.col0 + r] = F.Dinv[nd.col0 + r] * acc;
      else U[nd.u_off + r - nd.nc] = f[r] + acc;
    }
  }
  for (int s = (int)F.nodes.size() - 1; s >= 0; --s) {
    const auto& nd = F.nodes[s];
    const int m = nd.nc + nd.nr;
    const T* W = F.W.data() + nd.w_off;
    for (int i = 0; i < nd.nc; ++i) {
      T acc(0.0);
      for (int k = 0; k < m; ++k) {
        const T g = k < nd.nc ? z[nd.col0 + k] : x[F.rows[nd.row_off + k - nd.nc]];
        acc = acc + W[(int64_t)k * nd.nc + i] * g;
      }
      x[nd.col0 + i] = acc;
    }
  }
  for (int i = 0; i < n; ++i) b[i] = x[F.iperm[i]];
}

// ====================================================================== C ABI
extern "C" {

int st_mg_default_options(st_mg_options* o) {
  if (!o) return fail(ST_MG_ERR_INVALID_ARG, "null options");
  o->omega = 0.5;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->lambda_crit = 0.1;
  o->coarsen = 0;
  o->max_levels = 0;
  o->min_coarse_slabs = 1;
  o->nodal_solve = 0;
  o->nodal_jacobi_sweeps = 3;
  o->use_A = 1;
  o->setup_threads = 0;
  o->slab_prec = 0;
  o->residual_prec = -1;
  o->use_graph = 1;
  std::memset(o->smoother, 0, sizeof(o->smoother));
  o->persistent_split = 0;
  o->factor_cache = 0;
  o->autotune = 0;
  o->nd_leaf = 0;
  o->split_k = 0;
  o->tc_split_k = 0;
  return ST_MG_OK;
}

int st_mg_setup(const st_mg_problem* prob, const st_mg_options* opt, void* stream, st_mg_t* out) {
  if (int rc = st_mg_setup_begin(prob, opt, stream, out)) return rc;
  if (int rc = st_mg_setup_finish(*out)) {
    st_mg_destroy(*out);
    *out = nullptr;
    return rc;
  }
  return ST_MG_OK;
}

int st_mg_setup_begin(const st_mg_problem* prob, const st_mg_options* opt, void* stream, st_mg_t* out) {
  return guarded([&]() { return do_setup(prob, opt, stream, out, false); });
}

int st_mg_setup_finish(st_mg_t h) {
  if (!h) return fail(ST_MG_ERR_INVALID_ARG, "null handle");
  if (!h->pending_upload) return fail(ST_MG_ERR_INVALID_ARG, "handle is not waiting for st_mg_setup_finish");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
    return fail(ST_MG_ERR_INVALID_ARG, "st_mg_setup_finish must run with the handle's device current");
  return guarded([&]() { return setup_device(*h); });
}

int st_mg_setup_host(const st_mg_problem* prob, const st_mg_options* opt, st_mg_t* out) {
  return guarded([&]() { return do_setup(prob, opt, nullptr, out, true); });
}

void st_mg_destroy(st_mg_t h) {
  if (!h) return;
  if (!h->host_only && !h->pending_upload) cudaStreamSynchronize(h->stream);
  delete h;
}

int st_mg_sizes(st_mg_t h, int64_t* n_edge, int64_t* n_node, int64_t* n_dof, int32_t* n_levels) {
  if (!h) return fail(ST_MG_ERR_INVALID_ARG, "null handle");
  if (n_edge) *n_edge = h->space[0].ne;
  if (n_node) *n_node = h->space[0].nn;
  if (n_dof) *n_dof = h->user_len;
  if (n_levels) *n_levels = (int32_t)h->lv.size();
  return ST_MG_OK;
}

int st_mg_level_info(st_mg_t h, int32_t level, int32_t* space_level, int32_t* N_t, double* tau, int64_t* n_edge,
                     int64_t* n_node) {
  if (!h) return fail(ST_MG_ERR_INVALID_ARG, "null handle");
  if (level < 0 || level >= (int32_t)h->lv.size()) return fail(ST_MG_ERR_INVALID_ARG, "level out of range");
  const auto& L = h->lv[level];
  if (space_level) *space_level = L.s;
  if (N_t) *N_t = L.N_t;
  if (tau) *tau = L.tau;
  if (n_edge) *n_edge = h->space[L.s].ne;
  if (n_node) *n_node = h->space[L.s].nn;
  return ST_MG_OK;
}

int st_mg_assemble_load(st_mg_t h, int32_t n_modes, const double* a, const double* k, const double* phase,
                        double* f_dev) {
  return st_mg_assemble_load_batch(h, 0, n_modes, a, k, phase, f_dev);
}

int st_mg_assemble_load_batch(st_mg_t h, int32_t batch, int32_t n_modes, const double* a, const double* k,
                              const double* phase, double* f_dev) {
  if (int rc = check_dev(h)) return rc;
  if (batch < 0 || batch >= h->B) return fail(ST_MG_ERR_INVALID_ARG, "batch index out of range");
  if (n_modes < 0 || (n_modes > 0 && (!a || !k || !phase))) return fail(ST_MG_ERR_INVALID_ARG, "bad load");
  if (int rc = check_ptrs({f_dev})) return rc;
  return guarded([&]() {
    Handle& H = *h;
    std::vector<double> b;
    space_load(H.space[0].mesh, n_modes, a, k, phase, b);
    // time weights c[n q + i] = int_{I_n} g(t) phi_i dt, 3-point Gauss-Legendre per slab
    // (a problem of a ragged batch: its own slab count over the common horizon T)
    const int Nb = H.ragged ? H.pnt[batch] : H.lv[0].N_t;
    const double taub = H.prob.T / Nb;
    const double x3 = std::sqrt(0.6);
    const double gx[3] = {0.5 * (1.0 - x3), 0.5, 0.5 * (1.0 + x3)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    std::vector<double> c((size_t)Nb * H.q, 0.0);
    for (int n = 0; n < Nb; ++n)
      for (int p = 0; p < 3; ++p) {
        const double t = (n + gx[p]) * taub;
        const double g = std::sin(M_PI * t / H.prob.T) + 1.0;
        c[(size_t)n * H.q] += taub * gw[p] * g;
        if (H.q == 2) c[(size_t)n * 2 + 1] += taub * gw[p] * g * (2.0 * gx[p] - 1.0);
      }
    // staging buffers of the handle (no allocation here: a cudaFree would wait for
    // every stream of the device)
    double* db = H.load_b;
    double* dc = H.load_c;
    CK(cudaMemcpyAsync(db, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice, H.stream));
    CK(cudaMemcpyAsync(dc, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, H.stream));
    const int seg = Nb * H.q;
    if (H.ragged)
      CK(outer_load(db, dc, f_dev + H.poff[batch], H.space[0].ne, seg, (int)H.prow, H.stream));
    else
      CK(outer_load(db, dc, f_dev + (int64_t)batch * seg, H.space[0].ne, seg, seg * H.B, H.stream));
    CK(cudaStreamSynchronize(H.stream));
    return ST_MG_OK;
  });
}

int st_mg_residual(st_mg_t h, int32_t level, const double* f_dev, const double* x_dev, double* r_dev,
                   double* norm_out) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev, r_dev})) return rc;
  return guarded([&]() {
    double nsq = 0.0;
    op_residual(*h, level, f_dev, x_dev, r_dev, norm_out ? &nsq : nullptr, true);
    if (norm_out) *norm_out = std::sqrt(nsq);
    return ST_MG_OK;
  });
}

int st_mg_slab_solve(st_mg_t h, int32_t level, const double* r_dev, double* y_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({r_dev, y_dev})) return rc;
  return guarded([&]() {
    const int cols = h->lv[level].N_t * h->lv[level].B;
    const int ld = cols * h->q;
    op_slab_cols(*h, level, r_dev, ld, 0, cols, y_dev, ld, 0, 1.0, 0);
    return check_tc(*h);
  });
}

int st_mg_smooth_S(st_mg_t h, int32_t level, const double* f_dev, double* x_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev})) return rc;
  return guarded([&]() {
    op_smooth_S(*h, level, f_dev, x_dev);
    return check_tc(*h);
  });
}

int st_mg_correct_A(st_mg_t h, int32_t level, const double* f_dev, double* x_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev})) return rc;
  return guarded([&]() {
    op_correct_A(*h, level, f_dev, x_dev);
    return ST_MG_OK;
  });
}

int st_mg_grad_T(st_mg_t h, int32_t level, const double* r_dev, double* y_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({r_dev, y_dev})) return rc;
  return guarded([&]() {
    op_grad_T(*h, level, r_dev, y_dev);
    return ST_MG_OK;
  });
}

int st_mg_nodal_solve(st_mg_t h, int32_t level, const double* y_dev, double* z_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({y_dev, z_dev})) return rc;
  return guarded([&]() {
    op_nodal_solve(*h, level, y_dev, z_dev);
    return ST_MG_OK;
  });
}

int st_mg_time_integrate(st_mg_t h, int32_t level, const double* z_dev, double* w_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({z_dev, w_dev})) return rc;
  return guarded([&]() {
    op_time_integrate(*h, level, z_dev, w_dev);
    return ST_MG_OK;
  });
}

int st_mg_grad_add(st_mg_t h, int32_t level, const double* w_dev, double* x_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({w_dev, x_dev})) return rc;
  return guarded([&]() {
    op_grad_add(*h, level, w_dev, x_dev);
    return ST_MG_OK;
  });
}

int st_mg_restrict(st_mg_t h, int32_t level, const double* r_dev, double* rc_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (level + 1 >= (int32_t)h->lv.size()) return fail(ST_MG_ERR_INVALID_ARG, "no coarser level");
  if (int rc = check_ptrs({r_dev, rc_dev})) return rc;
  return guarded([&]() {
    op_restrict(*h, level, r_dev, rc_dev);
    return ST_MG_OK;
  });
}

int st_mg_prolong_add(st_mg_t h, int32_t level, const double* ec_dev, double* x_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (level + 1 >= (int32_t)h->lv.size()) return fail(ST_MG_ERR_INVALID_ARG, "no coarser level");
  if (int rc = check_ptrs({ec_dev, x_dev})) return rc;
  return guarded([&]() {
    op_prolong_add(*h, level, ec_dev, x_dev);
    return ST_MG_OK;
  });
}

int st_mg_coarse_solve(st_mg_t h, const double* f_dev, double* x_dev) {
  if (int rc = check_dev(h)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev})) return rc;
  return guarded([&]() {
    op_coarse_solve(*h, f_dev, x_dev);
    return ST_MG_OK;
  });
}

int st_mg_vcycle(st_mg_t h, const double* f_dev, double* x_dev, double* rel_res_out) {
  if (int rc = check_dev(h)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev})) return rc;
  return guarded([&]() {
    run_vcycle(*h, f_dev, x_dev);
    if (int rc = check_tc(*h)) return rc;
    if (rel_res_out) {
      const double fn = f_norm(*h, f_dev);
      const double nsq = outer_res_norm_sq(*h, f_dev, x_dev);
      *rel_res_out = std::sqrt(nsq) / (fn > 0 ? fn : 1.0);
    }
    return ST_MG_OK;
  });
}

int st_mg_vcycle_residual_async(st_mg_t h, const double* f_dev, double* x_dev, double* r_dev) {
  if (int rc = check_dev(h)) return rc;
  if (h->ragged) return fail(ST_MG_ERR_INVALID_ARG, "not available for a ragged batch (batch_nt)");
  if (int rc = check_ptrs({f_dev, x_dev, r_dev})) return rc;
  return guarded([&]() {
    run_vcycle(*h, f_dev, x_dev);
    op_residual(*h, 0, f_dev, x_dev, r_dev, nullptr, true);
    return ST_MG_OK;
  });
}

int st_mg_solve(st_mg_t h, const double* f_dev, double* x_dev, double rtol, int32_t maxit, int32_t* iters,
                double* rel_res, double* history) {
  if (int rc = check_dev(h)) return rc;
  if (maxit < 0) return fail(ST_MG_ERR_INVALID_ARG, "bad solve arguments");
  if (int rc = check_ptrs({f_dev, x_dev})) return rc;
  return guarded([&]() { return solve_loop(*h, f_dev, x_dev, rtol, maxit, iters, rel_res, history); });
}

int st_mg_solve_host(st_mg_t h, const double* f_host, double* x_host, double rtol, int32_t maxit, int32_t* iters,
                     double* rel_res, double* history) {
  if (int rc = check_dev(h)) return rc;
  if (!f_host || !x_host || maxit < 0) return fail(ST_MG_ERR_INVALID_ARG, "bad solve arguments");
  return guarded([&]() {
    Handle& H = *h;
    const int64_t n = H.user_len;
    // device staging buffers are allocated on the first call and kept by the handle
    if (!H.stage_f) {
      H.stage_f = H.dalloc<double>(n);
      H.stage_x = H.dalloc<double>(n);
    }
    CK(cudaMemcpyAsync(H.stage_f, f_host, n * sizeof(double), cudaMemcpyHostToDevice, H.stream));
    CK(cudaMemcpyAsync(H.stage_x, x_host, n * sizeof(double), cudaMemcpyHostToDevice, H.stream));
    const int st = solve_loop(H, H.stage_f, H.stage_x, rtol, maxit, iters, rel_res, history);
    CK(cudaMemcpyAsync(x_host, H.stage_x, n * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    CK(cudaStreamSynchronize(H.stream));
    return st;
  });
}

int st_mg_debug_get(st_mg_t h, int32_t what, int32_t level, void* host_buf, int64_t* bytes) {
  if (!h || !bytes) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  if (level < 0 || level >= (int32_t)h->space.size()) return fail(ST_MG_ERR_INVALID_ARG, "space level out of range");
  const auto& S = h->space[level];
  const void* src = nullptr;
  int64_t nb = 0;
  std::vector<int32_t> tmp;
  switch (what) {
    case 1:
      tmp.resize(2 * S.mesh.ne);
      for (int64_t e = 0; e < S.mesh.ne; ++e) { tmp[2 * e] = S.mesh.edge_lo[e]; tmp[2 * e + 1] = S.mesh.edge_hi[e]; }
      src = tmp.data(); nb = (int64_t)tmp.size() * 4; break;
    case 2: src = S.mesh.int_edges.data(); nb = (int64_t)S.mesh.int_edges.size() * 4; break;
    case 3: src = S.mesh.int_verts.data(); nb = (int64_t)S.mesh.int_verts.size() * 4; break;
    case 4: src = S.M.rowptr.data(); nb = (int64_t)S.M.rowptr.size() * 8; break;
    case 5: src = S.M.col.data(); nb = (int64_t)S.M.col.size() * 4; break;
    case 6: src = S.M.val.data(); nb = (int64_t)S.M.val.size() * 8; break;
    case 7: src = S.K.val.data(); nb = (int64_t)S.K.val.size() * 8; break;
    case 8:
      tmp.resize(2 * S.gtail.size());
      for (size_t e = 0; e < S.gtail.size(); ++e) { tmp[2 * e] = S.gtail[e]; tmp[2 * e + 1] = S.ghead[e]; }
      src = tmp.data(); nb = (int64_t)tmp.size() * 4; break;
    case 9: src = S.Kn.rowptr.data(); nb = (int64_t)S.Kn.rowptr.size() * 8; break;
    case 10: src = S.Kn.col.data(); nb = (int64_t)S.Kn.col.size() * 4; break;
    case 11: src = S.Kn.val.data(); nb = (int64_t)S.Kn.val.size() * 8; break;
    case 12: src = S.Px.rowptr.data(); nb = (int64_t)S.Px.rowptr.size() * 8; break;
    case 13: src = S.Px.col.data(); nb = (int64_t)S.Px.col.size() * 4; break;
    case 14: src = S.Px.val.data(); nb = (int64_t)S.Px.val.size() * 8; break;
    default: return fail(ST_MG_ERR_INVALID_ARG, "unknown debug item");
  }
  if (!host_buf) {
    *bytes = nb;
    return ST_MG_OK;
  }
  if (*bytes < nb) return fail(ST_MG_ERR_INVALID_ARG, "debug buffer too small");
  if (nb) std::memcpy(host_buf, src, (size_t)nb);
  *bytes = nb;
  return ST_MG_OK;
}

int st_mg_debug_host_slab_solve(st_mg_t h, int32_t level, const double* r_host, double* y_host) {
  if (!h || !r_host || !y_host) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  if (!h->host_only) return fail(ST_MG_ERR_INVALID_ARG, "only for handles built by st_mg_setup_host");
  if (level < 0 || level >= (int32_t)h->lv.size()) return fail(ST_MG_ERR_INVALID_ARG, "level out of range");
  return guarded([&]() {
    Handle& H = *h;
    const auto& L = H.lv[level];
    const int ne = H.space[L.s].ne, q = H.q, ld = L.N_t * L.B * q;
    for (int n = 0; n < L.N_t * L.B; ++n) {
      if (q == 1) {
        std::vector<double> b(ne);
        for (int e = 0; e < ne; ++e) b[e] = r_host[(int64_t)e * ld + n];
        host_factor_apply(L.fr, b);
        for (int e = 0; e < ne; ++e) y_host[(int64_t)e * ld + n] = b[e];
      } else {
        const cplx c0(H.c0.x / L.tau, H.c0.y / L.tau), c1(H.c1.x / L.tau, H.c1.y / L.tau), s1(H.s1.x, H.s1.y);
        std::vector<cplx> b(ne);
        for (int e = 0; e < ne; ++e)
          b[e] = r_host[(int64_t)e * ld + 2 * n] * c0 + r_host[(int64_t)e * ld + 2 * n + 1] * c1;
        host_factor_apply(L.fc, b);
        for (int e = 0; e < ne; ++e) {
          y_host[(int64_t)e * ld + 2 * n] = 2.0 * b[e].re;
          y_host[(int64_t)e * ld + 2 * n + 1] = 2.0 * (s1 * b[e]).re;
        }
      }
    }
    return ST_MG_OK;
  });
}

int st_mg_convergence_rate(st_mg_t h, double* x_dev, int32_t max_iter, double floor, double* rates_host,
                           int32_t* n_rates, double* rate) {
  if (int rc = check_dev(h)) return rc;
  if (int rc = check_ptrs({x_dev})) return rc;
  if (max_iter < 1 || !(floor >= 0.0) || !rates_host || !n_rates || !rate)
    return fail(ST_MG_ERR_INVALID_ARG, "max_iter >= 1, floor >= 0 and non-null outputs required");
  return guarded([&]() {
    Handle& H = *h;
    const int64_t len = H.user_len;
    if (!H.zero_f) {
      H.zero_f = H.dalloc<double>(len);
      CK(cudaMemsetAsync(H.zero_f, 0, len * sizeof(double), H.stream));
    }
    const double n0 = f_norm(H, x_dev);       // the handle's deterministic l2 norm (blocking)
    double prev = n0, best = 0.0;
    int n = 0;
    while (n < max_iter) {
      run_vcycle(H, H.zero_f, x_dev);          // f = 0: x is the error of the iteration
      if (int rc = check_tc(H)) return rc;
      const double nx = f_norm(H, x_dev);
      const double q = prev > 0.0 ? nx / prev : 0.0;
      rates_host[n++] = q;
      best = std::max(best, q);
      prev = nx;
      if (nx == 0.0 || nx < floor * n0) break;
    }
    *n_rates = n;
    *rate = best;
    return ST_MG_OK;
  });
}

int st_mg_probe_fp64(st_mg_t h, double* tflops) {
  if (int rc = check_dev(h)) return rc;
  if (!tflops) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    Handle& H = *h;
    const int blocks = 8 * H.n_sm, iters = 1 << 14;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(fp64_probe(H.partial, blocks, 256, H.stream));   // warm-up
    CK(cudaEventRecord(e0, H.stream));
    CK(fp64_probe(H.partial, blocks, iters, H.stream));
    CK(cudaEventRecord(e1, H.stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
    return ST_MG_OK;
  });
}

int st_mg_batch_norms(st_mg_t h, const double* v_dev, double* norms_host) {
  if (int rc = check_dev(h)) return rc;
  if (h->ragged) return fail(ST_MG_ERR_INVALID_ARG, "not available for a ragged batch (batch_nt)");
  if (!norms_host) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  if (int rc = check_ptrs({v_dev})) return rc;
  return guarded([&]() {
    Handle& H = *h;
    const int seg = H.lv[0].N_t * H.q;
    CK(batch_norms_sq(v_dev, H.space[0].ne, H.B, seg, H.bn_partial, H.bn_out, H.stream));
    std::vector<double> sq(H.B);
    CK(cudaMemcpyAsync(sq.data(), H.bn_out, H.B * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    CK(cudaStreamSynchronize(H.stream));
    if (int rc = check_tc(H)) return rc;
    for (int b = 0; b < H.B; ++b) norms_host[b] = std::sqrt(sq[b]);
    return ST_MG_OK;
  });
}

int st_mg_batch_norms_async(st_mg_t h, const double* v_dev, double* norms_sq_dev) {
  if (int rc = check_dev(h)) return rc;
  if (h->ragged) return fail(ST_MG_ERR_INVALID_ARG, "not available for a ragged batch (batch_nt)");
  if (int rc = check_ptrs({v_dev})) return rc;
  if (!norms_sq_dev) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() {
    Handle& H = *h;
    CK(batch_norms_sq(v_dev, H.space[0].ne, H.B, H.lv[0].N_t * H.q, H.bn_partial, norms_sq_dev, H.stream));
    return ST_MG_OK;
  });
}

int st_mg_check(st_mg_t h) {
  if (int rc = check_dev(h)) return rc;
  return guarded([&]() { return check_tc(*h); });
}

int st_mg_batch_zero(st_mg_t h, int32_t batch, double* v_dev) {
  if (int rc = check_dev(h)) return rc;
  if (h->ragged) return fail(ST_MG_ERR_INVALID_ARG, "not available for a ragged batch (batch_nt)");
  if (batch < 0 || batch >= h->B) return fail(ST_MG_ERR_INVALID_ARG, "batch index out of range");
  if (int rc = check_ptrs({v_dev})) return rc;
  return guarded([&]() {
    Handle& H = *h;
    const int seg = H.lv[0].N_t * H.q;
    CK(zero_cols(v_dev, H.space[0].ne, seg * H.B, batch * seg, seg, H.stream));
    return ST_MG_OK;
  });
}

int st_mg_memory(st_mg_t h, int64_t* own_bytes, int64_t* factor_bytes) {
  if (int rc = check_dev(h)) return rc;
  int64_t fb = 0;
  std::vector<const void*> seen;
  auto add = [&](const void* p, int64_t b) {
    if (!p || std::find(seen.begin(), seen.end(), p) != seen.end()) return;
    seen.push_back(p);
    fb += b;
  };
  for (auto& L : h->lv) add(L.fac.get(), L.fac ? L.fac->mem.bytes : 0);
  for (auto& S : h->space) add(S.nf.get(), S.nf ? S.nf->mem.bytes : 0);
  if (own_bytes) *own_bytes = h->mem.bytes;
  if (factor_bytes) *factor_bytes = fb;
  return ST_MG_OK;
}

int st_mg_cache_stats(int64_t* bytes, int32_t* entries, int32_t* in_use, int64_t* hits, int64_t* misses) {
  auto& C = factor_cache();
  std::lock_guard<std::mutex> g(C.mu);
  int64_t b = 0;
  int32_t u = 0;
  for (auto& kv : C.map) {
    b += kv.second.bytes();
    if (kv.second.refs() > 1) ++u;
  }
  if (bytes) *bytes = b;
  if (entries) *entries = (int32_t)C.map.size();
  if (in_use) *in_use = u;
  if (hits) *hits = C.hits;
  if (misses) *misses = C.misses;
  return ST_MG_OK;
}

int st_mg_cache_trim(int64_t max_bytes, int64_t* bytes_after) {
  if (max_bytes < 0) return fail(ST_MG_ERR_INVALID_ARG, "max_bytes < 0");
  auto& C = factor_cache();
  std::vector<FactorCache::Entry> drop;   // freed after the lock is released
  int64_t total = 0;
  {
    std::lock_guard<std::mutex> g(C.mu);
    for (auto& kv : C.map) total += kv.second.bytes();
    while (total > max_bytes) {
      auto victim = C.map.end();
      for (auto it = C.map.begin(); it != C.map.end(); ++it)
        if (it->second.refs() == 1 && (victim == C.map.end() || it->second.last_use < victim->second.last_use))
          victim = it;
      if (victim == C.map.end()) break;   // everything left is in use
      total -= victim->second.bytes();
      drop.push_back(std::move(victim->second));
      C.map.erase(victim);
    }
  }
  drop.clear();
  if (bytes_after) *bytes_after = total;
  return ST_MG_OK;
}

int st_mg_launch_count(int64_t* count) {
  if (!count) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  *count = launch_count();
  return ST_MG_OK;
}

int st_mg_split_waves(st_mg_t h, int32_t level, int32_t* waves) {
  if (int rc = check_level(h, level)) return rc;
  if (!waves) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  *waves = h->lv[level].split_waves;
  return ST_MG_OK;
}

int st_mg_set_split_waves(st_mg_t h, int32_t level, int32_t waves) {
  if (int rc = check_level(h, level)) return rc;
  if (waves < 0 || waves > 64) return fail(ST_MG_ERR_INVALID_ARG, "split waves outside [0, 64]");
  h->lv[level].split_waves = waves;
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  return ST_MG_OK;
}

int st_mg_slab_copy(st_mg_t h, int32_t level, int32_t nodal, const double* v_dev, int32_t slab, double* out_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({v_dev, out_dev})) return rc;
  const auto& L = h->lv[level];
  if (slab < 0 || slab >= L.N_t * h->B) return fail(ST_MG_ERR_INVALID_ARG, "slab index out of range");
  return guarded([&]() {
    const auto& S = h->space[L.s];
    const int64_t ld = (int64_t)L.N_t * h->B * h->q;
    CK(slab_copy(v_dev, ld, (int64_t)slab * h->q, h->q, nodal ? S.nn : S.ne, out_dev, h->stream));
    return ST_MG_OK;
  });
}

int st_mg_residual_halo(st_mg_t h, int32_t level, const double* f_dev, const double* x_dev, const double* x_prev_dev,
                        double* r_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({f_dev, x_dev, r_dev})) return rc;
  if (x_prev_dev && !aligned16(x_prev_dev)) return fail(ST_MG_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  if (h->B != 1) return fail(ST_MG_ERR_INVALID_ARG, "time-slab sharding takes one problem per handle");
  return guarded([&]() {
    Handle& H = *h;
    op_residual(H, level, f_dev, x_dev, r_dev, nullptr, true);
    if (x_prev_dev) {
      const auto& L = H.lv[level];
      const auto& S = H.space[L.s];
      CK(halo_history(view(S), S.Mv, x_prev_dev, r_dev, (int64_t)L.N_t * H.q, H.prob.degree, H.stream));
    }
    return ST_MG_OK;
  });
}

int st_mg_time_integrate_carry(st_mg_t h, int32_t level, const double* z_dev, const double* carry_dev,
                               double* w_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (int rc = check_ptrs({z_dev, w_dev})) return rc;
  if (carry_dev && !aligned16(carry_dev)) return fail(ST_MG_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  if (h->B != 1) return fail(ST_MG_ERR_INVALID_ARG, "time-slab sharding takes one problem per handle");
  return guarded([&]() {
    Handle& H = *h;
    if (!carry_dev) {
      op_time_integrate(H, level, z_dev, w_dev);
    } else {
      const auto& L = H.lv[level];
      CK(time_integrate_carry(z_dev, carry_dev, w_dev, H.space[L.s].nn, L.N_t, H.prob.degree, H.stream));
    }
    return ST_MG_OK;
  });
}

int st_mg_time_carry(st_mg_t h, int32_t level, const double* ends_dev, int32_t n_prev, double* carry_dev) {
  if (int rc = check_level(h, level)) return rc;
  if (n_prev < 0) return fail(ST_MG_ERR_INVALID_ARG, "n_prev < 0");
  if (int rc = check_ptrs({carry_dev})) return rc;
  if (n_prev > 0)
    if (int rc = check_ptrs({ends_dev})) return rc;
  return guarded([&]() {
    Handle& H = *h;
    CK(time_carry(ends_dev, n_prev, H.space[H.lv[level].s].nn, H.prob.degree, carry_dev, H.stream));
    return ST_MG_OK;
  });
}

int st_mg_set_launch_overlap(int32_t on) {
  if (on != 0 && on != 1) return fail(ST_MG_ERR_INVALID_ARG, "launch overlap must be 0 or 1");
  set_launch_overlap(on != 0);
  return ST_MG_OK;
}

int st_mg_set_tc_mode(st_mg_t h, int32_t level, int32_t mode) {
  if (int rc = check_level(h, level)) return rc;
  if (mode < 0 || mode > 2) return fail(ST_MG_ERR_INVALID_ARG, "tensor-core mode must be 0, 1 or 2");
  if (h->lv[level].prec < 3)
    return fail(ST_MG_ERR_INVALID_ARG, "level has no 16-bit tensor-core factor (slab_prec 3 or 4)");
  h->lv[level].tc_mode = mode;
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  return ST_MG_OK;
}

int st_mg_factor_stats(st_mg_t h, int32_t level, double* macs_per_rhs, int64_t* factor_bytes, int32_t* depth) {
  if (int rc = check_level(h, level)) return rc;
  const auto& L = h->lv[level];
  const bool c = h->prob.degree == 1;
  const double macs = L.prec == 4 ? L.fac->dch.macs_per_rhs
                     : L.prec == 3 ? L.fac->dcb.macs_per_rhs
                     : L.prec == 1 ? (c ? L.fac->dcf.macs_per_rhs : L.fac->drf.macs_per_rhs)
                     : L.prec == 2 ? (c ? L.fac->dcd.macs_per_rhs : L.fac->drd.macs_per_rhs)
                                   : (c ? L.fac->dc.macs_per_rhs : L.fac->dr.macs_per_rhs);
  const int dep = L.prec == 4 ? L.fac->dch.max_depth
                  : L.prec == 3 ? L.fac->dcb.max_depth
                  : L.prec == 1 ? (c ? L.fac->dcf.max_depth : L.fac->drf.max_depth)
                  : L.prec == 2 ? (c ? L.fac->dcd.max_depth : L.fac->drd.max_depth)
                                : (c ? L.fac->dc.max_depth : L.fac->dr.max_depth);
  if (macs_per_rhs) *macs_per_rhs = macs;
  if (factor_bytes) *factor_bytes = L.fac->w_bytes;
  if (depth) *depth = dep;
  return ST_MG_OK;
}

const char* st_mg_strerror(int s) {
  switch (s) {
    case ST_MG_OK: return "ok";
    case ST_MG_ERR_INVALID_ARG: return "invalid argument";
    case ST_MG_ERR_OOM: return "out of memory";
    case ST_MG_ERR_CUDA: return "CUDA error";
    case ST_MG_ERR_DIVERGED: return "diverged";
    case ST_MG_ERR_NOT_CONVERGED: return "not converged";
    case ST_MG_ERR_NUMERIC: return "numerical breakdown (zero pivot)";
    case ST_MG_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* st_mg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
