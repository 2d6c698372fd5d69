// Nested-dissection multifrontal LDL^T (no pivoting) of the slab matrix
// A_slab (Section 2.1: every slab of a time level shares it, so it is factored
// once per level) and of the nodal matrix K_n (eq. AuxNodalSm).
//
// Matrices: DG(0) slab M + tau K (real SPD), DG(1) slab K + mu M with complex mu,
// Re mu > 0 (complex symmetric with SPD real part, so elimination without
// pivoting is stable), K_n (real SPD).
//
// Ordering: nested dissection guided by the positions of the unknowns (edge
// midpoints, vertices).  A set is cut in two by position along one axis, and the
// separator is the smaller of the two one-sided boundaries of the cut in the matrix
// graph (the unknowns of one part coupled to the other), which leaves the rest of
// the two parts uncoupled; the axis and the cut position (between 35% and 65% of the
// set) are chosen to make that separator smallest.  Each separator (and
// each leaf box) is one supernode; the factor is stored per supernode as
//   W_s = [ L11^{-1} ; -L21 L11^{-1} ]   (row-major, (nc + nr) x nc)
// which turns both triangular sweeps on the GPU into dense products.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <type_traits>

#include "host.h"

namespace stmg {

namespace {

inline double absv(double a) { return std::fabs(a); }
inline double absv(cplx a) { return std::sqrt(mag2(a)); }
inline double inv(double a) { return 1.0 / a; }
inline cplx inv(cplx a) { return cdiv(cplx(1.0, 0.0), a); }
inline double mul(double a, double b) { return a * b; }
inline cplx mul(cplx a, cplx b) { return a * b; }
inline bool isfin(double a) { return std::isfinite(a); }
inline bool isfin(cplx a) { return std::isfinite(a.re) && std::isfinite(a.im); }

// ---------------------------------------------------------------- thread pool
// Fixed set of worker threads; run(n, fn) executes fn(0..n-1) on the workers and the
// calling thread (dynamic scheduling by an atomic counter) and returns when all are done.
class Pool {
 public:
  explicit Pool(int nthreads) {
    for (int t = 1; t < nthreads; ++t) th_.emplace_back([this]() { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  int size() const { return (int)th_.size() + 1; }
  void run(int64_t n, const std::function<void(int64_t)>& fn) {
    if (n <= 0) return;
    if (th_.empty() || n == 1) {
      for (int64_t i = 0; i < n; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> g(mu_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      busy_ = (int)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [this]() { return busy_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work() {
    for (;;) {
      const int64_t i = next_.fetch_add(1);
      if (i >= n_) return;
      (*fn_)(i);
    }
  }
  void loop() {
    int64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&]() { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
      {
        std::lock_guard<std::mutex> g(mu_);
        if (--busy_ == 0) done_cv_.notify_one();
      }
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int64_t)>* fn_ = nullptr;
  int64_t n_ = 0, gen_ = 0;
  std::atomic<int64_t> next_{0};
  int busy_ = 0;
  bool stop_ = false;
};

// run fn(0..n-1) on the pool, or serially when pool is null
inline void pfor(Pool* pool, int64_t n, const std::function<void(int64_t)>& fn) {
  if (pool) {
    pool->run(n, fn);
  } else {
    for (int64_t i = 0; i < n; ++i) fn(i);
  }
}

// ---------------------------------------------------------------- dense kernels
// C[r + c ldc] -= sum_{k<K} A[r + k lda] * B[k bk + c bc] on an R x CC register tile.
template <int R, int CC>
inline void mk_sub(const double* A, int64_t lda, const double* B, int64_t bk, int64_t bc, double* C, int64_t ldc,
                   int64_t K) {
  double acc[CC][R] = {};
  for (int64_t k = 0; k < K; ++k) {
    const double* a = A + k * lda;
    for (int c = 0; c < CC; ++c) {
      const double b = B[k * bk + c * bc];
      for (int r = 0; r < R; ++r) acc[c][r] += a[r] * b;
    }
  }
  for (int c = 0; c < CC; ++c)
    for (int r = 0; r < R; ++r) C[r + c * ldc] -= acc[c][r];
}
template <int R, int CC>
inline void mk_sub(const cplx* A, int64_t lda, const cplx* B, int64_t bk, int64_t bc, cplx* C, int64_t ldc,
                   int64_t K) {
  double ar[CC][R] = {}, ai[CC][R] = {};
  for (int64_t k = 0; k < K; ++k) {
    const double* a = reinterpret_cast<const double*>(A + k * lda);
    double xr[R], xi[R];
    for (int r = 0; r < R; ++r) {
      xr[r] = a[2 * r];
      xi[r] = a[2 * r + 1];
    }
    for (int c = 0; c < CC; ++c) {
      const cplx b = B[k * bk + c * bc];
      for (int r = 0; r < R; ++r) {
        ar[c][r] += xr[r] * b.re - xi[r] * b.im;
        ai[c][r] += xr[r] * b.im + xi[r] * b.re;
      }
    }
  }
  for (int c = 0; c < CC; ++c) {
    double* cc = reinterpret_cast<double*>(C + c * ldc);
    for (int r = 0; r < R; ++r) {
      cc[2 * r] -= ar[c][r];
      cc[2 * r + 1] -= ai[c][r];
    }
  }
}
// the same for an arbitrary (small) tile
template <typename T>
inline void mk_sub_any(const T* A, int64_t lda, const T* B, int64_t bk, int64_t bc, T* C, int64_t ldc, int64_t M,
                       int64_t N, int64_t K) {
  for (int64_t c = 0; c < N; ++c)
    for (int64_t r = 0; r < M; ++r) {
      T acc(0.0);
      for (int64_t k = 0; k < K; ++k) acc = acc + A[r + k * lda] * B[k * bk + c * bc];
      C[r + c * ldc] = C[r + c * ldc] - acc;
    }
}

// C (M x N, column-major ldc) -= A (M x K, column-major lda) * B, B(k, c) = B[k bk + c bc].
// Serial; callers split the columns across threads.
template <typename T>
void gemm_sub(const T* A, int64_t lda, const T* B, int64_t bk, int64_t bc, T* C, int64_t ldc, int64_t M,
              int64_t N, int64_t K) {
  constexpr int R = 8;
  constexpr int CC = std::is_same<T, cplx>::value ? 2 : 4;
  if (M <= 0 || N <= 0 || K <= 0) return;
  int64_t r0 = 0;
  for (; r0 + R <= M; r0 += R) {
    int64_t c0 = 0;
    for (; c0 + CC <= N; c0 += CC) mk_sub<R, CC>(A + r0, lda, B + c0 * bc, bk, bc, C + r0 + c0 * ldc, ldc, K);
    if (c0 < N) mk_sub_any(A + r0, lda, B + c0 * bc, bk, bc, C + r0 + c0 * ldc, ldc, (int64_t)R, N - c0, K);
  }
  if (r0 < M) mk_sub_any(A + r0, lda, B, bk, bc, C + r0, ldc, M - r0, N, K);
}

constexpr int64_t kPanel = 64;   // panel width of the blocked LDL^T
constexpr int64_t kFrontPerThread = 1000;   // largest front order factored by a single thread
constexpr int64_t kColGroup = 16;   // columns per parallel task

// Partial LDL^T of the dense front F (m x m, column-major, lower triangle valid):
// eliminate the first nc columns; afterwards F[:, :nc] holds L (unit diagonal
// implied) below the diagonal and D on it, F[nc:, nc:] the Schur complement.
// Blocked right-looking: per panel of kPanel columns the diagonal block is factored
// column by column, the rows below it in parallel row chunks, then the trailing
// lower triangle is updated with W = L_panel D_panel as register-tiled products.
template <typename T>
bool front_ldlt(T* F, int64_t m, int64_t nc, Pool* pool) {
  std::vector<T> Wt;
  for (int64_t kb = 0; kb < nc; kb += kPanel) {
    const int64_t ke = std::min(kb + kPanel, nc), K = ke - kb;
    // diagonal block rows kb..ke-1 of the panel (left-looking inside the panel)
    for (int64_t k = kb; k < ke; ++k) {
      T* colk = F + k * m;
      for (int64_t j = kb; j < k; ++j) {
        const T t = mul(F[j * m + j], F[j * m + k]);   // D_j * L_kj
        for (int64_t i = k; i < ke; ++i) colk[i] = colk[i] - F[j * m + i] * t;
      }
      const T d = colk[k];
      if (!(absv(d) > 0.0) || !isfin(d)) return false;
      const T di = inv(d);
      for (int64_t i = k + 1; i < ke; ++i) colk[i] = mul(colk[i], di);
    }
    // rows below the diagonal block, in independent row chunks
    const int64_t rows = m - ke, chunk = 256;
    pfor(rows > chunk ? pool : nullptr, (rows + chunk - 1) / chunk, [&](int64_t ci) {
      const int64_t r0 = ke + ci * chunk, r1 = std::min(m, r0 + chunk);
      for (int64_t k = kb; k < ke; ++k) {
        T* colk = F + k * m;
        for (int64_t j = kb; j < k; ++j) {
          const T t = mul(F[j * m + j], F[j * m + k]);
          const T* colj = F + j * m;
          for (int64_t i = r0; i < r1; ++i) colk[i] = colk[i] - colj[i] * t;
        }
        const T di = inv(colk[k]);
        for (int64_t i = r0; i < r1; ++i) colk[i] = mul(colk[i], di);
      }
    });
    // trailing update: F[r][c] -= sum_k L[r][k] D_k L[c][k] for c >= ke, r >= c
    const int64_t P = m - ke;
    if (P <= 0) continue;
    Wt.resize((size_t)(K * P));
    for (int64_t k = 0; k < K; ++k) {
      const T d = F[(kb + k) * m + kb + k];
      const T* lk = F + (kb + k) * m + ke;
      T* w = Wt.data() + k * P;
      for (int64_t c = 0; c < P; ++c) w[c] = mul(d, lk[c]);
    }
    const int64_t ngroups = (P + kColGroup - 1) / kColGroup;
    pfor(P * P > 4096 ? pool : nullptr, ngroups, [&](int64_t g) {
      const int64_t c0 = ke + g * kColGroup, c1 = std::min(m, c0 + kColGroup);
      gemm_sub(F + kb * m + c0, m, Wt.data() + (c0 - ke), P, 1, F + c0 * m + c0, m, m - c0, c1 - c0, K);
    });
  }
  return true;
}

// X = L11^{-1} (nc x nc, column-major) for the unit lower triangle L11 of the front:
// forward substitution on groups of kColGroup columns, blocked by kPanel rows.
template <typename T>
void tri_inverse(const T* F, int64_t m, int64_t nc, T* X, Pool* pool) {
  const int64_t ngroups = (nc + kColGroup - 1) / kColGroup;
  pfor(nc > 128 ? pool : nullptr, ngroups, [&](int64_t g) {
    const int64_t j0 = g * kColGroup, j1 = std::min(nc, j0 + kColGroup), N = j1 - j0;
    for (int64_t j = j0; j < j1; ++j) {
      T* x = X + j * nc;
      std::fill(x, x + nc, T(0.0));
      x[j] = T(1.0);
    }
    for (int64_t b0 = (j0 / kPanel) * kPanel; b0 < nc; b0 += kPanel) {
      const int64_t b1 = std::min(nc, b0 + kPanel);
      for (int64_t k = b0; k < b1; ++k) {
        const T* lk = F + k * m;
        for (int64_t c = 0; c < N; ++c) {
          T* x = X + (j0 + c) * nc;
          const T xk = x[k];
          for (int64_t i = k + 1; i < b1; ++i) x[i] = x[i] - lk[i] * xk;
        }
      }
      if (b1 < nc)
        gemm_sub(F + b0 * m + b1, m, X + j0 * nc + b0, 1, nc, X + j0 * nc + b1, nc, nc - b1, N, b1 - b0);
    }
  });
}

struct NDNode {
  std::vector<int32_t> cols;   // original indices
  int child[2] = {-1, -1};
  int depth = 0;
};

}  // namespace

template <typename T>
int factor_nd_threads(const Csr& A, const std::vector<T>& val, const NDCoords& co, int leaf_max,
                      SupernodalFactor<T>& F, std::string& err, int nthreads) {
  const int32_t n = A.nrows;
  F = SupernodalFactor<T>();
  F.n = n;
  // ---------------- nested dissection tree (recursive, built bottom-up in postorder)
  std::vector<NDNode> tree;
  std::vector<int8_t> side(n, -1);
  std::vector<int32_t> rank(n, -1);
  std::function<int(std::vector<int32_t>&, int)> build = [&](std::vector<int32_t>& idx, int depth) -> int {
    NDNode node;
    node.depth = depth;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const std::vector<double>* cv3[3] = {&co.rx, &co.ry, &co.rz};
    for (int32_t i : idx)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], (*cv3[d])[i]);
        hi[d] = std::max(hi[d], (*cv3[d])[i]);
      }
    if ((int)idx.size() <= leaf_max || (hi[0] <= lo[0] && hi[1] <= lo[1] && hi[2] <= lo[2])) {
      node.cols = idx;
      tree.push_back(node);
      return (int)tree.size() - 1;
    }
    // Candidate cuts: each axis, the first h unknowns in coordinate order on one side,
    // h / |idx| in [0.35, 0.65].  With rank[i] the position of i in that order and
    // lo_nb / hi_nb the lowest / highest rank among i's neighbours in the set, i < h lies
    // on the boundary of the lower part iff hi_nb[i] >= h, and i >= h on the boundary of
    // the upper part iff lo_nb[i] < h; the cut with the smallest boundary wins.
    const int64_t m = (int64_t)idx.size();
    size_t best_sep = SIZE_MAX;
    int best_axis = -1;
    int64_t best_h = 0;
    std::vector<int32_t> best_ord;
    std::vector<int32_t> ord(idx);
    std::vector<int32_t> lo_nb(m), hi_nb(m), cnt_lo(m + 1), cnt_hi(m + 1);
    for (int axis = 0; axis < 3; ++axis) {
      if (!(hi[axis] > lo[axis])) continue;
      const std::vector<double>& cv = *cv3[axis];
      ord = idx;
      std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return cv[a] < cv[b] || (cv[a] == cv[b] && a < b); });
      for (int64_t q = 0; q < m; ++q) rank[ord[q]] = (int32_t)q;
      for (int64_t q = 0; q < m; ++q) {
        const int32_t i = ord[q];
        int32_t l = (int32_t)q, h = (int32_t)q;
        for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
          const int32_t r = rank[A.col[e]];
          if (r >= 0) { l = std::min(l, r); h = std::max(h, r); }
        }
        lo_nb[q] = l;
        hi_nb[q] = h;
      }
      // boundary sizes for every h at once: lower part {q < h: hi_nb[q] >= h},
      // upper part {q >= h: lo_nb[q] < h}, by difference arrays over h
      std::fill(cnt_lo.begin(), cnt_lo.end(), 0);
      std::fill(cnt_hi.begin(), cnt_hi.end(), 0);
      for (int64_t q = 0; q < m; ++q) {
        if (hi_nb[q] > q) { cnt_lo[q + 1]++; cnt_lo[hi_nb[q] + 1]--; }       // h in (q, hi_nb]
        if (lo_nb[q] < q) { cnt_hi[lo_nb[q] + 1]++; cnt_hi[q + 1]--; }       // h in (lo_nb, q]
      }
      int64_t run_lo = 0, run_hi = 0;
      for (int64_t h = 0; h <= m; ++h) {
        run_lo += cnt_lo[h];
        run_hi += cnt_hi[h];
        if (20 * h < 7 * m || 20 * h > 13 * m) continue;
        const size_t sep = (size_t)std::min(run_lo, run_hi);
        if (sep < best_sep) { best_sep = sep; best_axis = axis; best_h = h; best_ord = ord; }
      }
      for (int32_t i : idx) rank[i] = -1;
    }
    if (best_axis < 0) {
      node.cols = idx;
      tree.push_back(node);
      return (int)tree.size() - 1;
    }
    for (int64_t q = 0; q < m; ++q) side[best_ord[q]] = q < best_h ? 0 : 1;
    std::vector<int32_t> bnd[2], rest[2];
    for (int32_t i : idx) {
      bool cut = false;
      for (int64_t q = A.rowptr[i]; q < A.rowptr[i + 1] && !cut; ++q) {
        const int8_t sj = side[A.col[q]];
        cut = sj >= 0 && sj != side[i];
      }
      (cut ? bnd : rest)[side[i]].push_back(i);
    }
    for (int32_t i : idx) side[i] = -1;
    // separator: the smaller boundary; its side keeps only its interior
    const int sep = bnd[0].size() <= bnd[1].size() ? 0 : 1;
    std::vector<int32_t> L = rest[sep], R = rest[1 - sep], S = bnd[sep];
    R.insert(R.end(), bnd[1 - sep].begin(), bnd[1 - sep].end());
    if (S.empty()) {                     // halves not coupled: any single unknown separates
      std::vector<int32_t>& from = R.empty() ? L : R;
      S.push_back(from.back());
      from.pop_back();
    }
    int nch = 0;
    int ch[2] = {-1, -1};
    if (!L.empty()) ch[nch++] = build(L, depth + 1);
    if (!R.empty()) ch[nch++] = build(R, depth + 1);
    node.child[0] = ch[0];
    node.child[1] = ch[1];
    node.cols = S;
    tree.push_back(node);
    return (int)tree.size() - 1;
  };
  {
    std::vector<int32_t> all(n);
    for (int32_t i = 0; i < n; ++i) all[i] = i;
    build(all, 0);
  }
  const int nn = (int)tree.size();   // tree[] is already in postorder (children pushed first)
  F.perm.resize(n);
  F.iperm.resize(n);
  F.nodes.resize(nn);
  int32_t pos = 0;
  for (int s = 0; s < nn; ++s) {
    auto& nd = F.nodes[s];
    std::sort(tree[s].cols.begin(), tree[s].cols.end());
    nd.col0 = pos;
    nd.nc = (int32_t)tree[s].cols.size();
    nd.depth = tree[s].depth;
    nd.child[0] = tree[s].child[0];
    nd.child[1] = tree[s].child[1];
    for (int c = 0; c < 2; ++c)
      if (nd.child[c] >= 0) F.nodes[nd.child[c]].parent = s;
    for (int32_t i : tree[s].cols) { F.perm[pos] = i; F.iperm[i] = pos; ++pos; }
    F.max_depth = std::max(F.max_depth, nd.depth);
  }
  if (pos != n) { err = "nested dissection lost unknowns"; return 1; }
  for (int s = 0; s < nn; ++s)
    if (F.nodes[s].nc == 0) { err = "empty separator in nested dissection"; return 1; }

  // ---------------- symbolic: struct(s) = ancestors' indices coupled to subtree(s)
  std::vector<std::vector<int32_t>> st(nn);
  for (int s = 0; s < nn; ++s) {
    const auto& nd = F.nodes[s];
    const int32_t end = nd.col0 + nd.nc;
    std::vector<int32_t>& S = st[s];
    for (int32_t jl = 0; jl < nd.nc; ++jl) {
      const int32_t j = F.perm[nd.col0 + jl];
      for (int64_t q = A.rowptr[j]; q < A.rowptr[j + 1]; ++q) {
        const int32_t pi = F.iperm[A.col[q]];
        if (pi >= end) S.push_back(pi);
      }
    }
    for (int c = 0; c < 2; ++c) {
      const int ch = nd.child[c];
      if (ch < 0) continue;
      for (int32_t r : st[ch]) {
        if (r >= end) S.push_back(r);
        else if (r < nd.col0) { err = "symbolic factorisation: child structure escapes parent"; return 1; }
      }
    }
    std::sort(S.begin(), S.end());
    S.erase(std::unique(S.begin(), S.end()), S.end());
    F.nodes[s].nr = (int32_t)S.size();
  }

  // ---------------- offsets
  int64_t woff = 0, roff = 0, uoff = 0, goff = 0;
  F.gather_off.resize(nn);
  for (int s = 0; s < nn; ++s) {
    auto& nd = F.nodes[s];
    nd.w_off = woff;
    nd.row_off = roff;
    nd.u_off = uoff;
    F.gather_off[s] = goff;
    woff += (int64_t)(nd.nc + nd.nr) * nd.nc;
    roff += nd.nr;
    uoff += nd.nr;
    goff += nd.nc + nd.nr;
    // forward + backward multiply-adds of one right-hand side (triangular L11^{-1} counted once)
    F.flops_apply_per_rhs += 2.0 * ((double)nd.nc * (nd.nc + 1) / 2.0 + (double)nd.nr * nd.nc);
  }
  F.u_rows = uoff;
  F.W.assign(woff, T(0.0));
  F.rows.resize(roff);
  F.Dinv.assign(n, T(0.0));
  F.gsrc.assign(goff * 2, -1);
  for (int s = 0; s < nn; ++s)
    std::copy(st[s].begin(), st[s].end(), F.rows.begin() + F.nodes[s].row_off);

  // local position of permuted index r in front s
  auto local_pos = [&](int s, int32_t r) -> int64_t {
    const auto& nd = F.nodes[s];
    if (r >= nd.col0 && r < nd.col0 + nd.nc) return r - nd.col0;
    auto it = std::lower_bound(st[s].begin(), st[s].end(), r);
    if (it == st[s].end() || *it != r) return -1;
    return nd.nc + (it - st[s].begin());
  };

  // forward gather table
  for (int s = 0; s < nn; ++s) {
    const auto& nd = F.nodes[s];
    for (int c = 0; c < 2; ++c) {
      const int ch = nd.child[c];
      if (ch < 0) continue;
      const auto& cn = F.nodes[ch];
      for (int32_t ri = 0; ri < cn.nr; ++ri) {
        const int64_t p = local_pos(s, st[ch][ri]);
        if (p < 0) { err = "gather table: missing position"; return 1; }
        F.gsrc[(F.gather_off[s] + p) * 2 + c] = (int32_t)(cn.u_off + ri);
      }
    }
  }

  // ---------------- numeric multifrontal factorisation, one tree depth at a time
  // (supernodes of one depth are independent; a depth with at least one supernode per
  // thread and fronts of at most kFrontPerThread rows runs one supernode per thread,
  // otherwise the supernodes go one after another with all threads inside each front:
  // a large front factored by one thread streams its panels from memory and left the
  // whole depth waiting on the slowest thread, at 1/3 of the inner-parallel rate.
  // Either way every entry is computed in the same order, so the factor does not
  // depend on the schedule)
  std::vector<std::vector<T>> upd(nn);
  std::vector<std::vector<int>> by_depth(F.max_depth + 1);
  for (int s = 0; s < nn; ++s) by_depth[F.nodes[s].depth].push_back(s);
  const int nthr = std::max(1, nthreads);
  Pool pool(nthr);
  std::vector<char> bad(nn, 0);

  auto factor_node = [&](int s, Pool* inner) {
    const auto& nd = F.nodes[s];
    const int64_t nc = nd.nc, nr = nd.nr, m = nc + nr;
    std::vector<T> front((size_t)(m * m), T(0.0));
    for (int64_t jl = 0; jl < nc; ++jl) {
      const int32_t j = F.perm[nd.col0 + jl];
      for (int64_t q = A.rowptr[j]; q < A.rowptr[j + 1]; ++q) {
        const int32_t pi = F.iperm[A.col[q]];
        if (pi < nd.col0 + jl) continue;   // upper triangle: assembled from its own column
        const int64_t li = local_pos(s, pi);
        front[jl * m + li] = front[jl * m + li] + val[q];
      }
    }
    for (int c = 0; c < 2; ++c) {
      const int ch = nd.child[c];
      if (ch < 0) continue;
      const int64_t cr = F.nodes[ch].nr;
      std::vector<int64_t> map(cr);
      for (int64_t a = 0; a < cr; ++a) map[a] = local_pos(s, st[ch][a]);
      const std::vector<T>& U = upd[ch];
      for (int64_t b = 0; b < cr; ++b)
        for (int64_t a = b; a < cr; ++a) {
          int64_t ra = map[a], cb = map[b];
          if (ra < cb) std::swap(ra, cb);
          front[cb * m + ra] = front[cb * m + ra] + U[b * cr + a];
        }
      std::vector<T>().swap(upd[ch]);
    }
    if (!front_ldlt(front.data(), m, nc, inner)) {
      bad[s] = 1;
      return;
    }
    if (nr > 0) {
      upd[s].assign((size_t)(nr * nr), T(0.0));
      for (int64_t b = 0; b < nr; ++b)
        for (int64_t a = b; a < nr; ++a) upd[s][b * nr + a] = front[(nc + b) * m + nc + a];
    }
    for (int64_t k = 0; k < nc; ++k) F.Dinv[nd.col0 + k] = inv(front[k * m + k]);
    // X = L11^{-1}; W top = X (row-major lower), W bottom = -L21 X
    std::vector<T> X((size_t)(nc * nc));
    tri_inverse(front.data(), m, nc, X.data(), inner);
    T* W = F.W.data() + nd.w_off;
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t j = 0; j <= i; ++j) W[i * nc + j] = X[j * nc + i];
    if (nr > 0) {
      std::vector<T> Tb((size_t)(nr * nc), T(0.0));   // column-major nr x nc
      const int64_t ngroups = (nc + kColGroup - 1) / kColGroup;
      pfor(nr * nc > 16384 ? inner : nullptr, ngroups, [&](int64_t g) {
        const int64_t j0 = g * kColGroup, j1 = std::min(nc, j0 + kColGroup);
        gemm_sub(front.data() + j0 * m + nc, m, X.data() + j0 * nc + j0, 1, nc, Tb.data() + j0 * nr, nr, nr,
                 j1 - j0, nc - j0);
      });
      for (int64_t r = 0; r < nr; ++r)
        for (int64_t j = 0; j < nc; ++j) W[(nc + r) * nc + j] = Tb[j * nr + r];
    }
  };

  for (int d = F.max_depth; d >= 0; --d) {
    const auto& lst = by_depth[d];
    int64_t mmax = 0;
    for (int s : lst) mmax = std::max<int64_t>(mmax, (int64_t)F.nodes[s].nc + F.nodes[s].nr);
    if (((int)lst.size() >= nthr && mmax <= kFrontPerThread) || nthr == 1) {
      pool.run((int64_t)lst.size(), [&](int64_t i) { factor_node(lst[i], nullptr); });
    } else {
      for (int s : lst) factor_node(s, &pool);
    }
    for (int s : lst)
      if (bad[s]) {
        err = "zero or non-finite pivot in LDL^T";
        return 6;
      }
  }
  return 0;
}

template int factor_nd_threads<double>(const Csr&, const std::vector<double>&, const NDCoords&, int,
                                       SupernodalFactor<double>&, std::string&, int);
template int factor_nd_threads<cplx>(const Csr&, const std::vector<cplx>&, const NDCoords&, int,
                                     SupernodalFactor<cplx>&, std::string&, int);

}  // namespace stmg
