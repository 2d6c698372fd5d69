// Nested-dissection multifrontal LDL^T (no pivoting) of the slab matrix
// A_slab (Section 2.1: every slab of a time level shares it, so it is factored
// once per level) and of the nodal matrix K_n (eq. AuxNodalSm).
//
// Matrices: DG(0) slab M + tau K (real SPD), DG(1) slab K + mu M with complex mu,
// Re mu > 0 (complex symmetric with SPD real part, so elimination without
// pivoting is stable), K_n (real SPD).
//
// Ordering: geometric nested dissection on the integer "min corner" of each
// unknown (tail vertex of an edge, the vertex itself for a node).  Splitting the
// set at plane c of axis a into {m_a < c}, {m_a == c} (separator), {m_a > c}
// separates the matrix graph, because unknowns couple only inside a common cube
// and the two outer sets touch disjoint layers of cubes.  Each separator (and
// each leaf box) is one supernode; the factor is stored per supernode as
//   W_s = [ L11^{-1} ; -L21 L11^{-1} ]   (row-major, (nc + nr) x nc)
// which turns both triangular sweeps on the GPU into dense products.
#include <algorithm>
#include <cmath>
#include <functional>
#include <thread>

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

// y[i] -= a[i] * t  for i in [0, n)
inline void axpy_sub(double* y, const double* a, double t, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] -= a[i] * t;
}
inline void axpy_sub(cplx* y, const cplx* a, cplx t, int64_t n) {
  double* yd = reinterpret_cast<double*>(y);
  const double* ad = reinterpret_cast<const double*>(a);
  const double tr = t.re, ti = t.im;
  for (int64_t i = 0; i < n; ++i) {
    const double ar = ad[2 * i], ai = ad[2 * i + 1];
    yd[2 * i] -= ar * tr - ai * ti;
    yd[2 * i + 1] -= ar * ti + ai * tr;
  }
}
// y[i] -= a0[i]*t0 + a1[i]*t1 + a2[i]*t2 + a3[i]*t3
inline void axpy4_sub(double* y, const double* a0, const double* a1, const double* a2, const double* a3,
                      double t0, double t1, double t2, double t3, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] -= a0[i] * t0 + a1[i] * t1 + a2[i] * t2 + a3[i] * t3;
}
inline void axpy4_sub(cplx* y, const cplx* a0, const cplx* a1, const cplx* a2, const cplx* a3, cplx t0,
                      cplx t1, cplx t2, cplx t3, int64_t n) {
  double* yd = reinterpret_cast<double*>(y);
  const double* p0 = reinterpret_cast<const double*>(a0);
  const double* p1 = reinterpret_cast<const double*>(a1);
  const double* p2 = reinterpret_cast<const double*>(a2);
  const double* p3 = reinterpret_cast<const double*>(a3);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t r = 2 * i, m = 2 * i + 1;
    yd[r] -= (p0[r] * t0.re - p0[m] * t0.im) + (p1[r] * t1.re - p1[m] * t1.im) +
             (p2[r] * t2.re - p2[m] * t2.im) + (p3[r] * t3.re - p3[m] * t3.im);
    yd[m] -= (p0[r] * t0.im + p0[m] * t0.re) + (p1[r] * t1.im + p1[m] * t1.re) +
             (p2[r] * t2.im + p2[m] * t2.re) + (p3[r] * t3.im + p3[m] * t3.re);
  }
}

template <typename Fn>
void parallel_for(int64_t n, int nthreads, Fn fn) {
  if (nthreads <= 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  const int nt = (int)std::min<int64_t>(nthreads, n);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int64_t i = t; i < n; i += nt) fn(i);
    });
  for (auto& x : th) x.join();
}

// Partial LDL^T of the dense front F (m x m, column-major, lower triangle valid):
// eliminate the first nc columns; afterwards F[:, :nc] holds L (unit diagonal
// implied) below the diagonal and D on it, F[nc:, nc:] the Schur complement.
template <typename T>
bool front_ldlt(T* F, int64_t m, int64_t nc, int nthreads) {
  const int64_t NB = 32;
  for (int64_t kb = 0; kb < nc; kb += NB) {
    const int64_t ke = std::min(kb + NB, nc);
    for (int64_t k = kb; k < ke; ++k) {
      T* colk = F + k * m;
      for (int64_t j = kb; j < k; ++j) {
        const T t = mul(F[j * m + j], F[j * m + k]);   // D_j * L_kj
        axpy_sub(colk + k, F + j * m + k, t, m - k);
      }
      const T d = colk[k];
      if (!(absv(d) > 0.0) || !isfin(d)) return false;
      const T di = inv(d);
      for (int64_t i = k + 1; i < m; ++i) colk[i] = mul(colk[i], di);
    }
    // trailing update of columns ke..m-1 with the panel kb..ke-1
    const int64_t ncols = m - ke;
    auto update_col = [&](int64_t cc) {
      const int64_t c = ke + cc;
      T* colc = F + c * m;
      int64_t j = kb;
      for (; j + 4 <= ke; j += 4) {
        const T t0 = mul(F[j * m + j], F[j * m + c]);
        const T t1 = mul(F[(j + 1) * m + j + 1], F[(j + 1) * m + c]);
        const T t2 = mul(F[(j + 2) * m + j + 2], F[(j + 2) * m + c]);
        const T t3 = mul(F[(j + 3) * m + j + 3], F[(j + 3) * m + c]);
        axpy4_sub(colc + c, F + j * m + c, F + (j + 1) * m + c, F + (j + 2) * m + c, F + (j + 3) * m + c,
                  t0, t1, t2, t3, m - c);
      }
      for (; j < ke; ++j) {
        const T t = mul(F[j * m + j], F[j * m + c]);
        axpy_sub(colc + c, F + j * m + c, t, m - c);
      }
    };
    const int nt = (ncols * (m - ke) > 200000) ? nthreads : 1;
    parallel_for(ncols, nt, update_col);
  }
  return true;
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
  std::function<int(std::vector<int32_t>&, int)> build = [&](std::vector<int32_t>& idx, int depth) -> int {
    NDNode node;
    node.depth = depth;
    int axis = -1;
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int32_t i : idx) {
      const int32_t c[3] = {co.x[i], co.y[i], co.z[i]};
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], c[d]); hi[d] = std::max(hi[d], c[d]); }
    }
    if ((int)idx.size() > leaf_max) {
      int best = 1;
      for (int d = 0; d < 3; ++d)
        if (hi[d] - lo[d] > best) { best = hi[d] - lo[d]; axis = d; }
      if (best < 2) axis = -1;
    }
    if (axis < 0) {
      node.cols = idx;
      tree.push_back(node);
      return (int)tree.size() - 1;
    }
    const std::vector<int32_t>& cv = axis == 0 ? co.x : axis == 1 ? co.y : co.z;
    const int32_t cut = (lo[axis] + hi[axis]) / 2;
    std::vector<int32_t> L, S, R;
    for (int32_t i : idx) (cv[i] < cut ? L : cv[i] == cut ? S : R).push_back(i);
    int nch = 0;
    int ch[2] = {-1, -1};
    if (!L.empty()) ch[nch++] = build(L, depth + 1);
    if (!R.empty()) ch[nch++] = build(R, depth + 1);
    node.child[0] = ch[0];
    node.child[1] = ch[1];
    node.cols = S;
    if (S.empty()) {  // cannot happen for lattice coordinates with range >= 2; keep a valid tree anyway
      node.cols.clear();
    }
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

  // ---------------- numeric multifrontal factorisation
  std::vector<std::vector<T>> upd(nn);
  std::vector<T> front, Linv;
  for (int s = 0; s < nn; ++s) {
    const auto& nd = F.nodes[s];
    const int64_t nc = nd.nc, nr = nd.nr, m = nc + nr;
    front.assign(m * m, T(0.0));
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
    if (!front_ldlt(front.data(), m, nc, nthreads)) {
      err = "zero or non-finite pivot in LDL^T";
      return 6;
    }
    if (nr > 0) {
      upd[s].assign(nr * nr, T(0.0));
      for (int64_t b = 0; b < nr; ++b)
        for (int64_t a = b; a < nr; ++a) upd[s][b * nr + a] = front[(nc + b) * m + nc + a];
    }
    for (int64_t k = 0; k < nc; ++k) F.Dinv[nd.col0 + k] = inv(front[k * m + k]);
    // Linv = L11^{-1} (unit lower), column-major nc x nc
    Linv.assign(nc * nc, T(0.0));
    parallel_for(nc, nc > 256 ? nthreads : 1, [&](int64_t j) {
      T* x = Linv.data() + j * nc;
      x[j] = T(1.0);
      for (int64_t k = j; k < nc; ++k) {
        const T xk = x[k];
        axpy_sub(x + k + 1, front.data() + k * m + k + 1, xk, nc - k - 1);
      }
    });
    // W top = Linv (row-major), W bottom = -L21 Linv
    T* W = F.W.data() + nd.w_off;
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t j = 0; j <= i; ++j) W[i * nc + j] = Linv[j * nc + i];
    if (nr > 0)
      parallel_for(nc, nr * nc > 100000 ? nthreads : 1, [&](int64_t j) {
        // column j of -L21 Linv = -sum_{k>=j} Linv[k][j] * L21[:, k]
        std::vector<T> acc(nr, T(0.0));
        const T* lj = Linv.data() + j * nc;
        for (int64_t k = j; k < nc; ++k) axpy_sub(acc.data(), front.data() + k * m + nc, T(0.0) - lj[k], nr);
        for (int64_t r = 0; r < nr; ++r) W[(nc + r) * nc + j] = T(0.0) - acc[r];
      });
  }
  return 0;
}

template int factor_nd_threads<double>(const Csr&, const std::vector<double>&, const NDCoords&, int,
                                       SupernodalFactor<double>&, std::string&, int);
template int factor_nd_threads<cplx>(const Csr&, const std::vector<cplx>&, const NDCoords&, int,
                                     SupernodalFactor<cplx>&, std::string&, int);

}  // namespace stmg
