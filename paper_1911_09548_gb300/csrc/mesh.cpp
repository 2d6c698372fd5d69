// Kuhn and general tetrahedral meshes, Whitney (lowest-order Nedelec) and P1 assembly,
// discrete gradient, spatial prolongation and the space part of the load (Section 3 and
// eq. AuxNodalSm of the paper; uniform refinement as in Section 5.1).
//
// General meshes take the element geometry from the coordinates: with the rows
// r_k = x_k - x_0 (k = 1..3) and det = r_1 . (r_2 x r_3),
//   grad lam_1 = (r_2 x r_3) / det, grad lam_2 = (r_3 x r_1) / det,
//   grad lam_3 = (r_1 x r_2) / det, grad lam_0 = -(sum of the others), |T| = |det| / 6,
// and a local edge (i, j) whose global orientation is j -> i (vertex id of j lower)
// carries the Whitney function with the opposite sign.
//
// Every Kuhn tet of permutation (a,b,c) in a cube of side h is the chain
//   v0 = corner, v1 = v0 + h e_a, v2 = v1 + h e_b, v3 = v2 + h e_c,
// whose barycentric coordinates in cube-local units u are
//   lam = (1 - u_a, u_a - u_b, u_b - u_c, u_c),
// so h grad(lam) = (-e_a, e_a - e_b, e_b - e_c, e_c) and |T| = h^3/6.  Vertex ids
// increase along the chain, so the global orientation lo -> hi of a local edge
// (i, j), i < j, is i -> j and the Whitney function is lam_i grad lam_j - lam_j grad lam_i.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "host.h"

namespace stmg {

const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const int kDir[7][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {0, 0, 1}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
const int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

namespace {

int dir_code(int dx, int dy, int dz) {
  for (int d = 0; d < 7; ++d)
    if (kDir[d][0] == dx && kDir[d][1] == dy && kDir[d][2] == dz) return d;
  return -1;
}

// h * grad(lam_v) for the tet of permutation p (unit-cube gradients).
void unit_gradients(int p, double g[4][3]) {
  for (int v = 0; v < 4; ++v)
    for (int d = 0; d < 3; ++d) g[v][d] = 0.0;
  const int a = kPerm[p][0], b = kPerm[p][1], c = kPerm[p][2];
  g[0][a] = -1.0;
  g[1][a] = 1.0; g[1][b] = -1.0;
  g[2][b] = 1.0; g[2][c] = -1.0;
  g[3][c] = 1.0;
}

double dot3(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }
void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

// Reference element matrices (h = 1, coefficient 1) per permutation:
//   Mref = (1/|T|) int w_p . w_q,  Kref = (1/|T|) int curl w_p . curl w_q,
// using int lam_i lam_j = |T| (1 + delta_ij) / 20.
struct RefMats {
  double M[6][6][6], K[6][6][6];
  RefMats() {
    for (int p = 0; p < 6; ++p) {
      double g[4][3];
      unit_gradients(p, g);
      for (int e = 0; e < 6; ++e)
        for (int f = 0; f < 6; ++f) {
          const int i = kLocalEdge[e][0], j = kLocalEdge[e][1];
          const int k = kLocalEdge[f][0], l = kLocalEdge[f][1];
          auto I = [](int s, int t) { return (s == t ? 2.0 : 1.0) / 20.0; };
          M[p][e][f] = I(i, k) * dot3(g[j], g[l]) - I(i, l) * dot3(g[j], g[k]) -
                       I(j, k) * dot3(g[i], g[l]) + I(j, l) * dot3(g[i], g[k]);
          double ce[3], cf[3];
          cross3(g[i], g[j], ce);
          cross3(g[k], g[l], cf);
          K[p][e][f] = 4.0 * dot3(ce, cf);
        }
    }
  }
};
const RefMats& ref() {
  static RefMats r;
  return r;
}

// Build a CSR pattern from (row, col) pairs.
void pattern_from_pairs(std::vector<std::pair<int32_t, int32_t>>& pr, int32_t nrows, int32_t ncols, Csr& A) {
  std::sort(pr.begin(), pr.end());
  pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
  A.nrows = nrows;
  A.ncols = ncols;
  A.rowptr.assign(nrows + 1, 0);
  A.col.resize(pr.size());
  for (size_t t = 0; t < pr.size(); ++t) {
    A.rowptr[pr[t].first + 1]++;
    A.col[t] = pr[t].second;
  }
  for (int32_t r = 0; r < nrows; ++r) A.rowptr[r + 1] += A.rowptr[r];
  A.val.assign(pr.size(), 0.0);
}

int64_t find_pos(const Csr& A, int32_t r, int32_t c) {
  auto b = A.col.begin() + A.rowptr[r], e = A.col.begin() + A.rowptr[r + 1];
  auto it = std::lower_bound(b, e, c);
  return (it != e && *it == c) ? (int64_t)(it - A.col.begin()) : -1;
}

// Barycentric gradients g and volume of tet t of a general mesh; returns det.
double general_grads(const TetMesh& m, int64_t t, double g[4][3], double& vol) {
  const int32_t* tv = &m.tet_vert[t * 4];
  double r[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) r[k][d] = m.xyz[(int64_t)tv[k + 1] * 3 + d] - m.xyz[(int64_t)tv[0] * 3 + d];
  double c12[3], c20[3], c01[3];
  cross3(r[1], r[2], c12);
  cross3(r[2], r[0], c20);
  cross3(r[0], r[1], c01);
  const double det = dot3(r[0], c12);
  for (int d = 0; d < 3; ++d) {
    g[1][d] = c12[d] / det;
    g[2][d] = c20[d] / det;
    g[3][d] = c01[d] / det;
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  vol = std::fabs(det) / 6.0;
  return det;
}

// +1 if local edge le of tet t is oriented i -> j globally (kLocalEdge order), else -1.
inline double edge_sign(const TetMesh& m, int64_t t, int le) {
  return m.tet_vert[t * 4 + kLocalEdge[le][0]] < m.tet_vert[t * 4 + kLocalEdge[le][1]] ? 1.0 : -1.0;
}

// Local Whitney matrices (coefficient 1, times |T|) of a general tet, orientation included.
void general_element(const TetMesh& m, int64_t t, double Me[6][6], double Ke[6][6]) {
  double g[4][3], vol;
  general_grads(m, t, g, vol);
  auto I = [](int s, int u) { return (s == u ? 2.0 : 1.0) / 20.0; };
  for (int e = 0; e < 6; ++e)
    for (int f = 0; f < 6; ++f) {
      const int i = kLocalEdge[e][0], j = kLocalEdge[e][1];
      const int k = kLocalEdge[f][0], l = kLocalEdge[f][1];
      const double sg = edge_sign(m, t, e) * edge_sign(m, t, f) * vol;
      Me[e][f] = sg * (I(i, k) * dot3(g[j], g[l]) - I(i, l) * dot3(g[j], g[k]) - I(j, k) * dot3(g[i], g[l]) +
                       I(j, l) * dot3(g[i], g[k]));
      double ce[3], cf[3];
      cross3(g[i], g[j], ce);
      cross3(g[k], g[l], cf);
      Ke[e][f] = sg * 4.0 * dot3(ce, cf);
    }
}

// Children of the red refinement: parent-local vertex i (< 4) or midpoint code 4 + le of
// local edge le = (i, j) in kLocalEdge order.
const int kRedChild[8][4] = {
    {0, 4 + 0, 4 + 1, 4 + 2},          // (x0,  x01, x02, x03)
    {4 + 0, 1, 4 + 3, 4 + 4},          // (x01, x1,  x12, x13)
    {4 + 1, 4 + 3, 2, 4 + 5},          // (x02, x12, x2,  x23)
    {4 + 2, 4 + 4, 4 + 5, 3},          // (x03, x13, x23, x3)
    {4 + 0, 4 + 1, 4 + 2, 4 + 4},      // (x01, x02, x03, x13)
    {4 + 0, 4 + 1, 4 + 3, 4 + 4},      // (x01, x02, x12, x13)
    {4 + 1, 4 + 2, 4 + 4, 4 + 5},      // (x02, x03, x13, x23)
    {4 + 1, 4 + 3, 4 + 4, 4 + 5},      // (x02, x12, x13, x23)
};

// Barycentric coordinates, in the parent, of a child vertex code (exact dyadics).
void code_lambda(int code, double lam[4]) {
  for (int v = 0; v < 4; ++v) lam[v] = 0.0;
  if (code < 4) {
    lam[code] = 1.0;
  } else {
    lam[kLocalEdge[code - 4][0]] = 0.5;
    lam[kLocalEdge[code - 4][1]] = 0.5;
  }
}

}  // namespace

void vertex_xyz(const TetMesh& m, int64_t v, double x[3]) {
  if (m.n > 0) {
    int i, j, k;
    m.vijk((int)v, i, j, k);
    x[0] = (double)i / m.n; x[1] = (double)j / m.n; x[2] = (double)k / m.n;
  } else {
    for (int d = 0; d < 3; ++d) x[d] = m.xyz[v * 3 + d];
  }
}

std::vector<double> longest_edges(const TetMesh& m) {
  std::vector<double> h(m.nt, 0.0);
  for (int64_t t = 0; t < m.nt; ++t)
    for (int le = 0; le < 6; ++le) {
      double a[3], b[3];
      vertex_xyz(m, m.tet_vert[t * 4 + kLocalEdge[le][0]], a);
      vertex_xyz(m, m.tet_vert[t * 4 + kLocalEdge[le][1]], b);
      const double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      h[t] = std::max(h[t], std::sqrt(dot3(d, d)));
    }
  return h;
}

int build_general(int32_t nv, const double* xyz, int64_t nt, const int32_t* tets, int bc, TetMesh& m,
                  std::string& err) {
  m = TetMesh();
  m.n = 0;
  m.nv = nv;
  m.nt = nt;
  m.xyz.assign(xyz, xyz + (int64_t)nv * 3);
  m.tet_vert.assign(tets, tets + nt * 4);
  std::vector<char> used(nv, 0);
  for (int64_t q = 0; q < nt * 4; ++q) {
    if (m.tet_vert[q] < 0 || m.tet_vert[q] >= nv) { err = "mesh: vertex id out of range"; return 1; }
    used[m.tet_vert[q]] = 1;
  }
  for (int32_t v = 0; v < nv; ++v)
    if (!used[v]) { err = "mesh: a vertex belongs to no tet"; return 1; }
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* tv = &m.tet_vert[t * 4];
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (tv[a] == tv[b]) { err = "mesh: repeated vertex in a tet"; return 1; }
    double g[4][3], vol, hmax = 0.0;
    general_grads(m, t, g, vol);
    for (int le = 0; le < 6; ++le) {
      double d[3];
      for (int s = 0; s < 3; ++s)
        d[s] = m.xyz[(int64_t)tv[kLocalEdge[le][1]] * 3 + s] - m.xyz[(int64_t)tv[kLocalEdge[le][0]] * 3 + s];
      hmax = std::max(hmax, std::sqrt(dot3(d, d)));
    }
    if (!(vol > 1e-12 * hmax * hmax * hmax) || !std::isfinite(vol)) { err = "mesh: tet of zero volume"; return 1; }
  }
  // edges: sorted vertex pairs, lexicographic
  std::vector<std::pair<int32_t, int32_t>> ed;
  ed.reserve(nt * 6);
  for (int64_t t = 0; t < nt; ++t)
    for (int le = 0; le < 6; ++le) {
      const int32_t a = m.tet_vert[t * 4 + kLocalEdge[le][0]], b = m.tet_vert[t * 4 + kLocalEdge[le][1]];
      ed.emplace_back(std::min(a, b), std::max(a, b));
    }
  std::sort(ed.begin(), ed.end());
  ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
  m.ne = (int64_t)ed.size();
  m.edge_lo.resize(m.ne);
  m.edge_hi.resize(m.ne);
  for (int64_t e = 0; e < m.ne; ++e) { m.edge_lo[e] = ed[e].first; m.edge_hi[e] = ed[e].second; }
  auto edge_id = [&](int32_t a, int32_t b) -> int32_t {
    const std::pair<int32_t, int32_t> key(std::min(a, b), std::max(a, b));
    return (int32_t)(std::lower_bound(ed.begin(), ed.end(), key) - ed.begin());
  };
  m.tet_edge.resize(nt * 6);
  for (int64_t t = 0; t < nt; ++t)
    for (int le = 0; le < 6; ++le)
      m.tet_edge[t * 6 + le] = edge_id(m.tet_vert[t * 4 + kLocalEdge[le][0]], m.tet_vert[t * 4 + kLocalEdge[le][1]]);
  // boundary = faces of one tet only
  std::vector<std::array<int32_t, 3>> faces;
  faces.reserve(nt * 4);
  for (int64_t t = 0; t < nt; ++t)
    for (int skip = 0; skip < 4; ++skip) {
      std::array<int32_t, 3> f;
      int c = 0;
      for (int v = 0; v < 4; ++v)
        if (v != skip) f[c++] = m.tet_vert[t * 4 + v];
      std::sort(f.begin(), f.end());
      faces.push_back(f);
    }
  std::sort(faces.begin(), faces.end());
  std::vector<char> bvert(nv, 0), bedge(m.ne, 0);
  for (size_t i = 0; i < faces.size();) {
    size_t j = i;
    while (j < faces.size() && faces[j] == faces[i]) ++j;
    if (j - i > 2) { err = "mesh: a face is shared by more than two tets"; return 1; }
    if (j - i == 1) {
      const auto& f = faces[i];
      for (int a = 0; a < 3; ++a) bvert[f[a]] = 1;
      bedge[edge_id(f[0], f[1])] = bedge[edge_id(f[0], f[2])] = bedge[edge_id(f[1], f[2])] = 1;
    }
    i = j;
  }
  m.vert_iid.assign(nv, -1);
  for (int32_t v = 0; v < nv; ++v)
    if (bc == 1 ? v != 0 : !bvert[v]) {
      m.vert_iid[v] = (int32_t)m.int_verts.size();
      m.int_verts.push_back(v);
    }
  m.edge_iid.assign(m.ne, -1);
  for (int64_t e = 0; e < m.ne; ++e)
    if (bc == 1 || !bedge[e]) {
      m.edge_iid[e] = (int32_t)m.int_edges.size();
      m.int_edges.push_back((int32_t)e);
    }
  return 0;
}

void refine_red(const TetMesh& c, int bc, TetMesh& f) {
  const int32_t nv = (int32_t)(c.nv + c.ne);
  std::vector<double> xyz((int64_t)nv * 3);
  for (int64_t v = 0; v < c.nv; ++v) vertex_xyz(c, v, &xyz[v * 3]);
  for (int64_t e = 0; e < c.ne; ++e) {
    double a[3], b[3];
    vertex_xyz(c, c.edge_lo[e], a);
    vertex_xyz(c, c.edge_hi[e], b);
    for (int d = 0; d < 3; ++d) xyz[(c.nv + e) * 3 + d] = 0.5 * (a[d] + b[d]);
  }
  std::vector<int32_t> tets(c.nt * 32);
  for (int64_t t = 0; t < c.nt; ++t)
    for (int k = 0; k < 8; ++k)
      for (int v = 0; v < 4; ++v) {
        const int code = kRedChild[k][v];
        tets[(t * 8 + k) * 4 + v] = code < 4 ? c.tet_vert[t * 4 + code] : (int32_t)(c.nv + c.tet_edge[t * 6 + code - 4]);
      }
  std::string err;
  build_general(nv, xyz.data(), c.nt * 8, tets.data(), bc, f, err);   // children of a valid mesh are valid
  f.parent.resize(f.nt);
  for (int64_t t = 0; t < f.nt; ++t) f.parent[t] = (int32_t)(t / 8);
}

void build_kuhn(int n, TetMesh& m, int bc) {
  m.n = n;
  m.nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  m.nt = (int64_t)6 * n * n * n;
  m.edge_of.assign(m.nv * 7, -1);
  m.edge_lo.clear();
  m.edge_hi.clear();
  for (int v = 0; v < m.nv; ++v) {
    int i, j, k;
    m.vijk(v, i, j, k);
    for (int d = 0; d < 7; ++d) {
      const int i2 = i + kDir[d][0], j2 = j + kDir[d][1], k2 = k + kDir[d][2];
      if (i2 > n || j2 > n || k2 > n) continue;
      m.edge_of[(int64_t)v * 7 + d] = (int32_t)m.edge_lo.size();
      m.edge_lo.push_back(v);
      m.edge_hi.push_back(m.vid(i2, j2, k2));
    }
  }
  m.ne = (int64_t)m.edge_lo.size();
  m.tet_vert.resize(m.nt * 4);
  m.tet_edge.resize(m.nt * 6);
  m.tet_perm.resize(m.nt);
  int64_t t = 0;
  for (int ck = 0; ck < n; ++ck)
    for (int cj = 0; cj < n; ++cj)
      for (int ci = 0; ci < n; ++ci)
        for (int p = 0; p < 6; ++p, ++t) {
          int c[3] = {ci, cj, ck};
          int pos[4][3];
          for (int d = 0; d < 3; ++d) pos[0][d] = c[d];
          for (int s = 0; s < 3; ++s) {
            for (int d = 0; d < 3; ++d) pos[s + 1][d] = pos[s][d];
            pos[s + 1][kPerm[p][s]] += 1;
          }
          for (int s = 0; s < 4; ++s) m.tet_vert[t * 4 + s] = m.vid(pos[s][0], pos[s][1], pos[s][2]);
          for (int e = 0; e < 6; ++e) {
            const int a = kLocalEdge[e][0], b = kLocalEdge[e][1];
            const int code = dir_code(pos[b][0] - pos[a][0], pos[b][1] - pos[a][1], pos[b][2] - pos[a][2]);
            m.tet_edge[t * 6 + e] = m.edge_of[(int64_t)m.tet_vert[t * 4 + a] * 7 + code];
          }
          m.tet_perm[t] = p;
        }
  m.vert_iid.assign(m.nv, -1);
  m.int_verts.clear();
  for (int v = 0; v < m.nv; ++v) {
    int i, j, k;
    m.vijk(v, i, j, k);
    // Dirichlet: interior vertices; Neumann: all but vertex 0 (the grounded node of
    // the singular nodal problem)
    const bool unknown = bc == 1 ? v != 0 : (i > 0 && i < n && j > 0 && j < n && k > 0 && k < n);
    if (unknown) {
      m.vert_iid[v] = (int32_t)m.int_verts.size();
      m.int_verts.push_back(v);
    }
  }
  m.edge_iid.assign(m.ne, -1);
  m.int_edges.clear();
  for (int64_t e = 0; e < m.ne; ++e) {
    int a[3], b[3];
    m.vijk(m.edge_lo[e], a[0], a[1], a[2]);
    m.vijk(m.edge_hi[e], b[0], b[1], b[2]);
    bool on_face = false;
    for (int d = 0; d < 3; ++d)
      if ((a[d] == 0 && b[d] == 0) || (a[d] == n && b[d] == n)) on_face = true;
    if (!on_face || bc == 1) {   // Neumann: every edge is an unknown
      m.edge_iid[e] = (int32_t)m.int_edges.size();
      m.int_edges.push_back((int32_t)e);
    }
  }
}

void assemble_edge(const TetMesh& m, const double* nu, const double* sigma, Csr& M, Csr& K) {
  const int32_t ni = (int32_t)m.int_edges.size();
  std::vector<std::pair<int32_t, int32_t>> pr;
  pr.reserve(m.nt * 36);
  for (int64_t t = 0; t < m.nt; ++t)
    for (int e = 0; e < 6; ++e) {
      const int32_t r = m.edge_iid[m.tet_edge[t * 6 + e]];
      if (r < 0) continue;
      for (int f = 0; f < 6; ++f) {
        const int32_t c = m.edge_iid[m.tet_edge[t * 6 + f]];
        if (c >= 0) pr.emplace_back(r, c);
      }
    }
  pattern_from_pairs(pr, ni, ni, M);
  K = M;
  if (m.n == 0) {
    for (int64_t t = 0; t < m.nt; ++t) {
      double Me[6][6], Ke[6][6];
      general_element(m, t, Me, Ke);
      for (int e = 0; e < 6; ++e) {
        const int32_t r = m.edge_iid[m.tet_edge[t * 6 + e]];
        if (r < 0) continue;
        for (int f = 0; f < 6; ++f) {
          const int32_t c = m.edge_iid[m.tet_edge[t * 6 + f]];
          if (c < 0) continue;
          const int64_t q = find_pos(M, r, c);
          M.val[q] += sigma[t] * Me[e][f];
          K.val[q] += nu[t] * Ke[e][f];
        }
      }
    }
    return;
  }
  const double h = 1.0 / m.n;
  const RefMats& R = ref();
  for (int64_t t = 0; t < m.nt; ++t) {
    const int p = m.tet_perm[t];
    const double sm = sigma[t] * h / 6.0;          // |T| / h^2
    const double sk = nu[t] / (6.0 * h);           // |T| / h^4
    for (int e = 0; e < 6; ++e) {
      const int32_t r = m.edge_iid[m.tet_edge[t * 6 + e]];
      if (r < 0) continue;
      for (int f = 0; f < 6; ++f) {
        const int32_t c = m.edge_iid[m.tet_edge[t * 6 + f]];
        if (c < 0) continue;
        const int64_t q = find_pos(M, r, c);
        M.val[q] += sm * R.M[p][e][f];
        K.val[q] += sk * R.K[p][e][f];
      }
    }
  }
}

void assemble_nodal(const TetMesh& m, const double* sigma, Csr& Kn) {
  const int32_t ni = (int32_t)m.int_verts.size();
  std::vector<std::pair<int32_t, int32_t>> pr;
  for (int64_t t = 0; t < m.nt; ++t)
    for (int a = 0; a < 4; ++a) {
      const int32_t r = m.vert_iid[m.tet_vert[t * 4 + a]];
      if (r < 0) continue;
      for (int b = 0; b < 4; ++b) {
        const int32_t c = m.vert_iid[m.tet_vert[t * 4 + b]];
        if (c >= 0) pr.emplace_back(r, c);
      }
    }
  pattern_from_pairs(pr, ni, ni, Kn);
  const double h = m.n > 0 ? 1.0 / m.n : 0.0;
  for (int64_t t = 0; t < m.nt; ++t) {
    double g[4][3], s;
    if (m.n > 0) {
      unit_gradients(m.tet_perm[t], g);
      s = sigma[t] * h / 6.0;
    } else {
      double vol;
      general_grads(m, t, g, vol);
      s = sigma[t] * vol;
    }
    for (int a = 0; a < 4; ++a) {
      const int32_t r = m.vert_iid[m.tet_vert[t * 4 + a]];
      if (r < 0) continue;
      for (int b = 0; b < 4; ++b) {
        const int32_t c = m.vert_iid[m.tet_vert[t * 4 + b]];
        if (c < 0) continue;
        Kn.val[find_pos(Kn, r, c)] += s * dot3(g[a], g[b]);
      }
    }
  }
}

void gradient_pairs(const TetMesh& m, std::vector<int32_t>& tail, std::vector<int32_t>& head) {
  tail.resize(m.int_edges.size());
  head.resize(m.int_edges.size());
  for (size_t i = 0; i < m.int_edges.size(); ++i) {
    tail[i] = m.vert_iid[m.edge_lo[m.int_edges[i]]];
    head[i] = m.vert_iid[m.edge_hi[m.int_edges[i]]];
  }
}

Csr gradient_csr(const std::vector<int32_t>& tail, const std::vector<int32_t>& head, int32_t nnodes) {
  Csr G;
  G.nrows = (int32_t)tail.size();
  G.ncols = nnodes;
  G.rowptr.assign(G.nrows + 1, 0);
  for (int32_t e = 0; e < G.nrows; ++e) {
    int32_t c0 = tail[e], c1 = head[e];
    double v0 = -1.0, v1 = 1.0;
    if (c0 >= 0 && c1 >= 0 && c1 < c0) { std::swap(c0, c1); std::swap(v0, v1); }
    if (c0 >= 0) { G.col.push_back(c0); G.val.push_back(v0); }
    if (c1 >= 0) { G.col.push_back(c1); G.val.push_back(v1); }
    G.rowptr[e + 1] = (int64_t)G.col.size();
  }
  return G;
}

// Whitney interpolation: for fine edge f with tail at fine lattice point P and
// direction d, the midpoint in coarse lattice units is (2P + d)/4; inside the
// coarse tet containing it, P[f, (i,j)] = (lam_i (g_j . d) - lam_j (g_i . d)) / 2,
// the line integral of the coarse Whitney function along f (exact: it is linear).
//
// General meshes (fine = red refinement of coarse): the fine edge lies in the parent T of
// the first fine tet that has it; the barycentric coordinates in T of the fine vertices
// are exact dyadics (kRedChild), and since grad lam . (x_hi - x_lo) = lam(x_hi) - lam(x_lo)
// the entry for the coarse edge i -> j of T is
//   lam_i(mid) (lam_j(hi) - lam_j(lo)) - lam_j(mid) (lam_i(hi) - lam_i(lo)),
// no geometry needed.
void edge_prolongation(const TetMesh& coarse, const TetMesh& fine, Csr& P) {
  const int n = coarse.n;
  P.nrows = (int32_t)fine.int_edges.size();
  P.ncols = (int32_t)coarse.int_edges.size();
  P.rowptr.assign(P.nrows + 1, 0);
  P.col.clear();
  P.val.clear();
  if (fine.n == 0) {
    std::vector<int64_t> first(fine.ne, -1);   // t * 6 + le of the first fine tet with the edge
    for (int64_t t = 0; t < fine.nt; ++t)
      for (int le = 0; le < 6; ++le)
        if (first[fine.tet_edge[t * 6 + le]] < 0) first[fine.tet_edge[t * 6 + le]] = t * 6 + le;
    for (int32_t r = 0; r < P.nrows; ++r) {
      const int32_t e = fine.int_edges[r];
      const int64_t t = first[e] / 6;
      const int le = (int)(first[e] % 6);
      const int64_t T = fine.parent[t];
      const int k = (int)(t - 8 * T);
      int ca = kRedChild[k][kLocalEdge[le][0]], cb = kRedChild[k][kLocalEdge[le][1]];
      if (fine.tet_vert[t * 4 + kLocalEdge[le][0]] > fine.tet_vert[t * 4 + kLocalEdge[le][1]]) std::swap(ca, cb);
      double lo[4], hi[4], mid[4];
      code_lambda(ca, lo);
      code_lambda(cb, hi);
      for (int v = 0; v < 4; ++v) mid[v] = 0.5 * (lo[v] + hi[v]);
      std::vector<std::pair<int32_t, double>> row;
      for (int ce = 0; ce < 6; ++ce) {
        int i = kLocalEdge[ce][0], j = kLocalEdge[ce][1];
        if (coarse.tet_vert[T * 4 + i] > coarse.tet_vert[T * 4 + j]) std::swap(i, j);
        const double v = mid[i] * (hi[j] - lo[j]) - mid[j] * (hi[i] - lo[i]);
        const int32_t c = coarse.edge_iid[coarse.tet_edge[T * 6 + ce]];
        if (v != 0.0 && c >= 0) row.emplace_back(c, v);
      }
      std::sort(row.begin(), row.end());
      for (auto& cv : row) {
        P.col.push_back(cv.first);
        P.val.push_back(cv.second);
      }
      P.rowptr[r + 1] = (int64_t)P.col.size();
    }
    return;
  }
  for (int32_t r = 0; r < P.nrows; ++r) {
    const int32_t e = fine.int_edges[r];
    int a[3], b[3];
    fine.vijk(fine.edge_lo[e], a[0], a[1], a[2]);
    fine.vijk(fine.edge_hi[e], b[0], b[1], b[2]);
    int d[3], cube[3];
    double u[3];
    for (int s = 0; s < 3; ++s) {
      d[s] = b[s] - a[s];
      const double mid = (2.0 * a[s] + d[s]) / 4.0;
      cube[s] = std::min((int)std::floor(mid), n - 1);
      u[s] = mid - cube[s];
    }
    int perm = -1;
    for (int p = 0; p < 6 && perm < 0; ++p)
      if (u[kPerm[p][0]] >= u[kPerm[p][1]] && u[kPerm[p][1]] >= u[kPerm[p][2]]) perm = p;
    const int pa = kPerm[perm][0], pb = kPerm[perm][1], pc = kPerm[perm][2];
    const double lam[4] = {1.0 - u[pa], u[pa] - u[pb], u[pb] - u[pc], u[pc]};
    double g[4][3];
    unit_gradients(perm, g);
    const int64_t t = (int64_t)6 * (cube[0] + n * (cube[1] + n * cube[2])) + perm;
    std::vector<std::pair<int32_t, double>> row;
    for (int le = 0; le < 6; ++le) {
      const int i = kLocalEdge[le][0], j = kLocalEdge[le][1];
      const double gjd = g[j][0] * d[0] + g[j][1] * d[1] + g[j][2] * d[2];
      const double gid = g[i][0] * d[0] + g[i][1] * d[1] + g[i][2] * d[2];
      const double v = 0.5 * (lam[i] * gjd - lam[j] * gid);
      const int32_t c = coarse.edge_iid[coarse.tet_edge[t * 6 + le]];
      if (v != 0.0 && c >= 0) row.emplace_back(c, v);
    }
    std::sort(row.begin(), row.end());
    for (auto& cv : row) {
      P.col.push_back(cv.first);
      P.val.push_back(cv.second);
    }
    P.rowptr[r + 1] = (int64_t)P.col.size();
  }
}

void space_load(const TetMesh& m, int n_modes, const double* a, const double* k, const double* phase,
                std::vector<double>& b) {
  b.assign(m.int_edges.size(), 0.0);
  const double h = m.n > 0 ? 1.0 / m.n : 1.0;   // general meshes: g are true gradients
  const double sq5 = std::sqrt(5.0);
  const double al = (5.0 + 3.0 * sq5) / 20.0, be = (5.0 - sq5) / 20.0;
  std::vector<double> kxa(3 * n_modes);
  for (int md = 0; md < n_modes; ++md) cross3(k + 3 * md, a + 3 * md, &kxa[3 * md]);
  for (int64_t t = 0; t < m.nt; ++t) {
    double g[4][3], X[4][3], vol;
    if (m.n > 0) {
      unit_gradients(m.tet_perm[t], g);
      vol = h * h * h / 6.0;
    } else {
      general_grads(m, t, g, vol);
    }
    for (int v = 0; v < 4; ++v) vertex_xyz(m, m.tet_vert[t * 4 + v], X[v]);
    for (int q = 0; q < 4; ++q) {
      double lam[4] = {be, be, be, be};
      lam[q] = al;
      double x[3] = {0, 0, 0};
      for (int v = 0; v < 4; ++v)
        for (int s = 0; s < 3; ++s) x[s] += lam[v] * X[v][s];
      double jx[3] = {0, 0, 0};
      for (int md = 0; md < n_modes; ++md) {
        const double amp = M_PI * std::cos(M_PI * dot3(k + 3 * md, x) + phase[md]);
        for (int s = 0; s < 3; ++s) jx[s] += amp * kxa[3 * md + s];
      }
      for (int le = 0; le < 6; ++le) {
        const int32_t r = m.edge_iid[m.tet_edge[t * 6 + le]];
        if (r < 0) continue;
        const int i = kLocalEdge[le][0], j = kLocalEdge[le][1];
        const double sg = m.n > 0 ? 1.0 : edge_sign(m, t, le);
        double w[3];
        for (int s = 0; s < 3; ++s) w[s] = sg * (lam[i] * g[j][s] - lam[j] * g[i][s]) / h;
        b[r] += vol / 4.0 * dot3(jx, w);
      }
    }
  }
}

// ------------------------------------------------------------------ sparse helpers
Csr csr_transpose(const Csr& A) {
  Csr T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.rowptr.assign(T.nrows + 1, 0);
  for (int32_t c : A.col) T.rowptr[c + 1]++;
  for (int32_t r = 0; r < T.nrows; ++r) T.rowptr[r + 1] += T.rowptr[r];
  T.col.resize(A.col.size());
  T.val.resize(A.col.size());
  std::vector<int64_t> next(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int32_t r = 0; r < A.nrows; ++r)
    for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; ++q) {
      const int64_t dst = next[A.col[q]]++;
      T.col[dst] = r;
      T.val[dst] = A.val[q];
    }
  return T;
}

Csr csr_multiply(const Csr& A, const Csr& B) {
  Csr C;
  C.nrows = A.nrows;
  C.ncols = B.ncols;
  C.rowptr.assign(C.nrows + 1, 0);
  std::vector<double> acc(B.ncols, 0.0);
  std::vector<char> used(B.ncols, 0);
  std::vector<int32_t> cols;
  for (int32_t r = 0; r < A.nrows; ++r) {
    cols.clear();
    for (int64_t qa = A.rowptr[r]; qa < A.rowptr[r + 1]; ++qa) {
      const int32_t k = A.col[qa];
      const double av = A.val[qa];
      for (int64_t qb = B.rowptr[k]; qb < B.rowptr[k + 1]; ++qb) {
        const int32_t c = B.col[qb];
        if (!used[c]) { used[c] = 1; cols.push_back(c); }
        acc[c] += av * B.val[qb];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t c : cols) {
      C.col.push_back(c);
      C.val.push_back(acc[c]);
      acc[c] = 0.0;
      used[c] = 0;
    }
    C.rowptr[r + 1] = (int64_t)C.col.size();
  }
  return C;
}

Csr csr_galerkin(const Csr& P, const Csr& A) {
  Csr AP = csr_multiply(A, P);
  Csr Pt = csr_transpose(P);
  return csr_multiply(Pt, AP);
}

Csr nodal_from_gradient(const Csr& M, const std::vector<int32_t>& tail, const std::vector<int32_t>& head,
                        int32_t nnodes) {
  Csr G = gradient_csr(tail, head, nnodes);
  return csr_galerkin(G, M);
}

}  // namespace stmg
