// Host-side data structures of the space-time multigrid library: meshes, sparse
// matrices, nested-dissection LDL^T factors.  Device code never includes this.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace stmg {

struct cplx {
  double re = 0.0, im = 0.0;
  cplx() = default;
  cplx(double r, double i = 0.0) : re(r), im(i) {}
};
inline cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
inline cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
inline cplx operator*(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cplx operator*(double s, cplx b) { return {s * b.re, s * b.im}; }
inline cplx operator*(cplx b, double s) { return {s * b.re, s * b.im}; }
inline cplx cdiv(cplx a, cplx b) {
  double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
inline double mag2(cplx a) { return a.re * a.re + a.im * a.im; }
inline double mag2(double a) { return a * a; }

// Compressed sparse rows, columns sorted within a row.
struct Csr {
  int32_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)col.size(); }
};

// Tetrahedral mesh: the Kuhn mesh of [0,1]^3 with n cubes per side, or (n == 0) a
// general mesh given by coordinates, possibly a red refinement of a coarser one
// (conventions in include/st_mg.h).
struct TetMesh {
  int n = 0;                               // Kuhn cubes per side; 0 for a general mesh
  int64_t nv = 0, ne = 0, nt = 0;
  std::vector<int32_t> edge_lo, edge_hi;   // [ne]
  std::vector<int32_t> tet_vert;           // [nt*4] chain order
  std::vector<int32_t> tet_edge;           // [nt*6] local edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
  std::vector<int32_t> tet_perm;           // [nt] axis permutation index 0..5 (Kuhn)
  std::vector<int32_t> edge_of;            // [nv*7] edge id from vertex lo in direction code d, or -1 (Kuhn)
  std::vector<double> xyz;                 // [nv*3] coordinates (general meshes)
  std::vector<int32_t> parent;             // [nt] tet of the mesh this one refines, or empty
  std::vector<int32_t> edge_iid;           // [ne] interior index or -1
  std::vector<int32_t> int_edges;          // interior index -> edge id
  std::vector<int32_t> vert_iid;           // [nv] interior index or -1
  std::vector<int32_t> int_verts;
  int vid(int i, int j, int k) const { return i + (n + 1) * (j + (n + 1) * k); }
  void vijk(int v, int& i, int& j, int& k) const {
    i = v % (n + 1); j = (v / (n + 1)) % (n + 1); k = v / ((n + 1) * (n + 1));
  }
};

extern const int kPerm[6][3];      // axis permutations, lexicographic
extern const int kDir[7][3];       // edge direction codes, sorted by vertex-id offset
extern const int kLocalEdge[6][2];

// bc 0: Dirichlet u x n = 0 (interior edges and vertices are the unknowns);
// bc 1: Neumann (all edges; all vertices but vertex 0, which grounds the singular
// nodal matrix -- G annihilates constants, so the correction G z is unchanged)
void build_kuhn(int n, TetMesh& m, int bc = 0);
// General mesh from coordinates and tets (vertex order kept).  Returns 0, or 1 with a
// message in err for an invalid mesh (index out of range, a vertex in no tet, repeated
// vertex, zero volume, a face shared by more than two tets).
int build_general(int32_t nv, const double* xyz, int64_t nt, const int32_t* tets, int bc, TetMesh& m,
                  std::string& err);
// Red refinement of a general mesh (child k of tet t is tet 8 t + k; include/st_mg.h).
void refine_red(const TetMesh& coarse, int bc, TetMesh& fine);
// Longest edge of every tet (h_T of the coarsening rule).
std::vector<double> longest_edges(const TetMesh& m);
// Coordinates of every vertex (Kuhn or general).
void vertex_xyz(const TetMesh& m, int64_t v, double x[3]);

// Whitney edge matrices on interior edges: one CSR pattern, two value arrays.
void assemble_edge(const TetMesh& m, const double* nu, const double* sigma, Csr& M, Csr& K);
// P1 stiffness of div(sigma grad) on interior nodes.
void assemble_nodal(const TetMesh& m, const double* sigma, Csr& Kn);
// Discrete gradient on interior unknowns as (tail, head) interior node ids (-1 = boundary).
void gradient_pairs(const TetMesh& m, std::vector<int32_t>& tail, std::vector<int32_t>& head);
// Interpolation prolongation of Whitney functions, coarse (n) -> fine (2n), interior edges.
void edge_prolongation(const TetMesh& coarse, const TetMesh& fine, Csr& P);
// Space load b_e = int curl psi . w_e (4-point rule per tet), interior edges.
void space_load(const TetMesh& m, int n_modes, const double* a, const double* k,
                const double* phase, std::vector<double>& b);

// Sparse helpers.
Csr csr_transpose(const Csr& A);
Csr csr_multiply(const Csr& A, const Csr& B);
// Galerkin product P^T A P.
Csr csr_galerkin(const Csr& P, const Csr& A);
// K_n = G^T M G for G given as (tail, head) pairs.
Csr nodal_from_gradient(const Csr& M, const std::vector<int32_t>& tail,
                        const std::vector<int32_t>& head, int32_t nnodes);
// Gradient matrix G (edges x nodes, +-1) as CSR.
Csr gradient_csr(const std::vector<int32_t>& tail, const std::vector<int32_t>& head, int32_t nnodes);

// -------------------------------------------------------------- factorisation
// Nested-dissection supernodal LDL^T without pivoting of a symmetric (real) or
// complex-symmetric matrix, stored for the GPU as one dense block per supernode:
//   W_s = [ L11^{-1} ; -L21 L11^{-1} ]   ((nc + nr) x nc, row-major)
// so that the forward step of node s is [y_s ; g_s] = W_s f_s and the backward
// step is x_s = W_s^T [z_s ; x(rows)].
template <typename T>
struct SupernodalFactor {
  int32_t n = 0;                        // matrix order
  std::vector<int32_t> perm;            // perm[k] = original index at position k
  std::vector<int32_t> iperm;           // iperm[i] = position of original index i
  struct Node {
    int32_t col0 = 0, nc = 0, nr = 0;   // columns [col0, col0+nc) in permuted order
    int32_t depth = 0, parent = -1;
    int64_t w_off = 0;                  // offset of W_s (elements of T)
    int64_t row_off = 0;                // offset of struct(s) in rows[]
    int64_t u_off = 0;                  // first update-buffer row of this node
    int32_t child[2] = {-1, -1};
  };
  std::vector<Node> nodes;              // postorder
  std::vector<int32_t> rows;            // struct(s), permuted indices, sorted
  std::vector<T> W;                     // all W_s
  std::vector<T> Dinv;                  // [n] inverse pivots, permuted order
  // forward gather table: for node s, position p in [0, nc+nr): update-buffer rows
  // of children contributing to that position (-1 if none), two per position
  std::vector<int64_t> gather_off;      // per node offset into gsrc (in positions)
  std::vector<int32_t> gsrc;            // [sum (nc+nr)] * 2
  int32_t max_depth = 0;
  int64_t u_rows = 0;                   // total update-buffer rows
  double flops_apply_per_rhs = 0;       // multiply-adds (real or complex) of one forward+backward per rhs
};

struct NDCoords {                        // position of each unknown (edge midpoint, vertex)
  std::vector<double> rx, ry, rz;
};

// Factor A (pattern Csr with values given separately as T) with ND ordering from
// coords, using up to nthreads host threads inside large fronts.  Returns 0, or 1
// (structural error) / 6 (zero pivot) with a message in err.
template <typename T>
int factor_nd_threads(const Csr& pattern, const std::vector<T>& values, const NDCoords& c,
                      int leaf_max, SupernodalFactor<T>& F, std::string& err, int nthreads);

}  // namespace stmg
