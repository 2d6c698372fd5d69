/*
 * st_mg.h -- C ABI of the GB300 space-time multigrid library for the transient
 * eddy-current equation  sigma dA/dt + curl(nu curl A) = J  (Neumueller and
 * Schwalsberger, "A parallel space-time multigrid method for the eddy-current
 * equation", arXiv 1911.09548).
 *
 * The library builds, on one GPU, the all-at-once space-time system of Section 2.1
 * (lowest-order Nedelec elements in space, Section 3; DG(0) = implicit Euler or
 * DG(1) in time) and applies the space-time V-cycle of Section 2.1 with the hybrid
 * smoother of Section 4 (block-Jacobi S, eq. StandardSmoother, around the nodal
 * auxiliary-space correction A, eq. AuxNodalSm) to all time slabs at once, with
 * spatial coarsening where the rule of eq. CoarseningRule allows it.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  Mesh.  The finest mesh is the Kuhn mesh of [0,1]^3 with n_cube cubes per side:
 *    vertex (i,j,k) has id i + (n+1)(j + (n+1)k); cube (ci,cj,ck) has id
 *    ci + n(cj + n ck) and holds tets 6*cube + p, p = 0..5 indexing the axis
 *    permutations (x,y,z) in lexicographic order; the tet of permutation (a,b,c)
 *    is the vertex chain corner, +e_a, +e_b, +e_c.  Edges are sorted vertex pairs
 *    (lo, hi), numbered lexicographically and oriented lo -> hi.  Coarser space
 *    levels are the Kuhn meshes n/2, n/4, ... (uniform refinement, Section 5.1).
 *    Alternatively (st_mg_problem.mesh) a general start mesh refined uniformly; its
 *    conventions are given with st_mg_mesh below; edges are numbered the same way.
 *  Boundary.  Homogeneous Dirichlet u x n = 0 (default): unknowns are the interior
 *    edges (edges not contained in a boundary face), in increasing edge id order;
 *    Neumann (st_mg_problem.bc = 1): all edges in edge id order.
 *  Space-time vectors (f, x, r) of a time level with N_t slabs and degree p are
 *    double arrays  v[e * (N_t*(p+1)) + n*(p+1) + i]  -- edge-major, time
 *    contiguous -- for interior edge e, slab n, time basis function i
 *    (p = 1: Legendre phi_0 = 1, phi_1 = 2s - 1 on the slab, s in [0,1]).
 *  Nodal vectors use the same layout over interior vertices.
 *  Pointers named *_dev are device pointers (cudaMalloc / torch CUDA memory) on
 *  the device that was current at st_mg_setup; they are read/written on the
 *  handle's stream and the call returns after the work is queued unless it says
 *  otherwise.  The caller owns every buffer it passes; the handle owns all device
 *  memory it allocates (matrices, factors, workspace) until st_mg_destroy.
 *  Errors.  Every function returns an int status (ST_MG_OK = 0); no exception or
 *  abort crosses the ABI.  st_mg_last_error() gives a message for the calling
 *  thread's last failure.  A handle is not thread safe.
 */
#ifndef ST_MG_H
#define ST_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ST_MG_OK                0
#define ST_MG_ERR_INVALID_ARG   1
#define ST_MG_ERR_OOM           2
#define ST_MG_ERR_CUDA          3
#define ST_MG_ERR_DIVERGED      4
#define ST_MG_ERR_NOT_CONVERGED 5
#define ST_MG_ERR_NUMERIC       6   /* zero pivot in a factorisation */
#define ST_MG_ERR_TIMEOUT       7   /* a bounded device wait gave up (results of the call invalid) */

typedef struct st_mg_s* st_mg_t;

/* A general start mesh (Section 5.1: the spatial hierarchy comes from uniform refinement
 * of a coarse tetrahedral mesh).  Host arrays, read during setup only (the handle copies
 * what it needs).  The mesh must be conforming (a face belongs to one or two tets) with
 * tets of non-zero volume.  Each refinement is the red refinement of J. Bey (Computing 55,
 * 1995): coarse vertex ids are kept; the midpoint of coarse edge e (edges = sorted vertex
 * pairs numbered lexicographically) gets id n_vert + e; child k of coarse tet t is tet
 * 8 t + k with vertices, in terms of the parent's vertex order x0..x3 and midpoints x_ij:
 *   k=0 (x0,x01,x02,x03)   k=1 (x01,x1,x12,x13)  k=2 (x02,x12,x2,x23)   k=3 (x03,x13,x23,x3)
 *   k=4 (x01,x02,x03,x13)  k=5 (x01,x02,x12,x13) k=6 (x02,x03,x13,x23)  k=7 (x02,x12,x13,x23)
 * The boundary is the set of faces of one tet only; with bc = 0 the unknowns are the edges
 * and vertices on no boundary face. */
typedef struct {
    int32_t n_vert;          /* vertices of the start mesh (>= 4) */
    int32_t n_tet;           /* tets of the start mesh (>= 1) */
    const double* xyz;       /* host [n_vert * 3] coordinates */
    const int32_t* tet;      /* host [n_tet * 4] vertex ids in [0, n_vert), distinct per tet; every
                                vertex belongs to some tet */
    int32_t n_refine;        /* refinements to the finest mesh (0 .. 8; n_tet 8^n_refine <= 2^28) */
} st_mg_mesh;

/* Problem statement (Section 3, eq. EddyCurrent; Section 2.1 time stepping). */
typedef struct {
    int32_t n_cube;          /* cubes per side of the finest Kuhn mesh (>= 2, even if n_space_levels > 1);
                                ignored when mesh is given */
    int32_t n_space_levels;  /* nested meshes n_cube, n_cube/2, ... (or the finest general mesh and its
                                n_space_levels - 1 coarser ancestors, <= n_refine + 1) for coarsening (>= 1) */
    const double* nu;        /* host [n_tet] reluctivity 1/mu per finest tet, > 0 (n_tet = 6 n_cube^3, or
                                mesh->n_tet 8^n_refine in the child order above) */
    const double* sigma;     /* host [n_tet] conductivity per finest tet, > 0 */
    double T;                /* end time (> 0); the time interval is (0, T) */
    int32_t N_t;             /* number of time slabs on the finest level (>= 1) */
    int32_t degree;          /* DG degree in time: 0 (implicit Euler) or 1 */
    int32_t n_batch;         /* independent problems (right-hand sides) on the same mesh, materials
                                and time grid, solved together (0 or 1: one).  Vectors then hold
                                v[e * (B N_t q) + b * (N_t q) + n q + i] for problem b; needs N_t a
                                power of two (time coarsened to one slab per problem) */
    int32_t bc;              /* boundary condition (Section 3): 0 homogeneous Dirichlet u x n = 0 (the
                                unknowns are the interior edges, the nodal space the interior
                                vertices); 1 Neumann (all edges; all vertices but vertex 0, which
                                grounds the singular nodal matrix: G annihilates constants, so the
                                correction G z does not depend on the choice) */
    const st_mg_mesh* mesh;  /* NULL: the Kuhn mesh of the unit cube with n_cube cubes per side;
                                else a general start mesh refined mesh->n_refine times */
    const int32_t* batch_nt; /* NULL: every problem of a batch has N_t slabs.  Else (n_batch > 1) host
                                [n_batch]: problem b has batch_nt[b] slabs of step T / batch_nt[b] over
                                the same horizon T, batch_nt[b] = N_t / 2^k (a "ragged" batch, N_t =
                                the largest).  Problem b then enters the time hierarchy at the level
                                whose step is its own, and every level holds the problems that have
                                entered with that level's slab count, so the levels share one slab
                                factor each and one V-cycle advances every problem by one of its own
                                V-cycles.  The caller's f and x hold, per edge row, the problems one
                                after the other: problem b at columns sum_{b' < b} batch_nt[b'] q + n q
                                + i.  Needs time-only coarsening (coarsen = 1, or n_space_levels = 1).
                                st_mg_vcycle, st_mg_solve(_host), st_mg_assemble_load_batch and
                                st_mg_sizes use that layout; the per-level step entry points act on a
                                level's own layout (its problems' columns, level_info's N_t each);
                                st_mg_batch_norms, st_mg_batch_zero and st_mg_vcycle_residual_async
                                are not available */
} st_mg_problem;

/* Method parameters (Sections 2.1, 2.2, 4, 5). */
typedef struct {
    double omega;            /* damping of the block-Jacobi smoother S (paper: 0.5) */
    int32_t nu_pre;          /* pre-smoother S^nu_pre A S^nu_pre */
    int32_t nu_post;         /* post-smoother S^nu_post A S^nu_post */
    double lambda_crit;      /* coarsening rule threshold (paper: 0.1) */
    int32_t coarsen;         /* 0: eq. CoarseningRule, 1: time only ("Semi-time"),
                                2: space on the first transition only ("Full", Table FullMethod) */
    int32_t max_levels;      /* cap on the number of time levels (2 = two-grid); 0 = no cap */
    int32_t min_coarse_slabs;/* stop coarsening at <= this many slabs (>= 1) */
    int32_t nodal_solve;     /* 0: exact K_n^{-1} (factor), 1: damped Jacobi sweeps (weight 2/3) */
    int32_t nodal_jacobi_sweeps;
    int32_t use_A;           /* 1: hybrid smoother with A; 0: plain S only */
    int32_t setup_threads;   /* host threads for the factorisations; 0 = all cores */
    int32_t slab_prec;       /* slab-solve arithmetic: 0 FP64; 1 mixed: the FP64 factor rounded to
                                FP32 and applied in FP32 on every level but the coarsest (residual
                                FP64-accurate, factorisation and coarsest solve FP64, nodal K_n solve
                                FP32; the V-cycle acts as iterative refinement, Section 2.1's
                                premise that the slab inverse need only be approximated well);
                                2 double-float: the factor as FP32 (hi, lo) pairs applied with
                                error-free FP32 products and sums (about 48 significant bits), on the
                                FP32 pipes, which on GB300 run 58x the FP64 rate;
                                3 (DG(1) only) BF16 factor on the tensor cores (tcgen05, FP32
                                accumulation in tensor memory), coarsest level in FP64, nodal K_n
                                solve FP32 as in 1;
                                4 (DG(1) only) as 3 with an FP16 factor and FP16 operands: each
                                right-hand-side column of a slab solve is scaled by a power of two
                                into [1, 2) before the solve and back after it, since FP16 keeps 11
                                significant bits but only 5 exponent bits (a factor entry above 16384
                                in magnitude fails setup with ST_MG_ERR_NUMERIC).
                                Mode 2 solves K_n in double-float, mode 0 in FP64 */
    int32_t residual_prec;   /* space-time residual arithmetic: 0 FP64; 2 double-float (x split into
                                FP32 pairs once per call, error-free products and sums, f and r in
                                FP64); 1 FP32 inside the V-cycle: each V-cycle runs in correction form
                                (r = f - L x in double-float, e = V(r) from e = 0 with every residual
                                of the V-cycle in FP32 arithmetic on an FP32 copy of its iterate, then
                                x += e), while st_mg_solve's stopping test, st_mg_residual and the
                                correction's r stay double-float (the iteration's fixed point is
                                unchanged; the FP32 rounding is relative to r, which shrinks);
                                -1 (default): FP64 when slab_prec = 0, double-float otherwise */
    int32_t use_graph;       /* 1 (default): st_mg_vcycle / st_mg_solve capture the V-cycle's fixed
                                launch sequence into a CUDA graph once per (f, x) buffer pair and replay
                                it (needs a non-default stream; the first call captures, later calls
                                replay); 0: launch kernel by kernel */
    char smoother[16];       /* hybrid smoother as a product of S and A in the paper's notation, read
                                right to left (Section 4: "SA" applies A, then S), NUL-terminated, at
                                most 15 letters: the pre-smoother applies it right to left, the
                                post-smoother the same factors left to right.  Empty (default):
                                S^nu_pre A S^nu_pre and S^nu_post A S^nu_post (A only if use_A) */
    int32_t persistent_split;/* How slab and K_n solves with few right-hand sides (coarse time levels)
                                walk the tree depths: 0 two launches (product, reduction) per depth
                                and sweep; 1 one cooperative launch per sweep with grid barriers
                                between depths; 2 one launch per sweep in which every task waits only
                                for the tasks it reads from (children forward, parent backward).
                                Results are identical in all three. */
    int32_t factor_cache;    /* 1: take slab and K_n factors from, and leave new ones in, the
                                process-wide factor cache (key: device, mesh, space level, materials,
                                DG degree, tau, precision), so handles that share a mesh and a tau
                                share one device copy; 0 (default): the handle owns its factors */
    int32_t autotune;        /* 1: at setup, time each time level's slab solve for several tiled /
                                split-K thresholds (a tree depth whose tiles fill fewer than w waves
                                of the SMs runs split-K; w in {0, 1, 2, 4, 8, 16, 32}) and keep the fastest
                                per level (results change at rounding level, by the summation order
                                of the chosen kernels); 0 (default): w = 2 */
    int32_t nd_leaf;         /* nested dissection of the slab matrices stops at sets of at most this
                                many unknowns (the leaf supernodes); 0 (default): 512 with slab_prec 3
                                (BF16 solves are bound by the latency of the tree's dependent depths),
                                else 64 (the other solves are bound by arithmetic, so the least fill
                                wins).  Larger leaves mean a shallower tree and more fill */
    int32_t split_k;         /* K columns (unknowns of a supernode's column range) of one split-K work
                                item of the supernodal products (a warp multiplies kSkRows = 32 rows by
                                this many columns, then a fixed-order reduction sums the items of a
                                row block): 16 .. 1024, a multiple of 16; 0 (default): 32.  Narrower
                                items mean more items in flight and a shorter chain per item, more
                                partial sums to reduce; results change at rounding level */
    int32_t tc_split_k;      /* the same for the tensor-core split-K items of the 16-bit factors
                                (slab_prec 3, 4; complex columns, a multiple of the 32-column MMA
                                stage, 32 .. 4096); 0 (default): 256 */
} st_mg_options;

/* Fill *opt with the paper's defaults: omega 0.5, V(1,1), lambda_crit 0.1,
 * coarsening by the rule, no level cap, exact nodal solve, A on. */
int st_mg_default_options(st_mg_options* opt);

/* Build the hierarchy: meshes, matrices M_sigma, K_nu, G, K_n (Section 3,
 * eq. AuxNodalSm), spatial prolongations, the time levels with the coarsening
 * decision of eq. CoarseningRule, and one slab factor per time level (every slab
 * of a level shares A_slab, Section 2.1) plus one K_n factor per space level,
 * all uploaded to the current device.  `stream` is a cudaStream_t (NULL = legacy
 * default stream) used by every later call.  Host work (assembly and the sparse
 * factorisations) runs on setup_threads threads.  On success *out owns all of it. */
int st_mg_setup(const st_mg_problem* prob, const st_mg_options* opt, void* stream, st_mg_t* out);

/* st_mg_setup in two phases, for callers that build handles off their critical path.
 * st_mg_setup_begin does the host work (meshes, assembly, coarsening decisions,
 * factorisations, factor-cache lookups) and touches no device memory, so it may run
 * on any host thread that has made the target device current; the handle it returns
 * accepts only st_mg_setup_finish and st_mg_destroy.  st_mg_setup_finish uploads and
 * sizes the workspaces (device current = the handle's device; it synchronises the
 * legacy default stream).  st_mg_setup = begin + finish.  No counterpart in the paper. */
int st_mg_setup_begin(const st_mg_problem* prob, const st_mg_options* opt, void* stream, st_mg_t* out);
int st_mg_setup_finish(st_mg_t h);

/* Host-only variant of st_mg_setup for inspecting the setup without a GPU: builds
 * the meshes, matrices, hierarchy and factors on the host and allocates no device
 * memory.  Such a handle accepts only st_mg_sizes, st_mg_level_info,
 * st_mg_debug_get, st_mg_debug_host_slab_solve and st_mg_destroy; every other
 * call returns ST_MG_ERR_INVALID_ARG. */
int st_mg_setup_host(const st_mg_problem* prob, const st_mg_options* opt, st_mg_t* out);

void st_mg_destroy(st_mg_t h);

/* Sizes of the finest level: interior edges, interior nodes, space-time unknowns of
 * all problems (n_edge * n_batch * N_t * (degree+1)), and the number of time levels. */
int st_mg_sizes(st_mg_t h, int64_t* n_edge, int64_t* n_node, int64_t* n_dof, int32_t* n_levels);

/* Time level `level` (0 = finest): its space level, slab count and step tau. */
int st_mg_level_info(st_mg_t h, int32_t level, int32_t* space_level, int32_t* N_t, double* tau,
                     int64_t* n_edge, int64_t* n_node);

/* Right-hand side f on the finest level for J(x,t) = g(t) curl psi(x),
 * psi = sum_m a_m sin(pi k_m . x + phase_m), g(t) = sin(pi t / T) + 1:
 *   f[e, n, i] = int_{I_n} g phi_i dt * int_Omega curl psi . w_e dx
 * (3-point Gauss per slab, 4-point degree-2 rule per tet).  a, k: host [n_modes*3];
 * phase: host [n_modes].  f_dev: device, finest layout. */
int st_mg_assemble_load(st_mg_t h, int32_t n_modes, const double* a, const double* k,
                        const double* phase, double* f_dev);
/* The same for problem `batch` of a batched handle (st_mg_assemble_load = batch 0);
 * the other problems' entries of f_dev are left untouched. */
int st_mg_assemble_load_batch(st_mg_t h, int32_t batch, int32_t n_modes, const double* a, const double* k,
                              const double* phase, double* f_dev);

/* ---- individual steps of the hot path (each on time level `level`) ---- */

/* r = f - L x (Section 2.1: block lower-bidiagonal L with K_t(x)M + M_t(x)K on the
 * diagonal and N_t(x)M below).  If norm_out != NULL, also ||r||_2 (blocking). */
int st_mg_residual(st_mg_t h, int32_t level, const double* f_dev, const double* x_dev,
                   double* r_dev, double* norm_out);

/* y = (I (x) A_slab^{-1}) r: the slab solve of eq. StandardSmoother on every slab. */
int st_mg_slab_solve(st_mg_t h, int32_t level, const double* r_dev, double* y_dev);

/* One block-Jacobi sweep x <- x + omega (I (x) A_slab^{-1})(f - L x)  (eq. StandardSmoother). */
int st_mg_smooth_S(st_mg_t h, int32_t level, const double* f_dev, double* x_dev);

/* One nodal auxiliary-space correction x <- x + G L_t^{-1} K_n^{-1} G^T (f - L x)
 * (eq. AuxNodalSm; L_t^{-1} is the running sum Sigma_t for DG(0)). */
int st_mg_correct_A(st_mg_t h, int32_t level, const double* f_dev, double* x_dev);

/* Parts of A: y = G^T r (edge -> node, per time unknown);  z = K_n^{-1} y (or the
 * Jacobi sweeps of the options);  w = L_t^{-1} z (time integration);  x += G w. */
int st_mg_grad_T(st_mg_t h, int32_t level, const double* r_dev, double* y_dev);
int st_mg_nodal_solve(st_mg_t h, int32_t level, const double* y_dev, double* z_dev);
int st_mg_time_integrate(st_mg_t h, int32_t level, const double* z_dev, double* w_dev);
int st_mg_grad_add(st_mg_t h, int32_t level, const double* w_dev, double* x_dev);

/* Coarse-grid transfers between level and level+1: time (pairs of slabs, DG
 * prolongation blocks) and, where the hierarchy coarsens space, P_x.
 * restrict: rc = (P_t (x) P_x)^T r.  prolong_add: x += (P_t (x) P_x) ec. */
int st_mg_restrict(st_mg_t h, int32_t level, const double* r_dev, double* rc_dev);
int st_mg_prolong_add(st_mg_t h, int32_t level, const double* ec_dev, double* x_dev);

/* Exact solve L x = f on the coarsest level (one slab: slab factor; several slabs:
 * forward substitution in time).  x_dev is overwritten. */
int st_mg_coarse_solve(st_mg_t h, const double* f_dev, double* x_dev);

/* ---- the whole method ---- */

/* One V-cycle on the finest level (x updated in place).  If rel_res_out != NULL,
 * also ||f - L x|| / ||f|| after the cycle (blocking). */
int st_mg_vcycle(st_mg_t h, const double* f_dev, double* x_dev, double* rel_res_out);

/* V-cycles from the given x until ||f - L x|| / ||f|| <= rtol or maxit cycles.
 * iters, rel_res: host outputs; history (nullable): host [maxit + 1] relative
 * residuals (entry 0 = start).  Returns ST_MG_ERR_NOT_CONVERGED if maxit is
 * reached, ST_MG_ERR_DIVERGED on a non-finite residual or growth above 1e3 x. */
int st_mg_solve(st_mg_t h, const double* f_dev, double* x_dev, double rtol, int32_t maxit,
                int32_t* iters, double* rel_res, double* history);

/* The same solve from HOST buffers: f_host is copied to the device, x_host is the
 * start value and receives the result; copies are part of the call (blocking). */
int st_mg_solve_host(st_mg_t h, const double* f_host, double* x_host, double rtol, int32_t maxit,
                     int32_t* iters, double* rel_res, double* history);

/* Debug getters for bit-exact checks of the setup (host buffers).
 *  what: 1 edges [ne_all*2] int32 (lo, hi) of space level `level`;
 *        2 interior edge ids [n_edge] int32;  3 interior vertex ids [n_node] int32;
 *        4 CSR row pointer of the edge matrices [n_edge+1] int64; 5 CSR columns int32;
 *        6 M_sigma values double; 7 K_nu values double;
 *        8 G as (tail, head) interior node per interior edge [n_edge*2] int32 (-1 = boundary);
 *        9 K_n row pointer int64; 10 K_n columns int32; 11 K_n values double;
 *       12 P_x (level -> level+1 coarse) row pointer int64; 13 columns int32; 14 values double.
 * With host_buf == NULL, *bytes receives the size needed. */
int st_mg_debug_get(st_mg_t h, int32_t what, int32_t level, void* host_buf, int64_t* bytes);

/* Setup check for host-only handles: y = (I (x) A_slab^{-1}) r on time level
 * `level`, evaluated on the host with the same factor and complex transformation
 * the device path uses.  r_host, y_host: host arrays in the level's layout. */
int st_mg_debug_host_slab_solve(st_mg_t h, int32_t level, const double* r_host, double* y_host);

/* Convergence rate of the V-cycle by the power iteration of Section 5.1: V-cycles with
 * f = 0 from the start x_dev (device, finest layout, overwritten by the iterates, which
 * are then the errors), the l2 norm after each (the handle's deterministic reduction);
 * rates_host[k] = ||x_{k+1}|| / ||x_k|| for the *n_rates cycles run, *rate = the largest.
 * Stops after max_iter cycles, or when the norm reaches zero or falls below floor times
 * the start's (Section 5.1 stops at a total reduction of 1e-100 against underflow).
 * rates_host: host, max_iter doubles.  Blocking. */
int st_mg_convergence_rate(st_mg_t h, double* x_dev, int32_t max_iter, double floor, double* rates_host,
                           int32_t* n_rates, double* rate);

/* Measured FP64 FMA throughput of the handle's device in TFLOP/s (about 70 ms of
 * independent FMA chains on 8 blocks per SM; blocking).  The FP64 kernels of this
 * library are bound by this pipe, so it is the roof their efficiency is quoted against. */
int st_mg_probe_fp64(st_mg_t h, double* tflops);

/* One V-cycle on x (as st_mg_vcycle, graph replay included) followed by the finest
 * residual r = f - L x, both queued on the handle's stream with no host wait.  A
 * tensor-core wait that timed out during it is reported by the next st_mg_batch_norms
 * (or any blocking call that checks).  For pipelines that overlap several handles. */
int st_mg_vcycle_residual_async(st_mg_t h, const double* f_dev, double* x_dev, double* r_dev);

/* Per-problem l2 norms of a finest-level vector of a batched handle (e.g. r from
 * st_mg_residual): norms_host[b] = ||v_b||_2 for b < n_batch, deterministic order
 * (blocking).  Lets a caller stop or replace problems of a batch independently. */
int st_mg_batch_norms(st_mg_t h, const double* v_dev, double* norms_host);

/* The same per-problem sums of squares ||v_b||^2, queued on the handle's stream into
 * norms_sq_dev (device, n_batch doubles) with no host wait. */
int st_mg_batch_norms_async(st_mg_t h, const double* v_dev, double* norms_sq_dev);

/* Blocking: ST_MG_ERR_TIMEOUT if a bounded device wait of earlier work on the handle's
 * stream gave up (the flag is then cleared), else ST_MG_OK. */
int st_mg_check(st_mg_t h);

/* Zero problem `batch`'s entries of a finest-level vector (e.g. to start a new problem
 * in a freed slot of a batch while the other problems keep iterating). */
int st_mg_batch_zero(st_mg_t h, int32_t batch, double* v_dev);

/* Device bytes of a handle: own_bytes = its buffers (vectors, workspaces, meshes);
 * factor_bytes = the slab and K_n factors it references (shared with other handles
 * when they came from the factor cache). */
int st_mg_memory(st_mg_t h, int64_t* own_bytes, int64_t* factor_bytes);

/* Factor cache (st_mg_options.factor_cache, no counterpart in the paper: a serving
 * structure).  Stats: device bytes of all resident entries, the number of entries,
 * how many of them some live handle uses, and lookup hits and misses so far.  Any
 * pointer may be NULL. */
int st_mg_cache_stats(int64_t* bytes, int32_t* entries, int32_t* in_use, int64_t* hits, int64_t* misses);

/* Evict least-recently-used entries that no live handle uses until the cache holds at
 * most max_bytes (0: every unused entry).  *bytes_after (may be NULL) = what remains. */
int st_mg_cache_trim(int64_t max_bytes, int64_t* bytes_after);

/* Tiled / split-K threshold of a time level's slab solve, in waves of SMs (2 unless
 * st_mg_options.autotune chose another). */
int st_mg_split_waves(st_mg_t h, int32_t level, int32_t* waves);

/* Set that threshold (waves in [0, 64]; 0 = tiled at every depth that has any tile),
 * e.g. to repeat the choice an earlier autotuned run made.  Drops the captured V-cycle
 * graph, which the next V-cycle re-captures.  ST_MG_ERR_INVALID_ARG outside the range. */
int st_mg_set_split_waves(st_mg_t h, int32_t level, int32_t waves);

/* ---- time-slab sharding (Section 2.1: the all-at-once system is split along time into
 * groups of consecutive slabs, one per process group; only the block-bidiagonal L couples
 * a group to the one before it, and the time integration Sigma_t / L_t^{-1} of the nodal
 * correction, eq. AuxNodalSm, is a recurrence across all of them).  A handle set up for
 * one contiguous slab range (same mesh, materials and tau; n_batch 1) computes its part
 * with the calls below; the ranks exchange only one slab of x per residual and one slab
 * of nodal values per time integration (paper_1911_09548_gb300/shard.py does the
 * exchange over torch.distributed).  No counterpart in the paper's equations beyond the
 * splitting itself. ---- */

/* out_dev[row * q + i] = v_dev[row][slab * q + i] for every edge row (nodal = 0) or node
 * row (nodal = 1) of time level `level`: one slab, e.g. the last slab of x that the next
 * range needs as its halo.  out_dev: device, rows * q doubles. */
int st_mg_slab_copy(st_mg_t h, int32_t level, int32_t nodal, const double* v_dev, int32_t slab, double* out_dev);

/* r = f - L x on this handle's slab range when the range is preceded by another: slab 0
 * also receives the coupling -(N_t (x) M) x_prev of the block-bidiagonal L, x_prev_dev the
 * last slab of x of the range before ([edge * q + i], from st_mg_slab_copy); NULL = this
 * range starts at t = 0 (same as st_mg_residual).  Needs n_batch 1. */
int st_mg_residual_halo(st_mg_t h, int32_t level, const double* f_dev, const double* x_dev, const double* x_prev_dev,
                        double* r_dev);

/* w = L_t^{-1} z (st_mg_time_integrate) continued from w_{-1} = carry_dev[node * q + i],
 * the state at the end of the preceding ranges (st_mg_time_carry); NULL = zero. */
int st_mg_time_integrate_carry(st_mg_t h, int32_t level, const double* z_dev, const double* carry_dev,
                               double* w_dev);

/* The carry into range n_prev from the ranges before it: ends_dev[k][node * q + i] is the
 * last slab of range k's own L_t^{-1} z computed from a zero carry (k < n_prev, in time
 * order); c_0 = 0, c_{k+1} = end_k + T c_k with T = -K_t^{-1} N_t (1 for DG(0),
 * [[1,1],[0,0]] for DG(1), so T^len = T for any range length).  carry_dev: node rows * q.
 * n_prev = 0 writes zeros. */
int st_mg_time_carry(st_mg_t h, int32_t level, const double* ends_dev, int32_t n_prev, double* carry_dev);

/* How a 16-bit slab factor (slab_prec 3 BF16 or 4 FP16, DG(1)) is applied on time level
 * `level` (eq. StandardSmoother's slab inverse in every mode):
 *   0 (default) the tensor-core kernels (tcgen05); a tree depth with enough tiles runs as
 *     one persistent CTA per SM that walks the depth's (row tile, column block) tasks;
 *   1 the same factor on the CUDA cores with the same operand rounding -- the gathered
 *     FP32 right-hand sides rounded to 16 bits where they enter each product, products
 *     and sums in FP32, every tree depth tiled -- so that it differs from the tensor
 *     cores only in the FP32 summation order: the element-wise reference the tensor-core
 *     kernels are tested against (slower);
 *   2 the tensor-core kernels with one CTA per tile on those depths (the same products,
 *     results identical to mode 0 bit for bit).
 * Drops the captured V-cycle graph.  ST_MG_ERR_INVALID_ARG if the level has no 16-bit
 * factor or mode is not 0, 1 or 2. */
int st_mg_set_tc_mode(st_mg_t h, int32_t level, int32_t mode);

/* Process-wide: 1 queues the library's kernels with programmatic dependent launch, so
 * that a kernel's blocks may be scheduled while the previous kernel on the same stream
 * drains (each waits for that kernel's completion and memory before it reads or writes
 * anything; results are identical); 0 (default) queues them as plain stream launches,
 * which measured faster for the V-cycle's launch sequence on GB300.
 * Applies to launches queued after the call (a V-cycle graph captured earlier keeps its
 * launches).  No counterpart in the paper: a GPU scheduling choice. */
int st_mg_set_launch_overlap(int32_t on);

/* Number of CUDA kernels this library has launched since it was loaded (all handles). */
int st_mg_launch_count(int64_t* count);

/* Slab factor of time level `level`: multiply-adds of one forward+backward solve per
 * right-hand side (complex multiply-adds for DG(1), real for DG(0); the triangular
 * blocks L11^{-1} counted once), device bytes of its dense blocks, and the depth of
 * its nested-dissection tree (the solve launches 2 (depth+1) product kernels). */
int st_mg_factor_stats(st_mg_t h, int32_t level, double* macs_per_rhs, int64_t* factor_bytes, int32_t* depth);

/* Allocation-free l2 norm: norm_dev[0] = ||v||_2 for the n doubles at v_dev, queued
 * on `stream` (a cudaStream_t; NULL = legacy default stream).  The paper has no
 * counterpart; this is a library service for callers that cannot allocate device
 * memory at the point where they need the norm -- a control loop that must not stall
 * on cudaMalloc/cudaFree (both may synchronise the whole device), or a host framework
 * that owns the device allocator and forbids allocations by libraries.  It needs no
 * handle and calls no cudaMalloc, cudaFree or other allocating routine.
 * Its reduction is its own fixed-order two-stage sum (one partial per 4096
 * consecutive elements, then the partials in index order): deterministic for a given
 * n, and equal to the solver's norm (st_mg_residual's) only up to rounding, since the
 * two sum in different orders.
 * Scratch: the partial sums live in a file-scope device array of 32768 doubles
 * (256 KiB) that every GPU which loads the library holds until the process exits;
 * hence n <= 134217728 (larger n returns ST_MG_ERR_INVALID_ARG before any launch).
 * n = 0 writes 0.
 * The first call on a device, with that device current, looks the array up with
 * cudaGetSymbolAddress and keeps the address for the life of the process; make that
 * first call before any stream capture, and do not use the entry point on a device
 * after cudaDeviceReset (the module is then loaded anew and the kept address is
 * stale).  Every call shares the array and it keeps the last call's partial sums
 * (each call overwrites the entries it reads), so calls that overlap on the GPU
 * (other streams, other threads, before an earlier call finished) race and must be
 * serialised by the caller.  v_dev and norm_dev: device pointers, 8-byte aligned;
 * the result is written on the stream (read it after synchronising that stream). */
int st_mg_norm2_noalloc(const double* v_dev, int64_t n, void* stream, double* norm_dev);

const char* st_mg_strerror(int status);
const char* st_mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ST_MG_H */
