/*
 * st_mg_serve.h -- request loop (continuous batching) over the space-time multigrid
 * library of st_mg.h.  No counterpart in the paper: the paper solves one problem at a
 * time on a CPU cluster; this is the serving structure around its solver.
 *
 * A request asks for the solution, to a relative residual rtol, of one eddy-current
 * problem  s sigma dA/dt + curl(nu curl A) = J  on a registered Kuhn mesh (nu, sigma
 * registered per mesh; s = sigma_scale), with N_t slabs of length tau and DG degree
 * 0 or 1, and J given by the seeded excitation modes of st_mg_assemble_load.
 *
 * Canonical time scale.  Substituting t = s t' turns the request into the same
 * equation with conductivity sigma, slab length tau / s and horizon N_t tau / s,
 * whose load is the request's load divided by s (the time profile of J depends on
 * t / T only) and whose solution vector is the request's, unchanged.  Requests are
 * therefore grouped into classes keyed by (mesh, degree, N_t, tau / s); each class
 * is one batched handle (st_mg_problem.n_batch = slots) whose slab factors come from
 * the process-wide factor cache keyed by (mesh, space level, degree, tau / s 2^l,
 * precision), so classes that differ only in N_t share their factors.
 *
 * Continuous batching.  Every class runs its own pipeline of V-cycles on its own
 * CUDA stream; st_mg_server_step, without waiting for classes still on the device,
 * (1) finishes class builds whose host phase (st_mg_setup_begin, run on a worker
 * thread) is done, (2) collects the classes whose V-cycle has finished (per-slot
 * residual norms, copied to pinned memory behind the cycle) and retires slots that
 * reached rtol or max_cycles -- the solution is copied to the host, the slot zeroed
 * and freed, (3) admits queued requests into free slots of idle classes -- load
 * assembled into the slot, iterate zeroed -- creating a class when the device-memory
 * budget allows (evicting idle classes and unused cached factors first), and (4)
 * queues the next V-cycle, residual and norms of every idle class with occupied
 * slots.  Small classes thus advance at their own pace beside large ones.  A
 * problem's iterates do not depend on the other slots of its batch (the batched
 * operators act on each problem's columns separately), so a result is the same alone
 * and in the mix.
 *
 * The server is driven by one host thread (it is not thread safe); it uses the
 * device that was current at st_mg_server_create.
 */
#ifndef ST_MG_SERVE_H
#define ST_MG_SERVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_mg_server_s* st_mg_server_t;

typedef struct {
    int32_t slots;           /* problems per class handle (its n_batch), >= 1 */
    int64_t mem_budget;      /* device bytes for classes plus cached factors; 0: 80 % of the free
                                device memory at creation */
    int32_t max_cycles;      /* V-cycles after which a request returns ST_MG_ERR_NOT_CONVERGED */
    int32_t slab_prec;       /* st_mg_options.slab_prec for DG(1) classes; DG(0) classes use 1 (FP32)
                                when this is 3 or 4 (the tensor-core paths are DG(1) only) */
    int32_t nu;              /* V(nu, nu) cycle */
    double omega;            /* smoother damping */
    int32_t setup_threads;   /* host threads per class build (0: all cores) */
    int32_t keep_x;          /* 1: copy every solution to the host for st_mg_server_result */
    int32_t max_builds;      /* class builds (host phases) running at once, >= 1 (host memory and
                                cores: each factorises on all threads) */
} st_mg_server_options;

typedef struct {
    int32_t n_cube;          /* a mesh registered with st_mg_server_set_materials */
    int32_t degree;          /* 0 | 1 */
    int32_t N_t;             /* slabs, a power of two */
    double tau;              /* slab length (> 0); the horizon is N_t tau */
    double sigma_scale;      /* s > 0: conductivity s * the registered sigma */
    int32_t n_modes;         /* excitation as st_mg_assemble_load (copied at submission) */
    const double* a;         /* [n_modes][3] */
    const double* k;         /* [n_modes][3] */
    const double* phase;     /* [n_modes] */
    double rtol;             /* relative residual target (> 0) */
    double t_arrival;        /* arrival time, seconds on the monotonic clock (CLOCK_MONOTONIC);
                                <= 0: the time of submission */
} st_mg_request;

typedef struct {
    int64_t id;
    int32_t state;           /* 0 queued, 1 on the device (or its class is being built), 2 done */
    int32_t status;          /* when done: ST_MG_OK, ST_MG_ERR_NOT_CONVERGED, ST_MG_ERR_DIVERGED, or the
                                error of its class build */
    int32_t cycles;          /* V-cycles run for it */
    double rel_res;          /* ||f - L x|| / ||f|| at the end */
    double t_arrival, t_admit, t_done;   /* monotonic seconds */
    int64_t n_edge;          /* interior edges of its mesh */
    int64_t n_values;        /* length of its solution: n_edge * N_t * (degree + 1), layout of st_mg.h */
} st_mg_result;

typedef struct {
    int64_t submitted, completed, queued, active;
    int32_t classes, building;       /* resident class handles; of them, builds in progress */
    int64_t class_bytes;             /* device bytes of the class handles and their vectors */
    int64_t cache_bytes;             /* device bytes of the factor cache */
    int32_t cache_entries;
    int64_t cache_hits, cache_misses;
    int64_t vcycles;                 /* class V-cycles run (one covers every slot of a class) */
    int64_t slot_cycles;             /* of them, occupied slot V-cycles */
    int64_t dofs_smoothed;           /* sum over V-cycles of the occupied slots' space-time DoFs */
    int64_t evictions, deferrals;    /* classes evicted for memory; admissions put off for memory */
} st_mg_server_stats;

int st_mg_server_default_options(st_mg_server_options* opt);
int st_mg_server_create(const st_mg_server_options* opt, st_mg_server_t* out);

/* Register a mesh: Kuhn mesh n_cube^3 with n_space_levels nested levels and nu, sigma per
 * finest tet (host arrays of 6 n_cube^3, copied).  Once per mesh. */
int st_mg_server_set_materials(st_mg_server_t srv, int32_t n_cube, int32_t n_space_levels, const double* nu,
                               const double* sigma);

/* Queue a request; *id identifies it.  Invalid requests return ST_MG_ERR_INVALID_ARG. */
int st_mg_server_submit(st_mg_server_t srv, const st_mg_request* req, int64_t* id);

/* One scheduling round (see above).  The ids of requests finished in it go to
 * done_ids[0 .. min(*n_done, cap)); *n_done = how many finished.  When no class has
 * finished and none could start, it polls for a few milliseconds before returning, so
 * a caller may loop on it. */
int st_mg_server_step(st_mg_server_t srv, int64_t* done_ids, int32_t cap, int32_t* n_done);

/* State of a request.  When it is done, x_host (may be NULL) receives min(x_cap,
 * n_values) values of its solution (if keep_x), and with release = 1 the record is
 * freed (the id is unknown afterwards). */
int st_mg_server_result(st_mg_server_t srv, int64_t id, st_mg_result* res, double* x_host, int64_t x_cap,
                        int32_t release);

int st_mg_server_stats_get(st_mg_server_t srv, st_mg_server_stats* stats);

/* Waits for class builds in progress, then frees every class (cached factors stay in
 * the factor cache; st_mg_cache_trim frees them). */
void st_mg_server_destroy(st_mg_server_t srv);

#ifdef __cplusplus
}
#endif

#endif /* ST_MG_SERVE_H */
