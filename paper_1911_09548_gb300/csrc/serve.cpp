// Request loop with continuous batching over the space-time multigrid library
// (include/st_mg_serve.h).  Everything on the device goes through the public C ABI
// of include/st_mg.h: one batched handle per request class, one CUDA stream per
// class, class builds split into a host phase on a worker thread and a device phase
// on the serving thread.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <future>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/st_mg.h"
#include "../../include/st_mg_serve.h"

namespace stmg {
void set_last_error(const char* msg);
}

namespace {

int fail(int code, const std::string& msg) {
  stmg::set_last_error(msg.c_str());
  return code;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }

// all edges of the Kuhn mesh n^3 (axis, face-diagonal and body-diagonal): an upper
// bound of the interior edges, for memory estimates before a class exists
int64_t kuhn_edges(int64_t n) { return 3 * n * (n + 1) * (n + 1) + 3 * n * n * (n + 1) + n * n * n; }

struct Materials {
  int32_t nsl = 1;
  std::vector<double> nu, sigma;
};

struct Request {
  int64_t id = 0;
  int32_t n_cube = 0, degree = 0, N_t = 0;
  double tau = 0, s = 1, rtol = 0;
  std::vector<double> a, k, phase;
  std::string cls;
  int32_t state = 0, status = ST_MG_OK, cycles = 0, slot = -1;
  double rel = 1.0, fnorm = 0.0;
  double t_arrival = 0, t_admit = 0, t_done = 0;
  int64_t n_edge = 0, n_values = 0;
  std::vector<double> x;
};

struct Class {
  std::string key;
  int32_t n_cube = 0, degree = 0, N_t = 0;
  double tau_c = 0;                       // canonical slab length tau / s
  st_mg_problem prob{};
  st_mg_options opt{};
  st_mg_t h = nullptr;
  cudaStream_t stream = nullptr;
  std::future<int> build;                 // host phase on a worker thread
  std::string build_err;
  bool ready = false;
  double *f = nullptr, *x = nullptr, *r = nullptr;
  int64_t ne = 0, seg = 0, len = 0;
  int64_t est_bytes = 0, bytes = 0;
  int64_t last_use = 0;
  std::vector<int64_t> slot;              // request id per slot, -1 free
  bool in_flight = false;                 // a V-cycle + residual norms queued, not yet collected
  cudaEvent_t ev = nullptr;               // recorded after the norms' copy to the host
  double* norms_dev = nullptr;            // per-slot squared residual norms (device)
  double* norms_host = nullptr;           // the same, pinned host copy
  int occupied() const {
    int c = 0;
    for (int64_t v : slot) c += v >= 0;
    return c;
  }
};

}  // namespace

struct st_mg_server_s {
  st_mg_server_options opt{};
  int device = 0;
  std::map<int32_t, Materials> mats;
  std::map<int64_t, Request> req;
  std::deque<int64_t> queue;
  std::map<std::string, std::unique_ptr<Class>> cls;
  int64_t next_id = 1, tick = 0;
  std::map<std::string, int64_t> shape_bytes;   // measured bytes of a class per (mesh, degree, N_t)
  st_mg_server_stats st{};
};

namespace {

using Server = st_mg_server_s;

std::string class_key(int n, int deg, int N_t, double tau_c) {
  char buf[96];
  std::snprintf(buf, sizeof buf, "n%d deg%d Nt%d tau%a", n, deg, N_t, tau_c);
  return buf;
}

std::string shape_key(int n, int deg, int N_t) { return std::to_string(n) + "/" + std::to_string(deg) + "/" + std::to_string(N_t); }

// device bytes of a new class: measured on an earlier class of the same shape, else a
// bound (16 doubles per finest space-time DoF of every slot)
int64_t estimate_bytes(const Server& S, int n, int deg, int N_t) {
  auto it = S.shape_bytes.find(shape_key(n, deg, N_t));
  if (it != S.shape_bytes.end()) return it->second;
  return 16 * kuhn_edges(n) * (int64_t)N_t * (deg + 1) * S.opt.slots * (int64_t)sizeof(double);
}

int64_t cache_bytes() {
  int64_t b = 0;
  st_mg_cache_stats(&b, nullptr, nullptr, nullptr, nullptr);
  return b;
}

int64_t class_usage(const Server& S) {
  int64_t u = 0;
  for (auto& kv : S.cls) u += kv.second->ready ? kv.second->bytes : kv.second->est_bytes;
  return u;
}

void free_class(Class& c) {
  if (c.build.valid()) {
    c.build.wait();
    c.build.get();
  }
  if (c.h) st_mg_destroy(c.h);
  c.h = nullptr;
  for (double* p : {c.f, c.x, c.r, c.norms_dev})
    if (p) cudaFree(p);
  c.f = c.x = c.r = c.norms_dev = nullptr;
  if (c.norms_host) cudaFreeHost(c.norms_host);
  c.norms_host = nullptr;
  if (c.ev) cudaEventDestroy(c.ev);
  c.ev = nullptr;
  if (c.stream) cudaStreamDestroy(c.stream);
  c.stream = nullptr;
}

// Evict idle classes (least recently used first) and unused cached factors until
// `need` more bytes fit in the budget.  Classes with queued requests stay.
void make_room(Server& S, int64_t need) {
  auto fits = [&]() { return class_usage(S) + cache_bytes() + need <= S.opt.mem_budget; };
  if (fits()) return;
  std::vector<std::string> wanted;
  for (int64_t id : S.queue) wanted.push_back(S.req[id].cls);
  for (;;) {
    int64_t room = S.opt.mem_budget - class_usage(S) - need;
    st_mg_cache_trim(std::max<int64_t>(room, 0), nullptr);
    if (fits()) return;
    Class* victim = nullptr;
    for (auto& kv : S.cls) {
      Class& c = *kv.second;
      if (!c.ready || c.occupied() > 0) continue;
      if (std::find(wanted.begin(), wanted.end(), c.key) != wanted.end()) continue;
      if (!victim || c.last_use < victim->last_use) victim = &c;
    }
    if (!victim) return;
    free_class(*victim);
    S.cls.erase(victim->key);
    ++S.st.evictions;
  }
}

void finish_request(Server& S, Request& q, int status, std::vector<int64_t>& done) {
  q.status = status;
  q.state = 2;
  q.t_done = now_s();
  q.slot = -1;
  ++S.st.completed;
  done.push_back(q.id);
}

// Start a class: stream now, host phase of the setup on a worker thread.
Class* start_class(Server& S, const Request& q) {
  auto c = std::make_unique<Class>();
  c->key = q.cls;
  c->n_cube = q.n_cube;
  c->degree = q.degree;
  c->N_t = q.N_t;
  c->tau_c = q.tau / q.s;
  const Materials& m = S.mats.at(q.n_cube);
  c->prob.n_cube = q.n_cube;
  c->prob.n_space_levels = m.nsl;
  c->prob.nu = m.nu.data();
  c->prob.sigma = m.sigma.data();
  c->prob.T = c->tau_c * q.N_t;
  c->prob.N_t = q.N_t;
  c->prob.degree = q.degree;
  c->prob.n_batch = S.opt.slots;
  st_mg_default_options(&c->opt);
  c->opt.omega = S.opt.omega;
  c->opt.nu_pre = c->opt.nu_post = S.opt.nu;
  c->opt.slab_prec = (S.opt.slab_prec >= 3 && q.degree == 0) ? 1 : S.opt.slab_prec;
  c->opt.setup_threads = S.opt.setup_threads;
  c->opt.factor_cache = 1;
  c->opt.use_graph = 1;
  c->slot.assign(S.opt.slots, -1);
  c->est_bytes = estimate_bytes(S, q.n_cube, q.degree, q.N_t);
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  Class* cp = c.get();
  const int dev = S.device;
  cp->build = std::async(std::launch::async, [cp, dev]() {
    cudaSetDevice(dev);
    const int rc = st_mg_setup_begin(&cp->prob, &cp->opt, cp->stream, &cp->h);
    if (rc != ST_MG_OK) cp->build_err = st_mg_last_error();
    return rc;
  });
  S.cls[cp->key] = std::move(c);
  return cp;
}

// Device phase of a class whose host phase is done.  Returns the build status.
int finish_class(Server& S, Class& c) {
  int rc = c.build.get();
  if (rc == ST_MG_OK) rc = st_mg_setup_finish(c.h);
  if (rc != ST_MG_OK) {
    if (c.build_err.empty()) c.build_err = st_mg_last_error();
    return rc;
  }
  int64_t ne = 0, nd = 0;
  int32_t nl = 0;
  st_mg_sizes(c.h, &ne, nullptr, &nd, &nl);
  c.ne = ne;
  c.seg = (int64_t)c.N_t * (c.degree + 1);
  c.len = nd;
  for (double** p : {&c.f, &c.x, &c.r}) {
    if (cudaMalloc(p, (size_t)c.len * sizeof(double)) != cudaSuccess) {
      c.build_err = "cudaMalloc of the class vectors";
      return ST_MG_ERR_OOM;
    }
    if (cudaMemsetAsync(*p, 0, (size_t)c.len * sizeof(double), c.stream) != cudaSuccess) return ST_MG_ERR_CUDA;
  }
  if (cudaMalloc(&c.norms_dev, c.slot.size() * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c.norms_host, c.slot.size() * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming) != cudaSuccess) {
    c.build_err = "per-class norm buffers";
    return ST_MG_ERR_OOM;
  }
  int64_t own = 0, fac = 0;
  st_mg_memory(c.h, &own, &fac);
  c.bytes = own + 3 * c.len * (int64_t)sizeof(double);
  S.shape_bytes[shape_key(c.n_cube, c.degree, c.N_t)] = c.bytes;
  c.ready = true;
  c.last_use = ++S.tick;
  return ST_MG_OK;
}

int step(Server& S, std::vector<int64_t>& done) {
  // nothing on the device but builds in progress: wait a little for one of them
  // rather than return at once (a caller looping on step would spin against the
  // factorisation threads)
  {
    bool occupied = false;
    Class* building = nullptr;
    for (auto& kv : S.cls) {
      occupied = occupied || kv.second->occupied() > 0;
      if (!kv.second->ready && kv.second->build.valid()) building = kv.second.get();
    }
    if (!occupied && building) building->build.wait_for(std::chrono::milliseconds(5));
  }
  // (1) class builds whose host phase finished
  std::vector<std::string> failed;
  for (auto& kv : S.cls) {
    Class& c = *kv.second;
    if (c.ready || !c.build.valid()) continue;
    if (c.build.wait_for(std::chrono::seconds(0)) != std::future_status::ready) continue;
    const int rc = finish_class(S, c);
    if (rc != ST_MG_OK) {
      for (auto it = S.queue.begin(); it != S.queue.end();) {
        Request& q = S.req[*it];
        if (q.cls == c.key) {
          finish_request(S, q, rc, done);
          it = S.queue.erase(it);
        } else {
          ++it;
        }
      }
      failed.push_back(c.key);
    }
  }
  for (auto& k : failed) {
    free_class(*S.cls[k]);
    S.cls.erase(k);
  }
  if (class_usage(S) + cache_bytes() > S.opt.mem_budget) make_room(S, 0);

  // (2) collect the classes whose V-cycle has finished: per-slot residual norms,
  // retire slots that reached rtol or max_cycles
  bool progressed = false;
  for (auto& kv : S.cls) {
    Class& c = *kv.second;
    if (!c.in_flight) continue;
    const cudaError_t q = cudaEventQuery(c.ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return fail(ST_MG_ERR_CUDA, cudaGetErrorString(q));
    c.in_flight = false;
    progressed = true;
    if (int rc = st_mg_check(c.h)) return rc;
    ++S.st.vcycles;
    for (size_t b = 0; b < c.slot.size(); ++b) {
      if (c.slot[b] < 0) continue;
      Request& q2 = S.req[c.slot[b]];
      ++q2.cycles;
      ++S.st.slot_cycles;
      S.st.dofs_smoothed += c.ne * c.seg;
      q2.rel = std::sqrt(c.norms_host[b]) / q2.fnorm;
      int status = -1;
      if (!std::isfinite(q2.rel)) status = ST_MG_ERR_DIVERGED;
      else if (q2.rel <= q2.rtol) status = ST_MG_OK;
      else if (q2.cycles >= S.opt.max_cycles) status = ST_MG_ERR_NOT_CONVERGED;
      if (status < 0) continue;
      if (S.opt.keep_x) {
        q2.x.resize((size_t)q2.n_values);
        const size_t w = (size_t)c.seg * sizeof(double);
        if (cudaMemcpy2DAsync(q2.x.data(), w, c.x + (int64_t)b * c.seg, w * c.slot.size(), w, (size_t)c.ne,
                              cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess)
          return fail(ST_MG_ERR_CUDA, "copy of a solution to the host");
      }
      if (int rc = st_mg_batch_zero(c.h, (int)b, c.f)) return rc;
      if (int rc = st_mg_batch_zero(c.h, (int)b, c.x)) return rc;
      c.slot[b] = -1;
      finish_request(S, q2, status, done);
    }
    c.last_use = ++S.tick;
  }

  // (3) admission into free slots of idle classes, first come first served within a
  // class; new classes when the memory budget allows
  std::vector<Class*> admitted;
  for (auto it = S.queue.begin(); it != S.queue.end();) {
    Request& q = S.req[*it];
    auto ci = S.cls.find(q.cls);
    Class* c = ci == S.cls.end() ? nullptr : ci->second.get();
    if (!c) {
      int building = 0;
      for (auto& kv : S.cls) building += kv.second->ready ? 0 : 1;
      if (building >= S.opt.max_builds) {   // wait for a build slot
        ++it;
        continue;
      }
      const int64_t need = estimate_bytes(S, q.n_cube, q.degree, q.N_t);
      make_room(S, need);
      bool busy = false;   // anything on the device or being built: then waiting frees memory
      for (auto& kv : S.cls) busy = busy || kv.second->occupied() > 0 || !kv.second->ready;
      if (class_usage(S) + cache_bytes() + need > S.opt.mem_budget && busy) {
        ++S.st.deferrals;
        ++it;
        continue;
      }
      c = start_class(S, q);
      if (!c) return fail(ST_MG_ERR_CUDA, "cudaStreamCreate");
      ++it;
      continue;
    }
    if (!c->ready || c->in_flight) {   // a class's vectors change only between its V-cycles
      ++it;
      continue;
    }
    int b = -1;
    for (int j = 0; j < (int)c->slot.size() && b < 0; ++j)
      if (c->slot[j] < 0) b = j;
    if (b < 0) {
      ++it;
      continue;
    }
    int rc = st_mg_assemble_load_batch(c->h, b, (int)q.phase.size(), q.a.data(), q.k.data(), q.phase.data(), c->f);
    if (rc == ST_MG_OK) rc = st_mg_batch_zero(c->h, b, c->x);
    if (rc != ST_MG_OK) return rc;
    c->slot[b] = q.id;
    q.slot = b;
    q.state = 1;
    q.t_admit = now_s();
    q.n_edge = c->ne;
    q.n_values = c->ne * c->seg;
    c->last_use = ++S.tick;
    if (std::find(admitted.begin(), admitted.end(), c) == admitted.end()) admitted.push_back(c);
    it = S.queue.erase(it);
  }
  // ||f_b|| of the newly admitted problems (their classes are idle)
  std::vector<double> norms;
  for (Class* c : admitted) {
    norms.assign(c->slot.size(), 0.0);
    if (int rc = st_mg_batch_norms(c->h, c->f, norms.data())) return rc;
    for (size_t b = 0; b < c->slot.size(); ++b) {
      if (c->slot[b] < 0) continue;
      Request& q = S.req[c->slot[b]];
      if (q.cycles > 0 || q.fnorm > 0) continue;
      q.fnorm = norms[b];
      if (q.fnorm == 0.0) {   // zero load: x = 0 is the solution
        q.rel = 0.0;
        if (S.opt.keep_x) q.x.assign(q.n_values, 0.0);
        c->slot[b] = -1;
        finish_request(S, q, ST_MG_OK, done);
      }
    }
  }

  // (4) every idle class with occupied slots starts its next V-cycle at once: V-cycle,
  // finest residual, per-slot norms, their copy to the host and an event, all queued
  // on the class's stream -- classes advance independently of one another
  for (auto& kv : S.cls) {
    Class& c = *kv.second;
    if (!c.ready || c.in_flight || c.occupied() == 0) continue;
    if (int rc = st_mg_vcycle_residual_async(c.h, c.f, c.x, c.r)) return rc;
    if (int rc = st_mg_batch_norms_async(c.h, c.r, c.norms_dev)) return rc;
    if (cudaMemcpyAsync(c.norms_host, c.norms_dev, c.slot.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        c.stream) != cudaSuccess ||
        cudaEventRecord(c.ev, c.stream) != cudaSuccess)
      return fail(ST_MG_ERR_CUDA, "queueing a class V-cycle");
    c.in_flight = true;
    progressed = true;
  }

  // (5) nothing finished and nothing started: wait (briefly, polling) for the first
  // class to finish, so that a caller looping on step does not spin
  if (!progressed) {
    for (int it = 0; it < 200; ++it) {
      bool any = false, ready = false;
      for (auto& kv : S.cls)
        if (kv.second->in_flight) {
          any = true;
          if (cudaEventQuery(kv.second->ev) != cudaErrorNotReady) ready = true;
        }
      if (!any || ready) break;
      std::this_thread::sleep_for(std::chrono::microseconds(25));
    }
  }
  return ST_MG_OK;
}

void refresh_counts(Server& S) {
  S.st.queued = (int64_t)S.queue.size();
  S.st.active = 0;
  S.st.building = 0;
  for (auto& kv : S.cls) {
    S.st.active += kv.second->occupied();
    S.st.building += kv.second->ready ? 0 : 1;
  }
  S.st.classes = (int32_t)S.cls.size();
}

}  // namespace

extern "C" {

int st_mg_server_default_options(st_mg_server_options* o) {
  if (!o) return fail(ST_MG_ERR_INVALID_ARG, "null options");
  o->slots = 4;
  o->mem_budget = 0;
  o->max_cycles = 50;
  o->slab_prec = 3;
  o->nu = 2;
  o->omega = 0.5;
  o->setup_threads = 0;
  o->keep_x = 1;
  o->max_builds = 2;
  return ST_MG_OK;
}

int st_mg_server_create(const st_mg_server_options* opt, st_mg_server_t* out) {
  if (!opt || !out) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (opt->slots < 1 || opt->mem_budget < 0 || opt->max_cycles < 1 || opt->slab_prec < 0 || opt->slab_prec > 4 ||
      opt->nu < 0 || !(opt->omega > 0) || opt->max_builds < 1)
    return fail(ST_MG_ERR_INVALID_ARG, "invalid server options");
  auto S = std::make_unique<Server>();
  S->opt = *opt;
  if (cudaGetDevice(&S->device) != cudaSuccess) return fail(ST_MG_ERR_CUDA, "cudaGetDevice");
  if (S->opt.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(ST_MG_ERR_CUDA, "cudaMemGetInfo");
    S->opt.mem_budget = (int64_t)(0.8 * (double)fr);
  }
  *out = S.release();
  return ST_MG_OK;
}

int st_mg_server_set_materials(st_mg_server_t srv, int32_t n_cube, int32_t n_space_levels, const double* nu,
                               const double* sigma) {
  if (!srv || !nu || !sigma) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  if (n_cube < 2 || n_space_levels < 1 || (n_cube >> (n_space_levels - 1)) < 2 ||
      n_cube % (1 << (n_space_levels - 1)) != 0)
    return fail(ST_MG_ERR_INVALID_ARG, "invalid mesh");
  if (srv->mats.count(n_cube)) return fail(ST_MG_ERR_INVALID_ARG, "mesh already registered");
  const int64_t nt = (int64_t)6 * n_cube * n_cube * n_cube;
  Materials m;
  m.nsl = n_space_levels;
  m.nu.assign(nu, nu + nt);
  m.sigma.assign(sigma, sigma + nt);
  srv->mats[n_cube] = std::move(m);
  return ST_MG_OK;
}

int st_mg_server_submit(st_mg_server_t srv, const st_mg_request* r, int64_t* id) {
  if (!srv || !r || !id) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  if (!srv->mats.count(r->n_cube)) return fail(ST_MG_ERR_INVALID_ARG, "mesh not registered");
  if ((r->degree != 0 && r->degree != 1) || !pow2(r->N_t) || !(r->tau > 0) || !(r->sigma_scale > 0) ||
      !std::isfinite(r->tau / r->sigma_scale) || !(r->rtol > 0) || r->n_modes < 0 ||
      (r->n_modes > 0 && (!r->a || !r->k || !r->phase)))
    return fail(ST_MG_ERR_INVALID_ARG, "invalid request (degree 0|1, N_t a power of two, tau, s, rtol > 0)");
  Request q;
  q.id = srv->next_id++;
  q.n_cube = r->n_cube;
  q.degree = r->degree;
  q.N_t = r->N_t;
  q.tau = r->tau;
  q.s = r->sigma_scale;
  q.rtol = r->rtol;
  q.a.assign(r->a, r->a + 3 * r->n_modes);
  q.k.assign(r->k, r->k + 3 * r->n_modes);
  q.phase.assign(r->phase, r->phase + r->n_modes);
  q.cls = class_key(q.n_cube, q.degree, q.N_t, q.tau / q.s);
  q.t_arrival = r->t_arrival > 0 ? r->t_arrival : now_s();
  *id = q.id;
  srv->queue.push_back(q.id);
  srv->req[q.id] = std::move(q);
  ++srv->st.submitted;
  return ST_MG_OK;
}

int st_mg_server_step(st_mg_server_t srv, int64_t* done_ids, int32_t cap, int32_t* n_done) {
  if (!srv) return fail(ST_MG_ERR_INVALID_ARG, "null server");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != srv->device)
    return fail(ST_MG_ERR_INVALID_ARG, "st_mg_server_step must run with the server's device current");
  std::vector<int64_t> done;
  refresh_counts(*srv);
  int rc = ST_MG_OK;
  try {
    rc = step(*srv, done);
  } catch (const std::exception& e) {
    rc = fail(ST_MG_ERR_INVALID_ARG, e.what());
  }
  refresh_counts(*srv);
  for (size_t i = 0; i < done.size() && done_ids && (int32_t)i < cap; ++i) done_ids[i] = done[i];
  if (n_done) *n_done = (int32_t)done.size();
  return rc;
}

int st_mg_server_result(st_mg_server_t srv, int64_t id, st_mg_result* res, double* x_host, int64_t x_cap,
                        int32_t release) {
  if (!srv || !res) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  auto it = srv->req.find(id);
  if (it == srv->req.end()) return fail(ST_MG_ERR_INVALID_ARG, "unknown request id");
  const Request& q = it->second;
  res->id = q.id;
  res->state = q.state;
  res->status = q.status;
  res->cycles = q.cycles;
  res->rel_res = q.rel;
  res->t_arrival = q.t_arrival;
  res->t_admit = q.t_admit;
  res->t_done = q.t_done;
  res->n_edge = q.n_edge;
  res->n_values = q.n_values;
  if (q.state == 2) {
    if (x_host && !q.x.empty())
      std::memcpy(x_host, q.x.data(), (size_t)std::min<int64_t>(x_cap, (int64_t)q.x.size()) * sizeof(double));
    if (release) srv->req.erase(it);
  }
  return ST_MG_OK;
}

int st_mg_server_stats_get(st_mg_server_t srv, st_mg_server_stats* out) {
  if (!srv || !out) return fail(ST_MG_ERR_INVALID_ARG, "null argument");
  refresh_counts(*srv);
  int64_t cb = 0;
  for (auto& kv : srv->cls) cb += kv.second->ready ? kv.second->bytes : 0;
  srv->st.class_bytes = cb;
  st_mg_cache_stats(&srv->st.cache_bytes, &srv->st.cache_entries, nullptr, &srv->st.cache_hits,
                    &srv->st.cache_misses);
  *out = srv->st;
  return ST_MG_OK;
}

void st_mg_server_destroy(st_mg_server_t srv) {
  if (!srv) return;
  for (auto& kv : srv->cls) free_class(*kv.second);
  delete srv;
}

}  // extern "C"
