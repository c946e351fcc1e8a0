// Serving: continuous batching of independent Kohn-Sham calculations on one GPU.
//
// Requests are queued by ks_serve_submit and admitted in arrival order while the device
// memory they need fits the server's budget.  Every admitted request owns an engine (its
// states, potentials and tables stay resident on the device) and a CUDA stream; the engines'
// memory comes from the server's slab pool, so admitting and retiring a request neither
// allocates nor frees device memory once the pool has grown (cudaFree would synchronise the
// whole device).  A pool of worker threads runs the admitted requests in quanta -- one
// steepest-descent block iteration or one ETRS step -- and puts each request back in the ready
// queue after its quantum, so requests that arrive while others run are admitted as memory frees
// up and their kernels overlap on the device with the running ones.  Real-time requests on one
// grid geometry are batched: a worker takes up to eight of them that are ready and runs their
// step in lockstep, each H application one packed launch over all their states.  A finished
// request releases its device memory; its results wait on the host until polled.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace ks {

const char* last_error_cstr();

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kMaxGroup = 8;                  // real-time requests per lockstep group

struct Request {
  uint64_t id = 0;
  ks_cell_desc desc{};
  std::vector<double> pos, occ, c0;
  int kind = 0, count = 0;
  double dt = 0;
  size_t bytes = 0;
  // running state
  std::unique_ptr<EngineBase> eng;
  double t_create = 0, t_init = 0, t_orth = 0;   // seconds of the start's parts
  cudaStream_t stream = nullptr;
  int done = 0;
  std::vector<double> result, cout;
  // completion
  bool finished = false;
  ks_status status = KS_OK;
  std::string error;
  Clock::time_point t_submit, t_finish;
};

// Device bytes an engine for this cell will allocate (sphere and column counts exact, the
// rest from the allocation plan of the engine and the fused path).
size_t estimate_bytes(const ks_cell_desc& d) {
  int nG = 0;
  count_sphere(d.L, d.N, d.ecut, &nG);
  const double B = 2.0 * d.ecut * (d.L / (2.0 * M_PI)) * (d.L / (2.0 * M_PI));
  long ncols = 0;
  const int mmax = (int)std::floor(std::sqrt(B));
  for (int mx = -mmax; mx <= mmax; ++mx)
    for (int my = -mmax; my <= mmax; ++my)
      if (mx * mx + my * my <= B) ++ncols;
  const size_t N3 = (size_t)d.N * d.N * d.N;
  const size_t ns = (size_t)d.nstates;
  const bool fp64 = d.prec == KS_FP64;
  const size_t cb = fp64 ? 16 : 8;
  size_t b = 7 * ns * nG * cb + ns * nG * 16;         // six state buffers + complex128 staging
  b += N3 * (fp64 ? 8 : 4) * 4 + N3 * cb + N3 * 8;   // V_loc, V, density, Poisson work, FP64 V_loc
  const size_t nn = ns * ns;
  b += nn * 16 * 8 + nn * 16 * 152 / 4;               // dense matrices and split-K partials (152 SMs)
  if (fp64) {
    b += std::min<size_t>(ns, std::max<size_t>(1, (size_t(1) << 30) / (N3 * 16))) * N3 * 16;
  } else {
    b += 2 * ns * d.N * ncols * 8 + N3 * 4 * 2;       // column buffers, planes, density partials
    const size_t np = (size_t)d.natoms * d.nproj;
    b += 2 * np * nG * 8 + np * ns * 32 + np * ns * 16 * 40;   // projector block and its split image
    // projector values of the covered points per state (sphere points of every atom, 1/8 spare)
    const double rp = d.proj_rc * d.N / d.L;
    b += (size_t)(ns * (size_t)d.natoms * (4.19 * rp * rp * rp * 1.15 + 64.0)) * 8;
  }
  b += (size_t)d.natoms * 1400 * (d.nproj + 4) * 8;   // projector tables
  return b + (size_t(64) << 20);
}

}  // namespace

}  // namespace ks

struct ks_server_s {
  size_t budget = 0, in_use = 0;
  std::unique_ptr<ks::DevicePool> pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ks::Request*> pending;   // waiting for admission
  std::deque<ks::Request*> ready;     // admitted, waiting for a worker
  std::map<uint64_t, std::unique_ptr<ks::Request>> all;
  std::vector<std::thread> workers;
  uint64_t next_id = 1;
  int running = 0;
  bool stop = false;
  int device = 0;
  // worker seconds by activity, and the real-time group steps (ks_serve_stats)
  double t_start = 0, t_gs = 0, t_td = 0, t_finish = 0;
  double t_create = 0, t_init = 0, t_orth = 0;   // parts of t_start
  long n_start = 0, n_gs = 0, n_td_steps = 0, n_td_members = 0;
};

namespace ks {

namespace {

void finish(ks_server_s* s, Request* r, ks_status st, const std::string& err) {
  // called without the lock; releases device resources then publishes the result
  if (r->eng && st == KS_OK && r->cout.empty()) {
    try {
      const auto& geo = r->eng->geo();
      r->cout.resize((size_t)r->desc.nstates * geo.nG * 2);
      r->eng->get_states(r->cout.data(), r->stream);
    } catch (const Error& e) {
      st = e.st;
    }
  }
  if (r->stream) cudaStreamSynchronize(r->stream);   // the engine's blocks go back to the pool idle
  r->eng.reset();
  if (r->stream) {
    cudaStreamDestroy(r->stream);
    r->stream = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->finished = true;
  r->status = st;
  r->error = err;
  r->t_finish = Clock::now();
  s->in_use -= r->bytes;
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

// Create the engine and initial states of an admitted request (worker thread, no lock).
void start(ks_server_s* s, Request* r) {
  const auto t0 = Clock::now();
  KS_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
  r->eng = make_engine(r->desc, s->pool.get());
  const auto t1 = Clock::now();
  if (!r->c0.empty()) {
    r->eng->set_states(r->c0.data(), r->stream);
    r->c0.clear();
    r->c0.shrink_to_fit();
  } else {
    r->eng->randomize_states(0x9E3779B97F4A7C15ull ^ r->id, r->stream);
  }
  const auto t2 = Clock::now();
  if (r->kind == 1) r->eng->orthonormalize(nullptr, r->stream);
  if (r->kind == 0) r->result.assign(r->desc.nstates, 0.0);
  const auto t3 = Clock::now();
  r->t_create = std::chrono::duration<double>(t1 - t0).count();
  r->t_init = std::chrono::duration<double>(t2 - t1).count();
  r->t_orth = std::chrono::duration<double>(t3 - t2).count();
}

// One ETRS step of a group of started real-time requests in lockstep (td_step_engines) on the
// first one's stream, after the work already queued on the others' streams.
void td_group_quantum(const std::vector<Request*>& g) {
  std::vector<EngineBase*> es;
  for (Request* r : g) es.push_back(r->eng.get());
  cudaStream_t s0 = g[0]->stream;
  for (size_t i = 1; i < g.size(); ++i) {
    cudaEvent_t ev;
    KS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    KS_CUDA(cudaEventRecord(ev, g[i]->stream));
    KS_CUDA(cudaStreamWaitEvent(s0, ev, 0));
    KS_CUDA(cudaEventDestroy(ev));
  }
  std::vector<double> nrm(g.size()), e(g.size());
  td_step_engines(es, g[0]->dt, 1, nrm.data(), e.data(), s0);      // synchronous on s0
  for (size_t i = 0; i < g.size(); ++i) g[i]->result.push_back(e[i]);
}

// One quantum; returns true when the request has done all its work.
bool quantum(Request* r) {
  if (r->kind == 0) {
    r->eng->block_iteration(1, r->result.data(), r->stream);
  } else if (r->eng->precision() == KS_MIXED_BF16X3) {
    td_group_quantum(std::vector<Request*>{r});      // the same kernels as in a group
  } else {
    double nrm = 0, e = 0;
    r->eng->td_steps(r->dt, 1, 0, 1, &nrm, &e, nullptr, r->stream);
    r->result.push_back(e);
  }
  return ++r->done >= r->count;
}

void worker_loop(ks_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // admission: arrival order, while the budget allows
    while (!s->pending.empty() && s->in_use + s->pending.front()->bytes <= s->budget) {
      Request* r = s->pending.front();
      s->pending.pop_front();
      s->in_use += r->bytes;
      r->eng = nullptr;
      r->done = -1;                    // not started yet
      s->ready.push_back(r);
    }
    if (s->stop && s->ready.empty()) return;
    if (s->ready.empty()) {
      s->cv_work.wait(lk);
      continue;
    }
    Request* r = s->ready.front();
    s->ready.pop_front();
    // a started real-time request takes along the ready ones it can share launches with
    std::vector<Request*> group{r};
    if (r->kind == 1 && r->done >= 0 && r->eng) {
      for (auto it = s->ready.begin(); it != s->ready.end() && group.size() < kMaxGroup;) {
        Request* q = *it;
        if (q->kind == 1 && q->done >= 0 && q->eng && q->dt == r->dt && td_groupable(r->eng.get(), q->eng.get())) {
          group.push_back(q);
          it = s->ready.erase(it);
        } else {
          ++it;
        }
      }
    }
    s->running += (int)group.size();
    lk.unlock();
    ks_status st = KS_OK;
    std::string err;
    std::vector<bool> complete(group.size(), false);
    const auto t0 = Clock::now();
    int activity = 0;                                               // 0 start, 1 ground state, 2 real time
    try {
      if (group.size() > 1) {
        activity = 2;
        td_group_quantum(group);
        for (size_t i = 0; i < group.size(); ++i) complete[i] = ++group[i]->done >= group[i]->count;
      } else if (r->done < 0) {
        r->done = 0;
        start(s, r);
        complete[0] = r->count <= 0;
      } else {
        activity = r->kind == 0 ? 1 : 2;
        complete[0] = quantum(r);
      }
    } catch (const Error& e) {
      st = e.st;
      err = std::string("request failed: ") + last_error_cstr();
      complete.assign(group.size(), true);
    } catch (...) {
      st = KS_ERR_CUDA;
      err = "request failed";
      complete.assign(group.size(), true);
    }
    const auto t1 = Clock::now();
    for (size_t i = 0; i < group.size(); ++i)
      if (complete[i]) finish(s, group[i], st, err);
    const auto t2 = Clock::now();
    lk.lock();
    const double dq = std::chrono::duration<double>(t1 - t0).count();
    if (activity == 0) {
      s->t_start += dq;
      ++s->n_start;
      s->t_create += r->t_create;
      s->t_init += r->t_init;
      s->t_orth += r->t_orth;
    } else if (activity == 1) {
      s->t_gs += dq;
      ++s->n_gs;
    } else {
      s->t_td += dq;
      ++s->n_td_steps;
      s->n_td_members += (long)group.size();
    }
    s->t_finish += std::chrono::duration<double>(t2 - t1).count();
    s->running -= (int)group.size();
    for (size_t i = 0; i < group.size(); ++i)
      if (!complete[i]) s->ready.push_back(group[i]);
    s->cv_work.notify_all();
  }
}

}  // namespace

}  // namespace ks

extern "C" {

ks_status ks_serve_create(size_t mem_budget_bytes, ks_server* out) {
  return ks_serve_create_ex(mem_budget_bytes, 0, out);
}

ks_status ks_serve_create_ex(size_t mem_budget_bytes, int workers, ks_server* out) {
  if (out) *out = nullptr;
  try {
    if (!out) ks::fail(KS_ERR_ARG, "out is NULL");
    if (workers < 0 || workers > 64) ks::fail(KS_ERR_ARG, "workers=%d outside [0, 64]", workers);
    std::unique_ptr<ks_server_s> s(new ks_server_s);
    if (cudaGetDevice(&s->device) != cudaSuccess) {   // no device: requests fail when started
      cudaGetLastError();
      s->device = 0;
    }
    if (mem_budget_bytes == 0) {
      size_t fr = 0, tot = 0;
      KS_CUDA(cudaMemGetInfo(&fr, &tot));
      mem_budget_bytes = (size_t)(0.8 * (double)fr);
    }
    s->budget = mem_budget_bytes;
    s->pool.reset(new ks::DevicePool(size_t(4) << 30));             // 4 GB slabs
    const int nworkers = workers > 0 ? workers : 16;
    for (int i = 0; i < nworkers; ++i) s->workers.emplace_back(ks::worker_loop, s.get());
    *out = s.release();
    return KS_OK;
  } catch (const ks::Error& e) {
    return e.st;
  } catch (...) {
    ks::set_last_error("ks_serve_create: unexpected error");
    return KS_ERR_CUDA;
  }
}

ks_status ks_serve_destroy(ks_server s) {
  if (!s) return KS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // drop requests that were never admitted
    for (ks::Request* r : s->pending) {
      r->finished = true;
      r->status = KS_ERR_STATE;
    }
    s->pending.clear();
    s->cv_work.notify_all();
  }
  for (auto& t : s->workers) t.join();
  delete s;
  return KS_OK;
}

ks_status ks_serve_submit(ks_server s, const ks_cell_desc* desc, const double* c0, int kind, int count, double dt,
                          uint64_t* ticket) {
  try {
    if (!s || !desc || !ticket) ks::fail(KS_ERR_ARG, "server/desc/ticket is NULL");
    if (kind != 0 && kind != 1) ks::fail(KS_ERR_ARG, "kind must be 0 (block iterations) or 1 (ETRS steps)");
    if (count < 0 || count > 100000) ks::fail(KS_ERR_ARG, "count=%d out of range", count);
    if (kind == 1 && !(dt > 0 && dt < 10)) ks::fail(KS_ERR_ARG, "dt must be in (0, 10)");
    if (desc->nstates < 1 || desc->natoms < 0 || (desc->natoms > 0 && !desc->pos))
      ks::fail(KS_ERR_ARG, "bad cell description");
    std::unique_ptr<ks::Request> r(new ks::Request);
    r->desc = *desc;
    r->pos.assign(desc->pos, desc->pos + 3 * (size_t)desc->natoms);
    r->desc.pos = r->pos.data();
    if (desc->occ) {
      r->occ.assign(desc->occ, desc->occ + desc->nstates);
      r->desc.occ = r->occ.data();
    }
    r->bytes = ks::estimate_bytes(r->desc);   // validates the grid (KS_ERR_ARG)
    if (r->bytes > s->budget)
      ks::fail(KS_ERR_NOMEM, "request needs ~%zu bytes, above the server budget of %zu", r->bytes, s->budget);
    int nG = 0;
    ks::count_sphere(desc->L, desc->N, desc->ecut, &nG);
    if (c0) r->c0.assign(c0, c0 + (size_t)desc->nstates * nG * 2);
    r->kind = kind;
    r->count = count;
    r->dt = dt;
    r->t_submit = ks::Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    *ticket = r->id;
    s->pending.push_back(r.get());
    s->all[r->id] = std::move(r);
    s->cv_work.notify_all();
    return KS_OK;
  } catch (const ks::Error& e) {
    return e.st;
  } catch (...) {
    ks::set_last_error("ks_serve_submit: unexpected error");
    return KS_ERR_CUDA;
  }
}

ks_status ks_serve_stats(ks_server s, double* out, int nout) {
  if (!s || (!out && nout > 0) || nout < 0) {
    ks::set_last_error("server/out is NULL or nout < 0");
    return KS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const double v[14] = {s->t_start, s->t_gs, s->t_td, s->t_finish, (double)s->n_start, (double)s->n_gs,
                        (double)s->n_td_steps, (double)s->n_td_members,
                        s->pool ? (double)s->pool->reserved() : 0.0, s->t_create, s->t_init, s->t_orth,
                        s->pool ? (double)s->pool->grows() : 0.0, s->pool ? s->pool->grow_seconds() : 0.0};
  for (int i = 0; i < nout && i < 14; ++i) out[i] = v[i];
  return KS_OK;
}

ks_status ks_serve_result_info(ks_server s, uint64_t ticket, int* nresult, int* nstates, int* nG) {
  if (!s) {
    ks::set_last_error("server is NULL");
    return KS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    ks::set_last_error("unknown ticket");
    return KS_ERR_ARG;
  }
  ks::Request* r = it->second.get();
  int g = 0;
  try {
    ks::count_sphere(r->desc.L, r->desc.N, r->desc.ecut, &g);
  } catch (const ks::Error& e) {
    return e.st;
  }
  if (nresult) *nresult = r->kind == 0 ? r->desc.nstates : r->count;
  if (nstates) *nstates = r->desc.nstates;
  if (nG) *nG = g;
  return KS_OK;
}

ks_status ks_serve_poll(ks_server s, uint64_t ticket, int timeout_ms, double* result_out, double* c_out_opt,
                        double* latency_s_opt) {
  if (!s) {
    ks::set_last_error("server is NULL");
    return KS_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    ks::set_last_error("unknown ticket");
    return KS_ERR_ARG;
  }
  ks::Request* r = it->second.get();
  if (!r->finished) {
    if (timeout_ms <= 0) return KS_PENDING;
    const auto until = ks::Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!r->finished)
      if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !r->finished) {
        ks::set_last_error("poll timed out");
        return KS_ERR_TIMEOUT;
      }
  }
  const ks_status st = r->status;
  if (st != KS_OK) {
    ks::set_last_error(r->error.empty() ? "request failed" : r->error);
  } else {
    if (result_out) std::memcpy(result_out, r->result.data(), r->result.size() * sizeof(double));
    if (c_out_opt && !r->cout.empty()) std::memcpy(c_out_opt, r->cout.data(), r->cout.size() * sizeof(double));
    if (latency_s_opt) *latency_s_opt = std::chrono::duration<double>(r->t_finish - r->t_submit).count();
  }
  s->all.erase(it);
  return st;
}

}  // extern "C"
