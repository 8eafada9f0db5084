// Serving loop: continuous batching of independent ADER-CWENO solves on one
// GPU.
//
// submit -> FIFO queue -> admission (a free slot and the request's device
// footprint within the budget) -> host setup worker (mesh, stencils, FP64
// least-squares inverses on the device, initial state and CFL bound, on the
// slot's stream) -> the request joins the group of its configuration
// (dimension, order, PDE, precision, flux).
//
// Groups are per configuration and size class (a tick lasts as long as its
// members' steps together).  Each group advances all of its members by one
// time step per tick: one
// captured CUDA graph (the group's batch table copied from pinned host
// memory, then the batched reconstruction + predictor, flux and update
// kernels over all members' cells and faces), replayed every tick on the
// group's stream.  Between ticks the scheduler rewrites the table in place
// (members that joined or left, each member's time-step slot), so changes of
// membership need no new capture.  A member's last tick also copies its
// final state to pinned host memory; the scheduler retires it when that
// tick's event completes and admits waiting requests as slots and memory
// free up.  Groups tick concurrently on their own streams, and host setup of
// waiting requests overlaps with the ticks.  Every cell and face of a member
// gets the arithmetic of the single-solver kernels and no reduction spans
// members, so every result equals the same solve run alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/cweno.h"
#include "api_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Group;

struct Req {
  uint64_t id = 0;
  int dim = 2, order = 2, pde = 0, prec = 0, nsteps = 0, nvars = 4;
  double cfl = 0.5;
  int64_t nverts = 0, nc = 0;
  std::vector<double> xyz, period, Q0;
  std::vector<int32_t> cells;
  bool has_period = false;
  size_t est = 0;
  int status = CWENO_REQ_QUEUED;
  Clock::time_point t_submit, t_done;
  cweno_mesh* mesh = nullptr;
  cweno_solver* solver = nullptr;
  int slot = -1;
  int steps_done = 0;
  double* hout = nullptr;  // pinned: nc * nvars
  int* hstatus = nullptr;  // pinned
  std::vector<double> Qout;
  std::string err;
};

// One configuration's batch: its members, the pinned and device images of
// the batch table, the captured tick graph and the tick in flight.
struct Group {
  std::tuple<int, int, int, int, int, int> key;  // dim, order, pde, precision, flux, size class
  int flux = 0;
  std::unique_ptr<cw::Ops> ops;
  cudaStream_t stream = nullptr;
  void* htab = nullptr;
  void* dtab = nullptr;
  size_t tab_bytes = 0;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
  std::vector<Req*> members;    // stepping
  std::vector<Req*> ticking;    // members of the tick in flight
  std::vector<Req*> finishing;  // members whose final state that tick copies
  uint64_t ticks = 0;
};

}  // namespace

struct cweno_server {
  int dev = 0;
  size_t budget = 0, used = 0;
  int max_slots = 1, nworkers = 1, threads_per_setup = 1;
  std::vector<cudaStream_t> streams;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;    // submitted, waiting for admission
  std::deque<Req*> setup_q;  // admitted, waiting for a setup worker
  std::vector<Req*> ready;   // set up, waiting to join their group
  std::deque<std::pair<Req*, int>> retire_q;  // finished ticks: (request, its status word or -1 on failure)
  std::map<uint64_t, Req*> all;
  std::vector<std::unique_ptr<Group>> groups;  // scheduler thread only
  int active = 0;                              // admitted and not retired
  uint64_t next_id = 1, n_sub = 0, n_adm = 0, n_done = 0, peak = 0, ticks = 0, member_steps = 0;
  double cell_updates = 0.0;
  bool stop = false;
  std::thread sched, retirer;
  std::vector<std::thread> workers;
  // pinned host buffers are pooled: freeing pinned memory can synchronise the
  // whole device, which would stall the other requests
  std::mutex pin_mu;
  std::multimap<size_t, void*> pinned_free;
  std::vector<void*> pinned_all;
  std::map<void*, size_t> pinned_cap;
};

namespace {

void* pin_get(cweno_server* S, size_t bytes) {
  std::lock_guard<std::mutex> lk(S->pin_mu);
  auto it = S->pinned_free.lower_bound(bytes);
  if (it != S->pinned_free.end()) {
    void* p = it->second;
    S->pinned_free.erase(it);
    return p;
  }
  void* p = nullptr;
  size_t cap = std::max<size_t>(bytes, 4096);
  if (cudaMallocHost(&p, cap) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  S->pinned_all.push_back(p);
  S->pinned_cap[p] = cap;
  return p;
}

void pin_put(cweno_server* S, void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(S->pin_mu);
  S->pinned_free.insert({S->pinned_cap[p], p});
}

void release_slot(cweno_server* S, Req* r) {  // caller holds S->mu
  if (r->slot >= 0) S->free_slots.push_back(r->slot);
  r->slot = -1;
  S->used -= std::min(S->used, r->est);
  S->active -= 1;
}

void teardown(cweno_server* S, Req* r) {
  if (r->solver) cweno_solver_destroy(r->solver);
  r->solver = nullptr;
  if (r->mesh) cweno_mesh_destroy(r->mesh);
  r->mesh = nullptr;
  pin_put(S, r->hout);
  r->hout = nullptr;
  pin_put(S, r->hstatus);
  r->hstatus = nullptr;
  std::vector<double>().swap(r->xyz);
  std::vector<int32_t>().swap(r->cells);
  std::vector<double>().swap(r->Q0);
}

// Host setup of one admitted request (worker thread): mesh, solver, initial
// state and CFL bound on the slot's stream, complete when this returns.
int prepare(cweno_server* S, Req* r, std::string& err) {
  cudaStream_t st = S->streams[r->slot];
  int rc = cweno_mesh_create(r->dim, r->nverts, r->xyz.data(), r->nc, r->cells.data(),
                             r->has_period ? r->period.data() : nullptr, &r->mesh);
  if (rc) return err = cweno_last_error(), rc;
  cweno_params p;
  cweno_default_params(&p, r->dim, r->pde);
  p.cfl = r->cfl;
  rc = cweno_setup(r->mesh, r->order, r->pde, r->prec, &p, st, &r->solver);
  if (rc) return err = cweno_last_error(), rc;
  size_t real = 0;
  cweno_solver_footprint(r->solver, &real);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->used = S->used - std::min(S->used, r->est) + real;
    r->est = real;
  }
  r->hout = (double*)pin_get(S, sizeof(double) * r->nc * r->nvars);
  r->hstatus = (int*)pin_get(S, sizeof(int));
  if (!r->hout || !r->hstatus) {
    err = "pinned host allocation failed";
    return CWENO_ENOMEM;
  }
  rc = cweno_set_state(r->solver, r->Q0.data(), 0);  // also the CFL bound of the first step
  if (rc) return err = cweno_last_error(), rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err = std::string("setup: ") + cudaGetErrorString(e), CWENO_ECUDA;
  return CWENO_OK;
}

void worker_main(cweno_server* S) {
  cudaSetDevice(S->dev);
  cw::g_setup_threads = S->threads_per_setup;
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->setup_q.empty(); });
      if (S->stop) return;
      r = S->setup_q.front();
      S->setup_q.pop_front();
    }
    std::string err;
    int rc = prepare(S, r, err);
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc) {
      r->status = CWENO_REQ_ERROR;
      r->err = err;
      r->t_done = Clock::now();
      if (r->slot >= 0) cudaStreamSynchronize(S->streams[r->slot]);
      teardown(S, r);
      release_slot(S, r);
      S->n_done++;
    } else {
      r->status = CWENO_REQ_RUNNING;
      S->ready.push_back(r);
    }
    S->cv.notify_all();
  }
}

// Size class of a request: cells below 4096, 16384, 65536 or above.  A tick
// lasts as long as its group's members take together, so requests of very
// different sizes tick in different groups (concurrently): a small request
// does not wait for the steps of large ones.
int size_class(int64_t nc) {
  int c = 0;
  for (int64_t lim = 4096; c < 3 && nc >= lim; lim *= 4) ++c;
  return c;
}

// The group of r's configuration and size class, created (with its tick
// graph) on first use.
Group* group_of(cweno_server* S, Req* r, std::string& err) {
  const int flux = r->solver->prm.flux;
  auto key = std::make_tuple(r->dim, r->order, r->pde, r->prec, flux, size_class(r->nc));
  for (auto& g : S->groups)
    if (g->key == key) return g.get();
  std::unique_ptr<Group> g(new Group());
  g->key = key;
  g->flux = flux;
  const int M = r->order - 1, fp32 = r->prec == CWENO_FP32_MIXED;
  const cw::RefElem& re = cw::ref_elem(r->dim, M);
  if (r->pde == CWENO_EULER && r->dim == 2) g->ops = cw::make_ops_euler2(M, fp32, re);
  else if (r->pde == CWENO_EULER && r->dim == 3) g->ops = cw::make_ops_euler3(M, fp32, re);
  else g->ops = cw::make_ops_mhd2(M, fp32, re);
  if (!g->ops) return err = "configuration not built", nullptr;
  cudaError_t e = g->ops->prepare();
  g->tab_bytes = g->ops->batch_bytes();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&g->htab, g->tab_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&g->dtab, g->tab_bytes);
  if (e == cudaSuccess) {
    std::memset(g->htab, 0, g->tab_bytes);
    cudaGraph_t graph;
    e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemcpyAsync(g->dtab, g->htab, g->tab_bytes, cudaMemcpyHostToDevice, g->stream);
      cudaError_t e2 = e1 == cudaSuccess ? g->ops->step_batch(g->dtab, flux, g->stream) : e1;
      e = cudaStreamEndCapture(g->stream, &graph);
      if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&g->graph, graph, 0);
        cudaGraphDestroy(graph);
      }
    }
  }
  if (e != cudaSuccess) {
    err = std::string("batch setup: ") + cudaGetErrorString(e);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->dtab) cudaFree(g->dtab);
    if (g->htab) cudaFreeHost(g->htab);
    if (g->done) cudaEventDestroy(g->done);
    if (g->stream) cudaStreamDestroy(g->stream);
    return nullptr;
  }
  S->groups.push_back(std::move(g));
  return S->groups.back().get();
}

// One tick of g: table of the members, graph launch, final-state copies of
// the members that reach their last step, completion event.
cudaError_t launch_tick(Group* g) {
  const int n = (int)g->members.size();
  std::vector<const cw::DevState*> ds(n);
  std::vector<const cw::PhysParams*> ph(n);
  std::vector<cw::DtArgs> dt(n);
  for (int k = 0; k < n; ++k) {
    cweno_solver* s = g->members[k]->solver;
    ds[k] = &s->ds;
    ph[k] = &s->ph;
    dt[k].fixed = 0.0;  // the CFL bound computed on the device
    dt[k].cfl = s->prm.cfl;
    dt[k].cur = s->cur;
  }
  g->ops->batch_fill(g->htab, n, ds.data(), ph.data(), dt.data());
  cudaError_t e = cudaGraphLaunch(g->graph, g->stream);
  if (e != cudaSuccess) return e;
  g->ticking = g->members;
  g->finishing.clear();
  for (Req* r : g->members) {
    if (r->steps_done + 1 < r->nsteps) continue;
    cweno_solver* s = r->solver;
    if ((e = s->ops->get_state(s->ds, s->ds.stage, g->stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(r->hout, s->ds.stage, sizeof(double) * r->nc * r->nvars, cudaMemcpyDeviceToHost,
                             g->stream)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(r->hstatus, s->ds.status, sizeof(int), cudaMemcpyDeviceToHost, g->stream)) !=
        cudaSuccess)
      return e;
    g->finishing.push_back(r);
  }
  if ((e = cudaEventRecord(g->done, g->stream)) != cudaSuccess) return e;
  g->in_flight = true;
  g->ticks++;
  return cudaSuccess;
}

void retire(cweno_server* S, Req* r, int status, const std::string& err) {
  teardown(S, r);
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = status;
  if (status == CWENO_REQ_ERROR) r->err = err;
  release_slot(S, r);
  S->n_done++;
  if (status == CWENO_REQ_DONE) S->cell_updates += (double)r->nc * r->nsteps;
  S->cv.notify_all();
}

// Retirement off the scheduler's path (copying a final state out of pinned
// memory and freeing a solver take milliseconds, during which no group
// would get its next tick): results, teardown, slot release.
void retirer_main(cweno_server* S) {
  cudaSetDevice(S->dev);
  for (;;) {
    std::pair<Req*, int> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->retire_q.empty(); });
      if (S->retire_q.empty()) return;  // stop with nothing left
      job = S->retire_q.front();
      S->retire_q.pop_front();
    }
    Req* r = job.first;
    if (job.second < 0) {
      retire(S, r, CWENO_REQ_ERROR, r->err);
      continue;
    }
    r->Qout.assign(r->hout, r->hout + r->nc * r->nvars);
    retire(S, r, job.second ? CWENO_REQ_ERROR : CWENO_REQ_DONE,
           "the solve produced NaN or non-positive density / pressure");
  }
}

void scheduler_main(cweno_server* S) {
  cudaSetDevice(S->dev);
  for (;;) {
    std::vector<Req*> joining;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) return;
      // admission: FIFO, while a slot is free and the footprint fits
      while (!S->queue.empty() && !S->free_slots.empty() && S->used + S->queue.front()->est <= S->budget) {
        Req* r = S->queue.front();
        S->queue.pop_front();
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        S->used += r->est;
        S->active += 1;
        S->n_adm++;
        S->peak = std::max<uint64_t>(S->peak, (uint64_t)S->active);
        S->setup_q.push_back(r);
        S->cv.notify_all();
      }
      joining.swap(S->ready);
    }
    bool progress = false;
    std::vector<Req*> waiting;  // their group's table is full: join at a later tick
    for (Req* r : joining) {
      if (r->nsteps == 0) {  // nothing to step: the initial state is the result
        r->t_done = Clock::now();
        r->Qout = r->Q0;
        retire(S, r, CWENO_REQ_DONE, "");
        continue;
      }
      std::string err;
      Group* g = group_of(S, r, err);
      if (!g) {
        r->t_done = Clock::now();
        retire(S, r, CWENO_REQ_ERROR, err);
        continue;
      }
      if ((int)g->members.size() >= g->ops->batch_max()) {
        waiting.push_back(r);
        continue;
      }
      g->members.push_back(r);
      progress = true;
    }
    if (!waiting.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->ready.insert(S->ready.begin(), waiting.begin(), waiting.end());
    }
    for (auto& gp : S->groups) {
      Group* g = gp.get();
      if (g->in_flight) {
        const cudaError_t q = cudaEventQuery(g->done);
        if (q == cudaErrorNotReady) continue;
        g->in_flight = false;
        progress = true;
        if (q != cudaSuccess) {  // a failed tick fails every member of the group
          for (Req* r : g->members) {
            r->t_done = Clock::now();
            retire(S, r, CWENO_REQ_ERROR, std::string("tick: ") + cudaGetErrorString(q));
          }
          g->members.clear();
          g->ticking.clear();
          g->finishing.clear();
          continue;
        }
        for (Req* r : g->ticking) {
          r->steps_done++;
          r->solver->cur ^= 1;
        }
        for (Req* r : g->finishing) {
          g->members.erase(std::find(g->members.begin(), g->members.end(), r));
          r->t_done = Clock::now();
          std::lock_guard<std::mutex> lk(S->mu);
          S->retire_q.push_back({r, *r->hstatus});
          S->cv.notify_all();
        }
        {
          std::lock_guard<std::mutex> lk(S->mu);
          S->ticks++;
          S->member_steps += g->ticking.size();
        }
        g->ticking.clear();
        g->finishing.clear();
      }
      if (!g->in_flight && !g->members.empty()) {
        const cudaError_t e = launch_tick(g);
        progress = true;
        if (e != cudaSuccess) {  // the whole group fails
          for (Req* r : g->members) {
            r->t_done = Clock::now();
            retire(S, r, CWENO_REQ_ERROR, std::string("tick launch: ") + cudaGetErrorString(e));
          }
          g->members.clear();
          g->in_flight = false;
        }
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

}  // namespace

extern "C" {

int serve_create(size_t mem_budget, int max_slots, int nworkers, cweno_server** out) {
  if (!out) return cw::fail(CWENO_EINVAL, "null output handle");
  *out = nullptr;
  std::unique_ptr<cweno_server> S(new cweno_server());
  if (cudaGetDevice(&S->dev) != cudaSuccess) return cw::fail(CWENO_ECUDA, "no CUDA device");
  if (mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cw::fail(CWENO_ECUDA, "cudaMemGetInfo failed");
    mem_budget = (size_t)(0.8 * (double)fr);
  }
  S->budget = mem_budget;
  // admitted requests (each with a stream for its setup); a group's batch
  // table holds at most 64 members (Ops::batch_max), requests beyond that
  // wait to join their group
  S->max_slots = std::min(max_slots > 0 ? max_slots : 256, 256);
  unsigned hc = std::max(1u, std::thread::hardware_concurrency());
  // one setup worker per host core by default: a worker builds one request's
  // mesh (host, single-threaded) and runs its stencil search and
  // least-squares setup on the device, so workers scale with the cores
  S->nworkers = nworkers > 0 ? nworkers : (int)std::max(2u, hc);
  S->threads_per_setup = (int)std::max(1u, hc / (unsigned)S->nworkers);
  S->streams.resize(S->max_slots);
  for (int k = 0; k < S->max_slots; ++k) {
    if (cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking) != cudaSuccess)
      return cw::fail(CWENO_ECUDA, "stream creation failed");
    S->free_slots.push_back(S->max_slots - 1 - k);
  }
  cweno_server* raw = S.get();
  for (int k = 0; k < S->nworkers; ++k) S->workers.emplace_back(worker_main, raw);
  S->sched = std::thread(scheduler_main, raw);
  S->retirer = std::thread(retirer_main, raw);
  *out = S.release();
  return CWENO_OK;
}

int serve_submit(cweno_server* S, const cweno_request* q, uint64_t* id) {
  if (!S || !q || !id) return cw::fail(CWENO_EINVAL, "null argument");
  if ((q->dim != 2 && q->dim != 3) || q->nv <= 0 || q->nc <= 0 || !q->xyz || !q->cells || !q->Q0 ||
      q->order < 2 || q->order > 5 || q->nsteps < 0 || !(q->cfl > 0) ||
      (q->pde != CWENO_EULER && q->pde != CWENO_MHD_GLM) ||
      (q->precision != CWENO_FP64 && q->precision != CWENO_FP32_MIXED))
    return cw::fail(CWENO_EINVAL, "bad request");
  std::unique_ptr<Req> r(new Req());
  r->dim = q->dim;
  r->order = q->order;
  r->pde = q->pde;
  r->prec = q->precision;
  r->nsteps = q->nsteps;
  r->cfl = q->cfl;
  r->nverts = q->nv;
  r->nc = q->nc;
  r->nvars = cweno_nvars(q->dim, q->pde);
  r->xyz.assign(q->xyz, q->xyz + q->nv * q->dim);
  r->cells.assign(q->cells, q->cells + q->nc * (q->dim + 1));
  r->Q0.assign(q->Q0, q->Q0 + q->nc * r->nvars);
  if (q->period) {
    r->has_period = true;
    r->period.assign(q->period, q->period + q->dim);
  }
  // faces <= (d+1) nc (every face counted from each side)
  r->est = cw::footprint_estimate(q->dim, q->nc, (q->dim + 1) * q->nc, q->order, q->pde, q->precision);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (r->est > S->budget)
    return cw::fail(CWENO_EBUSY, "request footprint " + std::to_string(r->est) + " B exceeds the server budget " +
                                     std::to_string(S->budget) + " B");
  r->id = S->next_id++;
  *id = r->id;
  S->all[r->id] = r.get();
  S->queue.push_back(r.release());
  S->n_sub++;
  S->cv.notify_all();
  return CWENO_OK;
}

int serve_poll(cweno_server* S, uint64_t id, int* status, double* Q_out, double* latency_s) {
  if (!S || !status) return cw::fail(CWENO_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return cw::fail(CWENO_ENOTFOUND, "unknown request id");
  Req* r = it->second;
  *status = r->status;
  if (latency_s)
    *latency_s = (r->status == CWENO_REQ_DONE || r->status == CWENO_REQ_ERROR)
                     ? std::chrono::duration<double>(r->t_done - r->t_submit).count()
                     : 0.0;
  if (r->status == CWENO_REQ_ERROR) {
    cw::fail(CWENO_ENAN, r->err);
  }
  if ((r->status == CWENO_REQ_DONE || r->status == CWENO_REQ_ERROR) && Q_out) {
    if (r->status == CWENO_REQ_DONE) std::memcpy(Q_out, r->Qout.data(), sizeof(double) * r->Qout.size());
    S->all.erase(it);
    delete r;
  }
  return CWENO_OK;
}

int serve_drain(cweno_server* S, double timeout_s) {
  if (!S) return cw::fail(CWENO_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  bool ok = S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return S->n_done == S->n_sub; });
  if (!ok) return cw::fail(CWENO_ETIMEDOUT, "requests still running after the timeout");
  return CWENO_OK;
}

int serve_stats(cweno_server* S, uint64_t* submitted, uint64_t* admitted, uint64_t* completed, uint64_t* peak_running,
                double* cell_updates) {
  if (!S) return cw::fail(CWENO_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (submitted) *submitted = S->n_sub;
  if (admitted) *admitted = S->n_adm;
  if (completed) *completed = S->n_done;
  if (peak_running) *peak_running = S->peak;
  if (cell_updates) *cell_updates = S->cell_updates;
  return CWENO_OK;
}

int serve_batch_stats(cweno_server* S, uint64_t* ticks, uint64_t* member_steps) {
  if (!S) return cw::fail(CWENO_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticks) *ticks = S->ticks;
  if (member_steps) *member_steps = S->member_steps;
  return CWENO_OK;
}

void serve_destroy(cweno_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  for (auto& t : S->workers) t.join();
  if (S->sched.joinable()) S->sched.join();
  if (S->retirer.joinable()) S->retirer.join();
  cudaSetDevice(S->dev);
  for (auto& g : S->groups) {
    cudaStreamSynchronize(g->stream);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->dtab) cudaFree(g->dtab);
    if (g->htab) cudaFreeHost(g->htab);
    if (g->done) cudaEventDestroy(g->done);
    if (g->stream) cudaStreamDestroy(g->stream);
  }
  S->groups.clear();
  for (auto& kv : S->all) {
    Req* r = kv.second;
    if (r->slot >= 0) cudaStreamSynchronize(S->streams[r->slot]);
    teardown(S, r);
    delete r;
  }
  for (cudaStream_t st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (void* p : S->pinned_all) cudaFreeHost(p);
  delete S;
}

}  // extern "C"
