// Continuous-batching request server (host runtime, C ABI qmc_server_*).
//
// A request is a VMC evaluation job for one registered wavefunction (a
// molecule at one geometry): draw or upload its walkers, run n_steps
// Metropolis steps (App. B), evaluate the local energies and reduce them to
// the mean and variance (Sec. 1's Monte Carlo estimate).  Requests arrive at
// any time; each is admitted as soon as a stream slot is free and its device
// memory fits in the server's arena (the HBM budget), so requests that arrive
// while others run start immediately and their kernels overlap on the device.
// Memory comes from one arena allocated at creation (first-fit free list with
// coalescing): admission never calls cudaMalloc.  Every request's result is a
// pure function of (wavefunction, walkers or seed, n_steps, step), independent
// of what else is in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "wf_internal.cuh"

using namespace qmc;

namespace {

thread_local std::string g_srv_err;

qmc_status sfail(qmc_status s, const std::string& m) {
  g_srv_err = m;
  return s;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// first-fit allocator over [0, size) with coalescing free list
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void reset(size_t n) {
    size = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, base = it->first + n;
        free_.erase(it);
        if (rest) free_[base] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }
};

struct Pending {
  qmc_request req;
  int64_t ticket;
  double t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;  // the stream of the current request (one of the two below)
  cudaStream_t lo = nullptr;      // lowest priority: large requests
  cudaStream_t hi = nullptr;      // highest priority: the others
  bool big = false;               // the current request is a large one
  cudaEvent_t done = nullptr;
  bool busy = false;
  Pending job{};
  size_t off = 0, bytes = 0;
  double* host = nullptr;  // pinned [6]: mean, variance, non-finite count, accepted moves, status word (bytes of [4])
  bool cancelled = false;  // qmc_server_cancel while in flight: reported as cancelled on retirement
  double t_admit = 0.0;
};

}  // namespace

struct qmc_server {
  int device = 0;
  int64_t big_walkers = 65536;  // requests with at least this many walkers are large
  int32_t max_big = 2;          // large requests in flight at once
  void* arena_base = nullptr;
  Arena arena;
  std::vector<qmc_wf*> wfs;
  std::vector<InitSpec> homes;
  std::deque<Pending> queue;
  std::vector<Slot> slots;
  std::vector<qmc_result> results;
  int64_t next_ticket = 0;
};

namespace {

// electrons dealt to nuclei in proportion to Z with alternating spins (up
// electrons first), the positions the initial walkers are drawn around
InitSpec make_homes(const qmc_wf* wf) {
  const HostSpec& h = wf->spec;
  std::vector<int> ups, downs;
  int c = 0;
  for (int a = 0; a < h.na; ++a)
    for (int k = 0; k < (int)std::lround(h.z[a]); ++k) (c++ % 2 == 0 ? ups : downs).push_back(a);
  for (int k = 0; (int)ups.size() < h.nup; ++k) ups.push_back(k % h.na);
  for (int k = 0; (int)downs.size() < h.ndn; ++k) downs.push_back(k % h.na);
  InitSpec s{};
  s.n_elec = h.nup + h.ndn;
  for (int i = 0; i < s.n_elec; ++i) {
    const int a = i < h.nup ? ups[i] : downs[i - h.nup];
    for (int d = 0; d < 3; ++d) s.home_xyz[i][d] = wf->dev.atom_xyz[a][d];
  }
  return s;
}

size_t request_bytes(qmc_wf* wf, int64_t W) {
  const int N = wf->dev.n_elec;
  return a256(sizeof(double) * 3 * N * W) + a256(sizeof(double) * W) + a256(sizeof(int64_t) * W) +
         a256(sizeof(double) * 8) + a256(qmc_workspace_size(wf, W));
}

qmc_status launch_job(qmc_server* srv, Slot& sl) {
  const qmc_request& r = sl.job.req;
  qmc_wf* wf = srv->wfs[r.wf_id];
  const int64_t W = r.n_walkers;
  const int N = wf->dev.n_elec;
  char* p = static_cast<char*>(srv->arena_base) + sl.off;
  double* walkers = reinterpret_cast<double*>(p);
  p += a256(sizeof(double) * 3 * N * W);
  double* e_loc = reinterpret_cast<double*>(p);
  p += a256(sizeof(double) * W);
  int64_t* acc = reinterpret_cast<int64_t*>(p);
  p += a256(sizeof(int64_t) * W);
  double* stats = reinterpret_cast<double*>(p);  // mean, variance, non-finite count, accepted moves
  p += a256(sizeof(double) * 8);
  void* ws = p;
  const size_t ws_bytes = qmc_workspace_size(wf, W);
  cudaStream_t st = sl.stream;
  cudaError_t e;
  if (r.walkers) e = cudaMemcpyAsync(walkers, r.walkers, sizeof(double) * 3 * N * W, cudaMemcpyHostToDevice, st);
  else e = launch_init_walkers(srv->homes[r.wf_id], W, W, walkers, r.seed, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(int64_t) * W, st);
  // the workspace's status word records a bounded device wait that gave up,
  // over the whole request (cleared once here, read at retirement)
  int* status = workspace_status(wf, ws, W);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return sfail(QMC_ERR_CUDA, std::string("request setup: ") + cudaGetErrorString(e));
  qmc_status s = QMC_OK;
  if (r.n_steps > 0)
    s = sample_call(wf, walkers, W, W, r.n_steps, r.step, r.seed, 0, 0, nullptr, acc, ws, ws_bytes, st, false);
  if (s == QMC_OK) s = local_energy_call(wf, walkers, W, W, e_loc, nullptr, ws, ws_bytes, st, false);
  if (s != QMC_OK) return sfail(s, std::string("request kernels: ") + qmc_last_error());
  e = launch_mean_var_finite(e_loc, W, stats, st);
  if (e == cudaSuccess) e = launch_sum_counts(acc, W, stats + 3, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.host, stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
  sl.host[4] = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sl.host[4], status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) return sfail(QMC_ERR_CUDA, std::string("request reduction: ") + cudaGetErrorString(e));
  return QMC_OK;
}

}  // namespace

extern "C" {

qmc_status qmc_server_create(int32_t device, size_t hbm_budget_bytes, int32_t max_in_flight, qmc_server** out) {
  if (!out || max_in_flight < 1 || max_in_flight > 256 || hbm_budget_bytes < (1u << 20))
    return sfail(QMC_ERR_ARG, "bad server arguments");
  *out = nullptr;
  qmc_server* srv = new qmc_server();
  srv->device = device;
  DeviceGuard guard(device);
  cudaError_t e = cudaMalloc(&srv->arena_base, hbm_budget_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return sfail(QMC_ERR_OOM, std::string("server arena: ") + cudaGetErrorString(e));
  }
  srv->arena.reset(hbm_budget_bytes);
  srv->slots.resize(max_in_flight);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (auto& sl : srv->slots) {
    e = cudaStreamCreateWithPriority(&sl.lo, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.hi, cudaStreamNonBlocking, greatest);
    sl.stream = sl.hi;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.host, sizeof(double) * 6);
    if (e != cudaSuccess) {
      qmc_server_destroy(srv);
      return sfail(QMC_ERR_CUDA, std::string("server slots: ") + cudaGetErrorString(e));
    }
  }
  *out = srv;
  return QMC_OK;
}

void qmc_server_destroy(qmc_server* srv) {
  if (!srv) return;
  {
    DeviceGuard guard(srv->device);
    for (auto& sl : srv->slots) {
      for (cudaStream_t q : {sl.lo, sl.hi})
        if (q) cudaStreamSynchronize(q);
      if (sl.done) cudaEventDestroy(sl.done);
      for (cudaStream_t q : {sl.lo, sl.hi})
        if (q) cudaStreamDestroy(q);
      if (sl.host) cudaFreeHost(sl.host);
    }
    if (srv->arena_base) cudaFree(srv->arena_base);
  }
  delete srv;
}

qmc_status qmc_server_add_wf(qmc_server* srv, qmc_wf* wf, int32_t* wf_id) {
  if (!srv || !wf || !wf_id) return sfail(QMC_ERR_ARG, "null argument");
  if (wf->device != srv->device) return sfail(QMC_ERR_ARG, "wavefunction lives on another device");
  srv->wfs.push_back(wf);
  srv->homes.push_back(make_homes(wf));
  *wf_id = (int32_t)srv->wfs.size() - 1;
  return QMC_OK;
}

qmc_status qmc_server_submit(qmc_server* srv, const qmc_request* req, int64_t* ticket) {
  if (!srv || !req || !ticket) return sfail(QMC_ERR_ARG, "null argument");
  if (req->wf_id < 0 || req->wf_id >= (int32_t)srv->wfs.size()) return sfail(QMC_ERR_ARG, "unknown wavefunction");
  if (req->n_walkers < 1 || req->n_steps < 0 || (req->n_steps > 0 && !(req->step > 0.0)))
    return sfail(QMC_ERR_ARG, "bad request sizes");
  if (request_bytes(srv->wfs[req->wf_id], req->n_walkers) > srv->arena.size)
    return sfail(QMC_ERR_OOM, "request larger than the whole device-memory budget");
  Pending p{*req, srv->next_ticket++, now_s()};
  srv->queue.push_back(p);
  *ticket = p.ticket;
  return QMC_OK;
}

qmc_status qmc_server_progress(qmc_server* srv, int32_t* n_in_flight, int32_t* n_queued) {
  if (!srv) return sfail(QMC_ERR_ARG, "null server");
  DeviceGuard guard(srv->device);
  // retire finished requests
  for (auto& sl : srv->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    qmc_result res{};
    res.ticket = sl.job.ticket;
    res.wf_id = sl.job.req.wf_id;
    res.n_walkers = sl.job.req.n_walkers;
    res.t_submit = sl.job.t_submit;
    res.t_admit = sl.t_admit;
    res.t_done = now_s();
    int timed_out = 0;
    std::memcpy(&timed_out, &sl.host[4], sizeof(int));
    if (sl.cancelled) {
      res.status = QMC_ERR_CANCELLED;
      res.e_mean = res.e_var = res.accept_rate = NAN;
    } else if (q == cudaSuccess && timed_out) {
      res.status = QMC_ERR_TIMEOUT;
      res.e_mean = res.e_var = res.accept_rate = NAN;
    } else if (q == cudaSuccess) {
      res.status = QMC_OK;
      res.e_mean = sl.host[0];
      res.e_var = sl.host[1];
      res.n_nonfinite = (int64_t)sl.host[2];
      const double moves = (double)sl.job.req.n_walkers * sl.job.req.n_steps;
      res.accept_rate = moves > 0 ? sl.host[3] / moves : 0.0;
    } else {
      res.status = QMC_ERR_CUDA;
      res.e_mean = res.e_var = res.accept_rate = NAN;
    }
    srv->results.push_back(res);
    srv->arena.release(sl.off, sl.bytes);
    sl.busy = false;
    sl.cancelled = false;
  }
  // Admit queued requests in arrival order while a slot and memory are free.
  // Large requests (>= big_walkers walkers) keep their arrival order among
  // themselves and at most max_big of them run at once, on low-priority
  // streams; smaller requests may pass a large one that has to wait, and run
  // on high-priority streams, so their kernels fill the device between the
  // large requests' blocks instead of queueing behind them.  Memory stays
  // first-come: a request that does not fit stops the admission.
  qmc_status status = QMC_OK;
  int n_big = 0;
  for (auto& sl : srv->slots) n_big += (sl.busy && sl.big) ? 1 : 0;
  for (auto it = srv->queue.begin(); it != srv->queue.end();) {
    const bool big = srv->big_walkers > 0 && it->req.n_walkers >= srv->big_walkers;
    if (big && n_big >= srv->max_big) {
      ++it;
      continue;
    }
    Slot* free_slot = nullptr;
    for (auto& sl : srv->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    if (!free_slot) break;
    Pending& head = *it;
    const size_t need = request_bytes(srv->wfs[head.req.wf_id], head.req.n_walkers);
    size_t off;
    if (!srv->arena.alloc(need, &off)) break;
    Slot& sl = *free_slot;
    sl.job = head;
    sl.off = off;
    sl.bytes = need;
    sl.busy = true;
    sl.t_admit = now_s();
    sl.big = big;
    sl.stream = big ? sl.lo : sl.hi;
    n_big += big ? 1 : 0;
    it = srv->queue.erase(it);
    const qmc_status s = launch_job(srv, sl);
    if (s != QMC_OK) {
      // report the request as failed and keep serving the others
      cudaStreamSynchronize(sl.stream);
      qmc_result res{};
      res.ticket = sl.job.ticket;
      res.wf_id = sl.job.req.wf_id;
      res.n_walkers = sl.job.req.n_walkers;
      res.status = s;
      res.t_submit = sl.job.t_submit;
      res.t_admit = res.t_done = now_s();
      res.e_mean = res.e_var = res.accept_rate = NAN;
      srv->results.push_back(res);
      srv->arena.release(sl.off, sl.bytes);
      sl.busy = false;
      n_big -= big ? 1 : 0;
      status = s;
    }
  }
  if (n_in_flight) {
    int k = 0;
    for (auto& sl : srv->slots) k += sl.busy ? 1 : 0;
    *n_in_flight = k;
  }
  if (n_queued) *n_queued = (int32_t)srv->queue.size();
  return status;
}

qmc_status qmc_server_results(qmc_server* srv, qmc_result* out, int32_t capacity, int32_t* n_out) {
  if (!srv || !n_out || (capacity > 0 && !out)) return sfail(QMC_ERR_ARG, "bad argument");
  const int32_t n = std::min<int32_t>(capacity, (int32_t)srv->results.size());
  for (int32_t k = 0; k < n; ++k) out[k] = srv->results[k];
  srv->results.erase(srv->results.begin(), srv->results.begin() + n);
  *n_out = n;
  return QMC_OK;
}

qmc_status qmc_server_cancel(qmc_server* srv, int64_t ticket) {
  if (!srv) return sfail(QMC_ERR_ARG, "null server");
  for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
    if (it->ticket == ticket) {  // never admitted: no device work, no memory
      qmc_result res{};
      res.ticket = ticket;
      res.status = QMC_ERR_CANCELLED;
      res.wf_id = it->req.wf_id;
      res.n_walkers = it->req.n_walkers;
      res.e_mean = res.e_var = res.accept_rate = NAN;
      res.t_submit = it->t_submit;
      res.t_admit = res.t_done = now_s();
      srv->results.push_back(res);
      srv->queue.erase(it);
      return QMC_OK;
    }
  for (auto& sl : srv->slots)
    if (sl.busy && sl.job.ticket == ticket) {  // in flight: its kernels finish, its result is dropped
      sl.cancelled = true;
      return QMC_OK;
    }
  return sfail(QMC_ERR_ARG, "ticket " + std::to_string(ticket) + " is neither queued nor in flight");
}

qmc_status qmc_server_set_policy(qmc_server* srv, int64_t big_walkers, int32_t max_big_in_flight) {
  if (!srv || big_walkers < 0 || max_big_in_flight < 1) return sfail(QMC_ERR_ARG, "bad policy arguments");
  srv->big_walkers = big_walkers;
  srv->max_big = max_big_in_flight;
  return QMC_OK;
}

size_t qmc_server_free_bytes(const qmc_server* srv) { return srv ? srv->arena.free_bytes() : 0; }

double qmc_server_clock(void) { return now_s(); }

const char* qmc_server_last_error(void) { return g_srv_err.c_str(); }

}  // extern "C"
