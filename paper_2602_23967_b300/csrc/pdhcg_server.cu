// pdhcg_server.cu — serving loop with continuous batching (pdhcg_server_*).
//
// Two host threads own the device side.
//   Admission thread: takes queued requests while a slot is free and their
//     device footprint fits the HBM budget.  The small ones it took are
//     created together with the batched creation path (one allocation, one
//     setup launch), then one large one, and the thread looks at the queue
//     again, so small requests never wait behind the preparation of several
//     large ones.  Creation runs on its own stream and overlaps the slices of
//     the running solves.  Finished handles go to a ready list.
//   Slice thread: at each slice boundary moves ready handles into free slots,
//     advances every live solve by one slice of 10 ms of device time
//     (PDHCG_SLICE_US) in a single pooled launch (iterates, anchors, PID and restart state stay
//     on the device between slices), then retires the solves that stopped:
//     copies their results and solutions to host memory in one batch and frees
//     their device memory and slot.
// Requests join and leave the running set at slice boundaries, i.e. at
// iteration granularity.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_problem.h"

namespace pdhcg {

// Deep copy of one submitted problem.
struct OwnedProblem {
  bool has_q = false;
  int32_t n = 0, m = 0;
  std::vector<int64_t> qp, ap;
  std::vector<int32_t> qc, ac;
  std::vector<double> qv, av, c, lc, uc, lv, uv;
  pdhcg_csr Q{}, A{};
  void bind() {
    Q = pdhcg_csr{n, n, int64_t(qc.size()), qp.data(), qc.data(), qv.data()};
    A = pdhcg_csr{m, n, int64_t(ac.size()), ap.data(), ac.data(), av.data()};
  }
  CreateInput input() const {
    return CreateInput{has_q ? &Q : nullptr, &A, c.data(), lc.data(), uc.data(), lv.data(), uv.data()};
  }
};

struct Request {
  uint64_t ticket = 0;
  OwnedProblem prob;
  size_t bytes = 0;
  std::chrono::steady_clock::time_point t_submit;
};

struct Live {
  uint64_t ticket = 0;
  pdhcg_problem* P = nullptr;
  size_t bytes = 0;
  int slot = -1;
  std::chrono::steady_clock::time_point t_submit;
};

static double seconds_since(std::chrono::steady_clock::time_point t) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
}

struct Done {
  pdhcg_result res{};
  std::vector<double> x, y;
};

}  // namespace pdhcg

struct pdhcg_server {
  size_t budget = 0;
  int max_slots = 0;
  size_t max_queue = 0;
// A slice advances every live solve for PDHCG_SLICE_US microseconds of device
// time (instances differ in cost per step, so a fixed step count would leave the
// CTAs of small instances idle while the largest finish); with
// PDHCG_SLICE_US = 0, for PDHCG_SLICE_ITERS steps instead.
#ifndef PDHCG_SLICE_US
#define PDHCG_SLICE_US 10000
#endif
#ifndef PDHCG_SLICE_ITERS
#define PDHCG_SLICE_ITERS 256
#endif
  int64_t slice_iters = PDHCG_SLICE_US > 0 ? 0 : PDHCG_SLICE_ITERS;
  uint64_t slice_ns = uint64_t(PDHCG_SLICE_US) * 1000u;
  pdhcg_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // admission thread: new requests, freed capacity, stop
  std::condition_variable cv_work;  // slice thread: ready handles, stop
  std::deque<pdhcg::Request> queue;
  std::vector<pdhcg::Live> ready;   // created and set up, waiting for a slot
  int reserved = 0;                 // requests taken for creation, ready or live (<= max_slots)
  cudaStream_t admit_stream = nullptr;
  // large requests' multi-CTA groups run in a cooperative launch of their own on
  // group_stream, beside the pool launch of the slice
  cudaStream_t group_stream = nullptr;  // lowest priority: waiting pool CTAs go first
  int prio_low = 0, prio_high = 0;
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
  std::thread admitter;
  cudaMemPool_t pool = nullptr;     // device arenas of admitted requests (stream-ordered)
  void* pinned_stage = nullptr;     // creation's host staging, reused
  size_t pinned_stage_bytes = 0;
  std::unordered_map<uint64_t, pdhcg::Done> done;
  std::unordered_map<uint64_t, int> pending;  // ticket -> 1 (queued or live)
  uint64_t next_ticket = 1;
  pdhcg_server_stats stats{};
  bool stop = false;
  std::thread worker;
  // device side (worker thread only)
  pdhcg::SolverState* d_states = nullptr;  // max_slots, indexed by slot
  void* d_launch = nullptr;                 // launch descriptors of one slice
  size_t launch_bytes = 0;
  pdhcg::SolverState* h_states = nullptr;   // pinned copy of d_states
  pdhcg::SolverState* h_init = nullptr;     // pinned initial states, by slot
  double* h_sol = nullptr;                  // pinned staging of finished solutions
  size_t h_sol_len = 0;
  double* d_out = nullptr;                  // per-slot solution buffers live in each handle
  std::vector<pdhcg::Live> live;
  std::vector<int> free_slots;
  std::string worker_error;
};

namespace pdhcg {

static void copy_csr(const pdhcg_csr* M, std::vector<int64_t>& rp, std::vector<int32_t>& ci,
                     std::vector<double>& v) {
  rp.assign(M->rowptr, M->rowptr + M->nrows + 1);
  ci.assign(M->col, M->col + M->nnz);
  v.assign(M->val, M->val + M->nnz);
}

// Creation and device setup of admitted requests on the admission stream (one
// batch: one allocation, one setup launch), then they join the ready list.
static void admit_batch(pdhcg_server* S, std::vector<Request>& admit) {
  const auto t_adm0 = std::chrono::steady_clock::now();
  std::vector<CreateInput> in;
  in.reserve(admit.size());
  for (auto& r : admit) {
    r.prob.bind();
    in.push_back(r.prob.input());
  }
  std::vector<pdhcg_problem*> handles(admit.size(), nullptr);
  CreateAlloc al;
  al.pool = S->pool;
  al.pinned = &S->pinned_stage;
  al.pinned_bytes = &S->pinned_stage_bytes;
  int rc = create_impl(int(admit.size()), in.data(), &S->prm, S->admit_stream, handles.data(), true, &al);
  if (rc != PDHCG_OK && admit.size() > 1) {
    // fall back to one-by-one so one bad request fails alone
    for (size_t i = 0; i < admit.size(); ++i) {
      rc = create_impl(1, &in[i], &S->prm, S->admit_stream, &handles[i], true, &al);
      if (rc != PDHCG_OK) handles[i] = nullptr;
    }
  } else if (rc != PDHCG_OK) {
    handles[0] = nullptr;
  }
  // creation synchronised its stream; the solves run on the slice stream
  for (auto* h : handles)
    if (h) h->stream = S->stream;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < admit.size(); ++i) {
      if (!handles[i]) {
        Done d;
        d.res.status = PDHCG_NUMERICAL_ERROR;
        d.res.latency_seconds = seconds_since(admit[i].t_submit);
        S->done[admit[i].ticket] = std::move(d);
        S->pending.erase(admit[i].ticket);
        S->stats.rejected++;
        S->stats.hbm_in_use -= admit[i].bytes;
        S->reserved--;
        continue;
      }
      Live l;
      l.ticket = admit[i].ticket;
      l.P = handles[i];
      l.bytes = admit[i].bytes;
      l.t_submit = admit[i].t_submit;
      S->ready.push_back(l);
      S->stats.admitted++;
    }
    S->stats.admit_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_adm0).count();
  }
  S->cv_work.notify_one();
}

// Takes queued requests while a slot and the HBM budget allow.  Small requests
// are created together as one batch; large ones (multi-CTA groups) one per
// round, after the small ones taken in that round, so a large request's host
// preparation and setup never holds back small requests queued meanwhile.
static void admit_loop(pdhcg_server* S) {
  cudaSetDevice(S->device);
  std::deque<Request> large;  // taken from the queue, not yet created
  while (true) {
    std::vector<Request> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      auto can_take = [&] {
        return !S->queue.empty() && S->reserved < S->max_slots &&
               S->stats.hbm_in_use + S->queue.front().bytes <= S->budget;
      };
      if (large.empty()) S->cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return S->stop || can_take(); });
      if (S->stop) break;
      while (can_take()) {
        S->stats.hbm_in_use += S->queue.front().bytes;  // reserved until retirement
        S->reserved++;
        admit.push_back(std::move(S->queue.front()));
        S->queue.pop_front();
      }
      S->stats.queued = int32_t(S->queue.size());
    }
    std::vector<Request> small;
    for (auto& r : admit) {
      const OwnedProblem& p = r.prob;
      const int64_t work = int64_t(p.qc.size()) + 2 * int64_t(p.ac.size()) + p.n + p.m;
      if (work < kGroupWork) small.push_back(std::move(r));
      else large.push_back(std::move(r));
    }
    if (!small.empty()) admit_batch(S, small);
    if (!large.empty()) {
      std::vector<Request> one;
      one.push_back(std::move(large.front()));
      large.pop_front();
      admit_batch(S, one);
    }
  }
}

static void worker_loop(pdhcg_server* S) {
  cudaSetDevice(S->device);
  while (true) {
    // a failed copy or synchronisation of this round: every live solve then
    // retires with PDHCG_NUMERICAL_ERROR (its state cannot be trusted)
    cudaError_t ce = cudaSuccess;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->live.empty())
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return S->stop || !S->ready.empty(); });
      if (S->stop) break;
      // ---- ready handles take free slots (their initial state goes to the slot) ----
      for (auto& l : S->ready) {
        l.slot = S->free_slots.back();
        S->free_slots.pop_back();
        S->h_init[l.slot] = initial_state(l.P);
        const cudaError_t e = cudaMemcpyAsync(S->d_states + l.slot, S->h_init + l.slot, sizeof(SolverState),
                                              cudaMemcpyHostToDevice, S->stream);
        if (ce == cudaSuccess) ce = e;
        S->live.push_back(l);
      }
      S->ready.clear();
      S->stats.live = int32_t(S->live.size());
    }
    if (S->live.empty()) continue;
    // ---- one slice over every live solve (states addressed by slot) ----
    const auto t_slice0 = std::chrono::steady_clock::now();
    const int count = int(S->live.size());
    std::vector<pdhcg_problem*> probs(static_cast<size_t>(count));
    std::vector<double*> xo(static_cast<size_t>(count)), yo(static_cast<size_t>(count));
    std::vector<int> slots(static_cast<size_t>(count));
    for (int i = 0; i < count; ++i) {
      const Live& l = S->live[size_t(i)];
      probs[size_t(i)] = l.P;
      xo[size_t(i)] = l.P->x_stage;
      yo[size_t(i)] = l.P->y_stage;
      slots[size_t(i)] = l.slot;
    }
    int rc = ce == cudaSuccess ? launch_pool_slice(probs.data(), count, S->d_states, xo.data(), yo.data(),
                                                   S->slice_iters, slots.data(), S->d_launch, S->launch_bytes,
                                                   S->slice_ns, S->group_stream, S->ev_ready, S->ev_done)
                               : PDHCG_E_CUDA;
    {
      cudaError_t e = cudaMemcpyAsync(S->h_states, S->d_states, sizeof(SolverState) * size_t(S->max_slots),
                                      cudaMemcpyDeviceToHost, S->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
      if (e != cudaSuccess && rc == PDHCG_OK) rc = PDHCG_E_CUDA;
    }
    if (rc != PDHCG_OK) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->worker_error = std::string("slice: ") + (ce != cudaSuccess ? cudaGetErrorString(ce) : "launch or copy failed");
    }
    const auto t_slice1 = std::chrono::steady_clock::now();
    // ---- retire finished solves: their solutions come back in one batch ----
    std::vector<int> fin;
    size_t need = 0;
    for (int i = 0; i < count; ++i) {
      const SolverState& st = S->h_states[S->live[size_t(i)].slot];
      if (st.status != 0 || st.device_error || rc != PDHCG_OK) {
        fin.push_back(i);
        need += size_t(S->live[size_t(i)].P->n) + size_t(S->live[size_t(i)].P->m_user);
      }
    }
    if (need > S->h_sol_len) {
      if (S->h_sol) cudaFreeHost(S->h_sol);
      S->h_sol = nullptr;
      S->h_sol_len = 0;
      if (cudaMallocHost(&S->h_sol, sizeof(double) * need * 2) == cudaSuccess) S->h_sol_len = need * 2;
    }
    size_t off = 0;
    bool sol_ok = S->h_sol != nullptr;
    if (S->h_sol) {
      cudaError_t e = cudaSuccess;
      for (int i : fin) {
        const pdhcg_problem* P = S->live[size_t(i)].P;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(S->h_sol + off, P->x_stage, sizeof(double) * size_t(P->n), cudaMemcpyDeviceToHost,
                              S->stream);
        off += size_t(P->n);
        if (P->m_user && e == cudaSuccess)
          e = cudaMemcpyAsync(S->h_sol + off, P->y_stage, sizeof(double) * size_t(P->m_user),
                              cudaMemcpyDeviceToHost, S->stream);
        off += size_t(P->m_user);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
      sol_ok = e == cudaSuccess;
    }
    std::vector<Live> keep;
    keep.reserve(size_t(count));
    std::vector<char> done_flag(static_cast<size_t>(count), 0);
    for (int i : fin) done_flag[size_t(i)] = 1;
    off = 0;
    std::vector<std::pair<uint64_t, Done>> out;
    out.reserve(fin.size());
    for (int i = 0; i < count; ++i) {
      Live& l = S->live[size_t(i)];
      if (!done_flag[size_t(i)]) {
        keep.push_back(l);
        continue;
      }
      const SolverState& st = S->h_states[l.slot];
      Done d;
      fill_result(l.P, st, &d.res);
      if (st.device_error || rc != PDHCG_OK || !sol_ok) d.res.status = PDHCG_NUMERICAL_ERROR;
      const size_t n = size_t(l.P->n), m = size_t(l.P->m_user);
      if (S->h_sol) {
        d.x.assign(S->h_sol + off, S->h_sol + off + n);
        d.y.assign(S->h_sol + off + n, S->h_sol + off + n + m);
      }
      off += n + m;
      pdhcg_destroy(l.P);
      d.res.latency_seconds = seconds_since(l.t_submit);
      out.emplace_back(l.ticket, std::move(d));
    }
    const auto t_retire1 = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t k = 0; k < out.size(); ++k) {
      const Live& l = S->live[size_t(fin[k])];
      S->done[out[k].first] = std::move(out[k].second);
      S->pending.erase(out[k].first);
      S->stats.completed++;
      S->stats.hbm_in_use -= l.bytes;
      S->reserved--;
      S->free_slots.push_back(l.slot);
    }
    if (!out.empty()) S->cv.notify_one();
    S->stats.launches++;
    S->stats.slice_seconds += std::chrono::duration<double>(t_slice1 - t_slice0).count();
    S->stats.retire_seconds += std::chrono::duration<double>(t_retire1 - t_slice1).count();
    S->live.swap(keep);
    S->stats.live = int32_t(S->live.size());
  }
}

}  // namespace pdhcg

using namespace pdhcg;

extern "C" {

int pdhcg_server_create(size_t hbm_budget_bytes, int max_slots, const pdhcg_params* params,
                        void* cuda_stream, pdhcg_server_t** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) {
    set_error("server_create: bad arguments");
    return PDHCG_E_INVALID;
  }
  *out = nullptr;
  auto* S = new pdhcg_server();
  if (params) {
    int rc = check_params_c(params);
    if (rc) {
      delete S;
      return rc;
    }
    S->prm = *params;
  } else {
    pdhcg_default_params(&S->prm);
  }
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->max_queue = size_t(max_slots) * 64;
  S->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&S->device);
  // one slice's descriptors, queue and group scratch (at most 2048 group CTAs)
  S->launch_bytes = batch_scratch_bytes(max_slots, std::min(max_slots, 1024), 2048);
  if (cudaMalloc(&S->d_states, sizeof(SolverState) * size_t(max_slots)) != cudaSuccess ||
      cudaMalloc(&S->d_launch, S->launch_bytes) != cudaSuccess ||
      cudaMallocHost(&S->h_states, sizeof(SolverState) * size_t(max_slots)) != cudaSuccess ||
      cudaMallocHost(&S->h_init, sizeof(SolverState) * size_t(max_slots)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->admit_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&S->prio_low, &S->prio_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&S->group_stream, cudaStreamNonBlocking, S->prio_low) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    if (S->d_states) cudaFree(S->d_states);
    if (S->d_launch) cudaFree(S->d_launch);
    if (S->h_states) cudaFreeHost(S->h_states);
    if (S->h_init) cudaFreeHost(S->h_init);
    if (S->admit_stream) cudaStreamDestroy(S->admit_stream);
    if (S->group_stream) cudaStreamDestroy(S->group_stream);
    if (S->ev_ready) cudaEventDestroy(S->ev_ready);
    if (S->ev_done) cudaEventDestroy(S->ev_done);
    delete S;
    set_error("server_create: allocation failed");
    return PDHCG_E_OOM;
  }
  {
    // a pool of its own that keeps freed arenas for reuse (no release at syncs)
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) == cudaSuccess) {
      uint64_t keep = uint64_t(hbm_budget_bytes);
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      S->pool = nullptr;  // fall back to cudaMalloc / cudaFree
    }
  }
  for (int i = max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->worker = std::thread(worker_loop, S);
  S->admitter = std::thread(admit_loop, S);
  *out = S;
  return PDHCG_OK;
}

int pdhcg_submit(pdhcg_server_t* S, const pdhcg_csr* Q, const pdhcg_csr* A, const double* c,
                 const double* lc, const double* uc, const double* lv, const double* uv, uint64_t* ticket) {
  if (!S || !A || !ticket) {
    set_error("submit: bad arguments");
    return PDHCG_E_INVALID;
  }
  Request r;
  CreateInput in{Q, A, c, lc, uc, lv, uv};
  int rc = footprint_of(in, S->prm, &r.bytes);  // validates the problem, host side only
  if (rc) return rc;
  if (r.bytes > S->budget) {
    set_error("submit: the problem alone exceeds the HBM budget");
    return PDHCG_E_OOM;
  }
  OwnedProblem& p = r.prob;
  p.n = A->ncols;
  p.m = A->nrows;
  p.has_q = Q != nullptr;
  if (Q) copy_csr(Q, p.qp, p.qc, p.qv);
  copy_csr(A, p.ap, p.ac, p.av);
  p.c.assign(c, c + p.n);
  p.lv.assign(lv, lv + p.n);
  p.uv.assign(uv, uv + p.n);
  if (p.m) {
    p.lc.assign(lc, lc + p.m);
    p.uc.assign(uc, uc + p.m);
  }
  r.t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= S->max_queue) {
      set_error("submit: queue full");
      return PDHCG_E_BUSY;
    }
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    S->pending[r.ticket] = 1;
    S->queue.push_back(std::move(r));
    S->stats.submitted++;
    S->stats.queued = int32_t(S->queue.size());
  }
  S->cv.notify_one();
  return PDHCG_OK;
}

int pdhcg_poll(pdhcg_server_t* S, uint64_t ticket, pdhcg_result* res, double* x_out, double* y_out) {
  if (!S) return PDHCG_E_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it == S->done.end()) {
    if (S->pending.count(ticket)) return PDHCG_PENDING;
    set_error("poll: unknown ticket");
    return PDHCG_E_NOT_FOUND;
  }
  if (res) *res = it->second.res;
  if (x_out && !it->second.x.empty()) std::memcpy(x_out, it->second.x.data(), sizeof(double) * it->second.x.size());
  if (y_out && !it->second.y.empty()) std::memcpy(y_out, it->second.y.data(), sizeof(double) * it->second.y.size());
  S->done.erase(it);
  return PDHCG_OK;
}

int pdhcg_server_get_stats(pdhcg_server_t* S, pdhcg_server_stats* st) {
  if (!S || !st) return PDHCG_E_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->stats;
  return PDHCG_OK;
}

void pdhcg_server_destroy(pdhcg_server_t* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  S->cv_work.notify_all();
  if (S->admitter.joinable()) S->admitter.join();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (auto& l : S->live) pdhcg_destroy(l.P);
  for (auto& l : S->ready) pdhcg_destroy(l.P);
  if (S->admit_stream) cudaStreamSynchronize(S->admit_stream);
  if (S->admit_stream) cudaStreamDestroy(S->admit_stream);
  if (S->group_stream) {
    cudaStreamSynchronize(S->group_stream);
    cudaStreamDestroy(S->group_stream);
  }
  if (S->ev_ready) cudaEventDestroy(S->ev_ready);
  if (S->ev_done) cudaEventDestroy(S->ev_done);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  if (S->pinned_stage) cudaFreeHost(S->pinned_stage);
  if (S->h_init) cudaFreeHost(S->h_init);
  if (S->d_states) cudaFree(S->d_states);
  if (S->d_launch) cudaFree(S->d_launch);
  if (S->h_states) cudaFreeHost(S->h_states);
  if (S->h_sol) cudaFreeHost(S->h_sol);
  delete S;
}

}  // extern "C"
