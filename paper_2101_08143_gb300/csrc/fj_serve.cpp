// fj_serve.cpp - continuous-batching request server behind fj_submit/fj_poll.
//
// One worker thread per context owns the device side of serving:
//   * submitted requests wait in a FIFO queue (inputs already copied);
//   * a request is admitted when an in-flight slot is free and the device
//     memory it needs fits the remaining budget; it then runs on the slot's
//     own stream with its own workspace (graph build for inline requests,
//     H2D of s, the persistent solve, D2H of the quantities into the slot's
//     pinned buffer, an event);
//   * the worker polls the events of in-flight requests and retires them as
//     they finish, freeing memory and slots so that queued requests start
//     while others are still running on the GPU.
// Small requests get small persistent grids, so several run on the GPU at
// once; a request's grid depends only on its own size and the server's cap,
// so its results are the same bits alone or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fj_internal.cuh"

fj_status fj_build_graph_begin(int device, cudaStream_t st, int64_t n, int64_t m, const int32_t* src,
                               const int32_t* dst, const float* w, bool merge_duplicates, int64_t* host_words,
                               fj_graph** pending, int32_t* copy_src = nullptr, int32_t* copy_dst = nullptr,
                               float* copy_w = nullptr);
fj_status fj_build_graph_end(fj_graph* g, const int64_t* host_words, cudaStream_t st, fj_graph** out);
void fj_free_graph_arrays(fj_graph* g, cudaStream_t st);
size_t fj_solve_workspace_bytes(const fj_graph* g, int K, int inner_bytes, int num_sms);
fj_status fj_solve_device(const fj_graph* g, cudaStream_t st, int num_sms, int32_t k, const double* s, double* z,
                          double* quant, double* resid, int* status, char* ws, size_t ws_bytes, const fj_opts& o,
                          int* launches_out, int max_blocks, const double* z0, int* grid_out);

namespace fj {

constexpr int kSlotMaxK = 1024;  // columns per request (pinned result buffers)
constexpr int kBuildWords = 9;   // a graph build's host words (sizes, validation)
// page-locked bytes per slot: quant [k][5] | resid [k] | status words, then
// the build words
constexpr size_t kSlotResultBytes = (size_t)kSlotMaxK * 6 * 8 + 64 * 12;
constexpr size_t kSlotPinnedBytes = kSlotResultBytes + kBuildWords * 8;

struct Request {
  uint64_t id = 0;
  // input
  const fj_graph* graph = nullptr;  // caller's graph, or
  int64_t n = 0, m = 0;             // an inline edge list
  std::vector<int32_t> src, dst;
  std::vector<float> w;
  bool weighted = false;
  int32_t k = 0;
  std::vector<double> s;
  fj_opts opts{};
  size_t mem_est = 0;
  // running state
  int slot = -1;
  int block_cap = 0;  // grid cap of the request's solve, fixed at admission
  fj_graph* own_graph = nullptr;
  fj_graph* building = nullptr;  // inline graph whose build is in flight (ev marks its end)
  char* dev = nullptr;  // one device allocation: s | quant | resid | status | workspace
  cudaEvent_t ev = nullptr;
  int launches = 0;
  // result
  bool done = false;
  fj_status rc = FJ_OK;
  std::vector<fj_quant> quant;
  fj_info info{};
  std::chrono::steady_clock::time_point t_submit, t_start;
};

struct Slot {
  cudaStream_t stream = nullptr;
  double* pinned = nullptr;  // quant [k][5] | resid [k] | status words
  bool busy = false;
};

struct Server {
  int device = 0;
  int num_sms = 0;
  int max_inflight = 16;
  int64_t budget = 0;
  int max_blocks = 0;  // per-request grid cap (0: automatic, see block_cap)
  int64_t used = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> inflight;
  std::unordered_map<uint64_t, Request*> all;
  std::deque<Slot> slots;  // grows in place: references to slots stay valid
  std::thread worker;
  std::string init_error;

  ~Server() {
    {
      std::lock_guard<std::mutex> lock(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (worker.joinable()) worker.join();
    cudaSetDevice(device);
    for (auto& sl : slots) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    for (auto& kv : all) delete kv.second;
  }
};

namespace {

size_t estimate_bytes(const Request& r, int num_sms) {
  // inline graph: sort buffers + CSR + sliced ELL, about 80 bytes per entry
  size_t b = 0;
  int64_t n = r.graph ? r.graph->n : r.n;
  if (!r.graph) b += (size_t)(2 * r.m + 64) * 80 + (size_t)n * 64;
  const int K = std::min<int>(32, r.k);
  const int inner = r.opts.precision == FJ_PREC_FP64 ? 8 : 4;
  b += (size_t)n * K * (24 + 6 * inner) + (size_t)num_sms * 4 * 16 * K * 16 + (size_t)n * r.k * 8 + (1 << 20);
  return b;
}

// Grid cap of one request's solve: the configured one, else the device's
// co-resident solve blocks (two per SM) shared by the in-flight requests, so
// that they run side by side instead of one at a time.
int block_cap(const Server& S) {
  if (S.max_blocks > 0) return S.max_blocks;
  return std::max(1, 2 * S.num_sms / std::max(1, S.max_inflight));
}

void finish(Server& S, Request* r, fj_status rc) {
  r->rc = rc;
  r->done = true;
  r->info.status = rc;
  r->info.columns = r->k;
}

int64_t* build_words(Server& S, const Request* r) {
  return reinterpret_cast<int64_t*>(reinterpret_cast<char*>(S.slots[r->slot].pinned) + kSlotResultBytes);
}

// Launches the request's own graph build on its slot's stream and records
// r->ev after the copy of the build's host words; the solve starts once that
// event has completed (start_solve), so the worker thread never waits for a
// build.  Returns an error code if it could not be started.
fj_status start_build(Server& S, Request* r) {
  Slot& sl = S.slots[r->slot];
  cudaStream_t st = sl.stream;
  cudaSetDevice(S.device);
  int32_t *ds = nullptr, *dd = nullptr;
  float* dw = nullptr;
  const size_t eb = (size_t)std::max<int64_t>(r->m, 1) * 4;
  if (malloc_async(&ds, eb, st) != cudaSuccess || malloc_async(&dd, eb, st) != cudaSuccess ||
      (r->weighted && malloc_async(&dw, eb, st) != cudaSuccess)) {
    cudaGetLastError();
    if (ds) cudaFreeAsync(ds, st);
    if (dd) cudaFreeAsync(dd, st);
    set_error("fj_submit_edges: out of device memory for the edge list");
    return FJ_ERR_OOM;
  }
  if (r->m > 0) {
    cudaMemcpyAsync(ds, r->src.data(), r->m * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dd, r->dst.data(), r->m * 4, cudaMemcpyHostToDevice, st);
    if (r->weighted) cudaMemcpyAsync(dw, r->w.data(), r->m * 4, cudaMemcpyHostToDevice, st);
  }
  fj_graph* pending = nullptr;
  fj_status rc = fj_build_graph_begin(S.device, st, r->n, r->m, ds, dd, r->weighted ? dw : nullptr,
                                      (r->opts.flags & FJ_MERGE_DUPLICATES) != 0, build_words(S, r), &pending);
  cudaFreeAsync(ds, st);
  cudaFreeAsync(dd, st);
  if (dw) cudaFreeAsync(dw, st);
  if (rc != FJ_OK) return rc;
  r->building = pending;
  cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  cudaEventRecord(r->ev, st);
  return FJ_OK;
}

// Launches the solve on the slot's stream (the graph is resident: the
// caller's, or the request's own once its build has ended).
fj_status start_solve(Server& S, Request* r) {
  Slot& sl = S.slots[r->slot];
  cudaStream_t st = sl.stream;
  cudaSetDevice(S.device);
  if (r->building) {
    fj_graph* og = nullptr;
    fj_graph* g0 = r->building;
    r->building = nullptr;
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
    fj_status rc = fj_build_graph_end(g0, build_words(S, r), st, &og);
    if (rc != FJ_OK) return rc;
    r->own_graph = og;
    std::vector<int32_t>().swap(r->src);
    std::vector<int32_t>().swap(r->dst);
    std::vector<float>().swap(r->w);
  }
  const fj_graph* g = r->graph ? r->graph : r->own_graph;
  const int64_t n = g->n;
  int Ks[64], launches = 0;
  for (int col = 0; col < r->k;) {
    int K = 32;
    while (K > r->k - col) K >>= 1;
    Ks[launches++] = K;
    col += K;
  }
  const int inner = r->opts.precision == FJ_PREC_FP64 ? 8 : 4;
  size_t ws = 0;
  for (int i = 0; i < launches; ++i) ws = std::max(ws, fj_solve_workspace_bytes(g, Ks[i], inner, S.num_sms));
  const size_t s_bytes = ((size_t)n * r->k * 8 + 255) & ~size_t(255);
  const size_t small = ((size_t)r->k * 6 * 8 + (size_t)launches * 12 + 255) & ~size_t(255);
  if (malloc_async(&r->dev, s_bytes + small + ws, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("fj_submit: out of device memory for the solve");
    return FJ_ERR_OOM;
  }
  double* ds = (double*)r->dev;
  double* dq = (double*)(r->dev + s_bytes);
  double* dres = dq + (size_t)r->k * 5;
  int* dstat = (int*)(dres + r->k);
  cudaMemcpyAsync(ds, r->s.data(), (size_t)n * r->k * 8, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(dstat, 0, (size_t)launches * 12, st);
  fj_opts o = r->opts;
  o.flags = FJ_DEVICE_PTRS;
  fj_status rc = fj_solve_device(g, st, S.num_sms, r->k, ds, nullptr, dq, dres, dstat, r->dev + s_bytes + small,
                                 ws, o, &r->launches, r->block_cap, nullptr, &r->info.blocks);
  if (rc != FJ_OK) return rc;
  cudaMemcpyAsync(sl.pinned, dq, (size_t)r->k * 6 * 8 + (size_t)launches * 12, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(r->dev, st);
  r->dev = nullptr;
  if (r->own_graph) fj_free_graph_arrays(r->own_graph, st);
  cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  cudaEventRecord(r->ev, st);
  std::vector<double>().swap(r->s);
  return FJ_OK;
}

void collect(Server& S, Request* r) {
  Slot& sl = S.slots[r->slot];
  const double* hq = sl.pinned;
  const double* hres = hq + (size_t)r->k * 5;
  const int* hstat = (const int*)(hres + r->k);
  r->quant.resize(r->k);
  memcpy(r->quant.data(), hq, (size_t)r->k * 5 * 8);
  int bits = 0, iters = 0, refines = 0;
  for (int i = 0; i < r->launches; ++i) {
    bits |= hstat[3 * i];
    iters = std::max(iters, hstat[3 * i + 1]);
    refines = std::max(refines, hstat[3 * i + 2]);
  }
  double worst = 0.0;
  for (int j = 0; j < r->k; ++j) worst = std::max(worst, hres[j]);
  fj_status rc = FJ_OK;
  if (bits & kErrTimeout)
    rc = FJ_ERR_TIMEOUT;
  else if (bits & kErrNumeric)
    rc = FJ_ERR_NUMERIC;
  else if (bits & kErrNotConverged)
    rc = FJ_ERR_NOT_CONVERGED;
  r->info.iterations = iters;
  r->info.refinements = refines;
  r->info.rel_residual = worst;
  r->info.warnings = (bits & kWarnOpinionRange) ? FJ_WARN_OPINION_RANGE : 0u;
  r->info.device_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->t_start).count();
  if (r->own_graph) {
    delete r->own_graph;  // arrays were freed stream-ordered at launch time
    r->own_graph = nullptr;
  }
  cudaEventDestroy(r->ev);
  r->ev = nullptr;
  finish(S, r, rc);
}

// A request that could not be started (or whose graph was bad): free what
// it holds on its slot's stream, release the slot, complete it with rc.
void abandon(Server& S, Request* r, fj_status rc) {
  cudaStream_t st = S.slots[r->slot].stream;
  S.slots[r->slot].busy = false;
  S.used -= (int64_t)r->mem_est;
  if (r->own_graph) {
    fj_free_graph_arrays(r->own_graph, st);
    delete r->own_graph;
    r->own_graph = nullptr;
  }
  if (r->dev) {
    cudaFreeAsync(r->dev, st);
    r->dev = nullptr;
  }
  if (r->ev) {
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
  }
  finish(S, r, rc);
  S.cv_done.notify_all();
}

void worker_loop(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.device);
  std::unique_lock<std::mutex> lock(S.mu);
  while (true) {
    if (S.stop) break;
    bool progress = false;
    // requests whose graph build ended start their solve; finished requests
    // retire (only this thread changes the in-flight list)
    for (size_t i = 0; i < S.inflight.size();) {
      Request* r = S.inflight[i];
      if (cudaEventQuery(r->ev) != cudaSuccess) {
        ++i;
        continue;
      }
      progress = true;
      if (r->building) {
        lock.unlock();
        const fj_status rc = start_solve(S, r);
        lock.lock();
        if (rc == FJ_OK) {
          ++i;
          continue;
        }
        abandon(S, r, rc);
      } else {
        collect(S, r);
        S.slots[r->slot].busy = false;
        S.used -= (int64_t)r->mem_est;
      }
      S.inflight.erase(S.inflight.begin() + i);
    }
    if (progress) S.cv_done.notify_all();
    // admit in arrival order while a slot and the memory budget allow
    while (!S.pending.empty() && (int)S.inflight.size() < S.max_inflight) {
      Request* r = S.pending.front();
      if (S.used + (int64_t)r->mem_est > S.budget && !S.inflight.empty()) break;
      S.pending.pop_front();
      int slot = 0;
      while (S.slots[slot].busy) ++slot;
      S.slots[slot].busy = true;
      r->slot = slot;
      r->block_cap = block_cap(S);
      S.used += (int64_t)r->mem_est;
      r->t_start = std::chrono::steady_clock::now();
      lock.unlock();
      const fj_status rc = r->graph ? start_solve(S, r) : start_build(S, r);
      lock.lock();
      if (rc != FJ_OK)
        abandon(S, r, rc);
      else
        S.inflight.push_back(r);
      progress = true;
    }
    if (!progress) {
      if (S.inflight.empty() && S.pending.empty())
        S.cv_work.wait(lock);
      else
        S.cv_work.wait_for(lock, std::chrono::microseconds(20));
    }
  }
  // shutdown: drain what is on the GPU, drop what is queued
  for (Request* r : S.inflight) {
    cudaStreamSynchronize(S.slots[r->slot].stream);
    if (r->building) {  // a build that ended: drop its graph
      fj_graph* og = nullptr;
      if (fj_build_graph_end(r->building, build_words(S, r), S.slots[r->slot].stream, &og) == FJ_OK) {
        fj_free_graph_arrays(og, S.slots[r->slot].stream);
        delete og;
      }
      r->building = nullptr;
      cudaEventDestroy(r->ev);
      r->ev = nullptr;
      cudaStreamSynchronize(S.slots[r->slot].stream);
      finish(S, r, FJ_ERR_ARG);
      continue;
    }
    collect(S, r);
  }
  S.inflight.clear();
  for (Request* r : S.pending) finish(S, r, FJ_ERR_ARG);
  S.pending.clear();
  S.cv_done.notify_all();
}

}  // namespace

Server* server_create(int device, int num_sms) {
  Server* S = new Server();
  S->device = device;
  S->num_sms = num_sms;
  cudaSetDevice(device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  S->budget = (int64_t)(free_b / 2);
  S->slots.resize(S->max_inflight);
  for (auto& sl : S->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&sl.pinned, kSlotPinnedBytes) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return nullptr;
    }
  }
  S->worker = std::thread(worker_loop, S);
  return S;
}

void server_destroy(Server* S) { delete S; }

fj_status server_config(Server* S, int32_t max_inflight, int64_t budget, int32_t max_blocks) {
  std::lock_guard<std::mutex> lock(S->mu);
  if (max_inflight > 0) {
    if (max_inflight > (int)S->slots.size()) {
      cudaSetDevice(S->device);
      size_t old = S->slots.size();
      S->slots.resize(max_inflight);
      for (size_t i = old; i < S->slots.size(); ++i) {
        if (cudaStreamCreateWithFlags(&S->slots[i].stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&S->slots[i].pinned, kSlotPinnedBytes) != cudaSuccess) {
          cudaGetLastError();
          S->slots.resize(i);
          set_error("fj_serve_config: could not create slot %zu", i);
          return FJ_ERR_CUDA;
        }
      }
    }
    S->max_inflight = max_inflight;
  }
  if (budget > 0) S->budget = budget;
  if (max_blocks >= 0) S->max_blocks = max_blocks;
  S->cv_work.notify_all();
  return FJ_OK;
}

fj_status server_submit(Server* S, Request* r, uint64_t* ticket) {
  r->t_submit = std::chrono::steady_clock::now();
  r->mem_est = estimate_bytes(*r, S->num_sms);
  std::lock_guard<std::mutex> lock(S->mu);
  if ((int64_t)r->mem_est > S->budget) {
    set_error("fj_submit: request needs about %zu bytes, the serving budget is %lld", r->mem_est,
              (long long)S->budget);
    delete r;
    return FJ_ERR_ADMIT;
  }
  r->id = S->next_id++;
  S->all[r->id] = r;
  S->pending.push_back(r);
  *ticket = r->id;
  S->cv_work.notify_all();
  return FJ_OK;
}

fj_status server_poll(Server* S, uint64_t ticket, int32_t timeout_us, fj_quant* out, fj_info* info) {
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    set_error("fj_poll: unknown or already collected ticket %llu", (unsigned long long)ticket);
    return FJ_ERR_TICKET;
  }
  Request* r = it->second;
  if (!r->done && timeout_us != 0) {
    auto pred = [&] { return r->done; };
    if (timeout_us < 0)
      S->cv_done.wait(lock, pred);
    else
      S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred);
  }
  if (!r->done) return FJ_PENDING;
  if (out && !r->quant.empty()) memcpy(out, r->quant.data(), r->quant.size() * sizeof(fj_quant));
  if (info) *info = r->info;
  const fj_status rc = r->rc;
  S->all.erase(it);
  delete r;
  if (rc != FJ_OK) set_error("fj_poll: request finished with status %d", (int)rc);
  return rc;
}

Request* request_new() { return new Request(); }
void request_set_graph(Request* r, const fj_graph* g) { r->graph = g; }
void request_set_edges(Request* r, int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const float* w) {
  r->n = n;
  r->m = m;
  r->src.assign(src, src + m);
  r->dst.assign(dst, dst + m);
  r->weighted = w != nullptr;
  if (w) r->w.assign(w, w + m);
}
void request_set_problem(Request* r, int32_t k, const double* s, int64_t n, const fj_opts& o) {
  r->k = k;
  r->s.assign(s, s + (size_t)n * k);
  r->opts = o;
}
void request_delete(Request* r) { delete r; }

}  // namespace fj
