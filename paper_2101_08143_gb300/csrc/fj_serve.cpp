// fj_serve.cpp - continuous-batching request server behind fj_submit/fj_poll.
//
// One worker thread per context owns the device side of serving:
//   * submitted requests wait in a queue (inputs already copied);
//   * a request is admitted when an in-flight slot is free and the device
//     memory it needs fits the remaining budget.  Admission goes in arrival
//     order, but a request that does not fit yet is passed over by later
//     requests that do, at most kMaxPassOver times; after that nothing behind
//     it is admitted until it fits, so a large request cannot starve;
//   * an admitted request builds its own graph (if it brought an edge list)
//     on its slot's stream; once the graph is resident the request is ready:
//       - a small graph (at most pack_max_nodes nodes) joins the next batch:
//         the ready small requests are solved together, their parts of equal
//         column count packed into shared persistent launches
//         (fj_solve_packed_device), on one of kBatchStreams batch streams;
//       - a larger graph runs its own persistent solve on its slot's stream;
//   * the worker polls the events of builds, solves and batches and retires
//     requests as they finish, freeing memory and slots at once, so queued
//     requests start while others are still running on the GPU.
// A request's grid (or block range in a batch) depends only on its own size
// and the server's per-request cap, so its results are the same bits alone
// or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fj_internal.cuh"

fj_status fj_build_graph_begin(int device, cudaStream_t st, int64_t n, int64_t m, const int32_t* src,
                               const int32_t* dst, const float* w, bool merge_duplicates, const fj::Layout& lay,
                               int64_t* host_words, fj_graph** pending, int32_t* copy_src = nullptr,
                               int32_t* copy_dst = nullptr, float* copy_w = nullptr);
fj_status fj_build_graph_end(fj_graph* g, const int64_t* host_words, cudaStream_t st, fj_graph** out);
void fj_free_graph_arrays(fj_graph* g, cudaStream_t st);
size_t fj_solve_workspace_bytes(const fj_graph* g, int K, int inner_bytes, int num_sms);
size_t fj_solve_workspace_bytes_blocks(const fj_graph* g, int K, int inner_bytes, int64_t blocks);
fj_status fj_solve_device(const fj_graph* g, cudaStream_t st, int num_sms, int32_t k, const double* s, double* z,
                          double* quant, double* resid, int* status, char* ws, size_t ws_bytes, const fj_opts& o,
                          int* launches_out, int max_blocks, const double* z0, int* grid_out);
fj_status fj_solve_packed_device(int K, int count, const fj::PackItem* items, cudaStream_t st, const fj_opts& o,
                                 char* bars);
int fj_pack_blocks(const fj_graph* g, int K, int cap);
fj_status fj_pack_capacity(int precision, int K, int num_sms, int* out);

namespace fj {

std::vector<std::pair<int, int>> plan_packs(const std::vector<int>& blocks, int capacity);

constexpr int kSlotMaxK = 1024;  // columns per request (pinned result buffers)
constexpr int kBuildWords = 9;   // a graph build's host words (sizes, validation)
// page-locked bytes per slot: quant [k][5] | resid [k] | status words, then
// the build words
constexpr size_t kSlotResultBytes = (size_t)kSlotMaxK * 6 * 8 + 64 * 12;
constexpr size_t kSlotPinnedBytes = kSlotResultBytes + kBuildWords * 8;
// later requests admitted ahead of one that does not fit, at most
constexpr int kMaxPassOver = 32;
constexpr int kBatchStreams = 4;
// requests of one batch, at most
constexpr int kBatchMaxRequests = 64;

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
  int passed = 0;  // later requests admitted while this one did not fit
  // running state
  int slot = -1;
  int block_cap = 0;  // grid cap of the request's solve, fixed at admission
  fj_graph* own_graph = nullptr;
  fj_graph* building = nullptr;  // inline graph whose build is in flight (ev marks its end)
  char* dev = nullptr;  // one device allocation: s | quant | resid | status | workspace
  cudaEvent_t ev = nullptr;        // end of the current stage (build, or own solve)
  cudaEvent_t ev_begin = nullptr;  // admission (start of the request's first GPU work)
  cudaEvent_t ev_end = nullptr;    // completion (own, or the batch's)
  bool in_batch = false;
  int launches = 0;  // status entries (launches, or batch parts)
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

struct Batch {
  cudaStream_t stream = nullptr;
  bool busy = false;
  std::vector<Request*> reqs;
  cudaEvent_t ev = nullptr;
};

struct Server {
  int device = 0;
  int num_sms = 0;
  int max_inflight = 16;
  int64_t budget = 0;
  int max_blocks = 0;  // per-request grid cap (0: automatic, see block_cap)
  // graphs up to this size are batched (0, the default: never; measured on
  // GB300, own launches on the slot streams serve both mixed and small-only
  // streams faster, so packing is the caller's choice)
  int64_t pack_max_nodes = 0;
  int64_t used = 0;
  int admitted = 0;  // requests holding a slot (admitted, not yet retired)
  uint64_t next_id = 1;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::list<Request*> pending;
  std::vector<Request*> inflight;  // building or running on their own
  std::vector<Request*> ready;     // small requests whose graph is resident, not yet batched
  std::unordered_map<uint64_t, Request*> all;
  std::deque<Slot> slots;  // grows in place: references to slots stay valid
  Batch batches[kBatchStreams];
  cudaEvent_t epoch = nullptr;  // device time origin of fj_info.t_begin_ms / t_end_ms
  std::thread worker;

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
    for (auto& b : batches)
      if (b.stream) cudaStreamDestroy(b.stream);
    if (epoch) cudaEventDestroy(epoch);
    for (auto& kv : all) delete kv.second;
  }
};

namespace {

int64_t request_n(const Request& r) { return r.graph ? r.graph->n : r.n; }

size_t estimate_bytes(const Request& r, int num_sms) {
  // inline graph: sort buffers + CSR + sliced ELL, about 80 bytes per entry
  size_t b = 0;
  const int64_t n = request_n(r);
  if (!r.graph) b += (size_t)(2 * r.m + 64) * 80 + (size_t)n * 64;
  const int K = std::min<int>(32, r.k);
  const int inner = r.opts.precision == FJ_PREC_FP64 ? 8 : 4;
  b += (size_t)n * K * (24 + 6 * inner) + (size_t)num_sms * 4 * 16 * K * 16 + (size_t)n * r.k * 8 + (1 << 20);
  return b;
}

// Grid cap of one request's solve: the configured one, else the device's
// co-resident solve blocks (two per SM) shared by the in-flight requests, so
// that they run side by side instead of one at a time; a request of more
// than kLargeRequestNodes nodes may use a quarter of them, since its latency
// grows with its work.  The cap depends only on the request and the
// configuration, never on the load, so a request's results are the same bits
// alone or in a mix.
constexpr int64_t kLargeRequestNodes = int64_t(1) << 17;
int block_cap(const Server& S, const Request& r) {
  if (S.max_blocks > 0) return S.max_blocks;
  const int share = std::max(1, 2 * S.num_sms / std::max(1, S.max_inflight));
  if (request_n(r) > kLargeRequestNodes) return std::max(share, 2 * S.num_sms / 4);
  return share;
}

// Launch widths of k columns: 32 at a time, then 16, 8, 4, 2, 1.
int widths(int k, int* Ks) {
  int count = 0;
  for (int col = 0; col < k;) {
    int K = 32;
    while (K > k - col) K >>= 1;
    Ks[count++] = K;
    col += K;
  }
  return count;
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
// r->ev after the copy of the build's host words; the request becomes ready
// once that event has completed, so the worker thread never waits for a
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
                                      (r->opts.flags & FJ_MERGE_DUPLICATES) != 0, Layout(), build_words(S, r),
                                      &pending);
  cudaFreeAsync(ds, st);
  cudaFreeAsync(dd, st);
  if (dw) cudaFreeAsync(dw, st);
  if (rc != FJ_OK) return rc;
  r->building = pending;
  cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  cudaEventRecord(r->ev, st);
  return FJ_OK;
}

// Ends the build of an inline graph (its event has completed): the graph
// becomes the request's own, and its host edge list is dropped.
fj_status end_build(Server& S, Request* r) {
  fj_graph* og = nullptr;
  fj_graph* g0 = r->building;
  r->building = nullptr;
  cudaEventDestroy(r->ev);
  r->ev = nullptr;
  fj_status rc = fj_build_graph_end(g0, build_words(S, r), S.slots[r->slot].stream, &og);
  if (rc != FJ_OK) return rc;
  r->own_graph = og;
  std::vector<int32_t>().swap(r->src);
  std::vector<int32_t>().swap(r->dst);
  std::vector<float>().swap(r->w);
  return FJ_OK;
}

// Launches the request's own solve on its slot's stream (the graph is
// resident: the caller's, or the request's own).
fj_status start_solve(Server& S, Request* r) {
  Slot& sl = S.slots[r->slot];
  cudaStream_t st = sl.stream;
  cudaSetDevice(S.device);
  const fj_graph* g = r->graph ? r->graph : r->own_graph;
  const int64_t n = g->n;
  int Ks[64];
  const int launches = widths(r->k, Ks);
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
  o.flags = FJ_DEVICE_PTRS | (r->opts.flags & FJ_QUANTITY_TOL);
  fj_status rc = fj_solve_device(g, st, S.num_sms, r->k, ds, nullptr, dq, dres, dstat, r->dev + s_bytes + small,
                                 ws, o, &r->launches, r->block_cap, nullptr, &r->info.blocks);
  if (rc != FJ_OK) return rc;
  cudaMemcpyAsync(sl.pinned, dq, (size_t)r->k * 6 * 8 + (size_t)launches * 12, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(r->dev, st);
  r->dev = nullptr;
  if (r->own_graph) fj_free_graph_arrays(r->own_graph, st);
  cudaEventCreate(&r->ev);
  cudaEventRecord(r->ev, st);
  r->ev_end = r->ev;
  std::vector<double>().swap(r->s);
  return FJ_OK;
}

// Solves the requests of batch B together on its stream: each request's
// parts (launches of 32/16/8/4/2/1 columns), grouped by width, are packed
// into shared persistent launches, each part on its own block range of at
// most the request's grid cap.  Per request, the small outputs keep the
// layout of an own solve (quant | resid | status per part), so collect()
// reads them the same way.
fj_status start_batch(Server& S, Batch& B) {
  cudaStream_t st = B.stream;
  cudaSetDevice(S.device);
  struct Part {
    int req, col, K, blocks;
    size_t ws;
  };
  const int prec = B.reqs[0]->opts.precision;
  std::vector<Part> parts;
  std::vector<size_t> base(B.reqs.size());
  size_t off = 0;
  for (size_t i = 0; i < B.reqs.size(); ++i) {
    Request* r = B.reqs[i];
    const int64_t n = (r->graph ? r->graph : r->own_graph)->n;
    int Ks[64];
    r->launches = widths(r->k, Ks);
    base[i] = off;
    off += ((size_t)n * r->k * 8 + 255) & ~size_t(255);
    off += ((size_t)r->k * 6 * 8 + (size_t)r->launches * 12 + 255) & ~size_t(255);
  }
  const size_t bars_off = off;
  off += 64 * FJ_PACK_MAX;
  // parts by width, then packs
  const int inner = prec == FJ_PREC_FP64 ? 8 : 4;
  size_t ws_need = 0;
  std::vector<std::vector<std::pair<int, int>>> packs_of_width;
  std::vector<int> width_begin;
  for (int K : {32, 16, 8, 4, 2, 1}) {
    int cap = 0;
    fj_status rc = fj_pack_capacity(prec, K, S.num_sms, &cap);
    if (rc != FJ_OK) return rc;
    const int begin = (int)parts.size();
    for (size_t i = 0; i < B.reqs.size(); ++i) {
      Request* r = B.reqs[i];
      const fj_graph* g = r->graph ? r->graph : r->own_graph;
      int Ks[64];
      const int nw = widths(r->k, Ks);
      int col = 0;
      for (int j = 0; j < nw; ++j) {
        if (Ks[j] == K) {
          const int b = fj_pack_blocks(g, K, std::min(cap, r->block_cap));
          parts.push_back({(int)i, col, K, b, fj_solve_workspace_bytes_blocks(g, K, inner, b)});
        }
        col += Ks[j];
      }
    }
    std::vector<int> blocks;
    for (int j = begin; j < (int)parts.size(); ++j) blocks.push_back(parts[j].blocks);
    std::vector<std::pair<int, int>> packs = plan_packs(blocks, cap);
    for (auto& pr : packs) {
      pr.first += begin;
      pr.second += begin;
      size_t sum = 0;
      for (int j = pr.first; j < pr.second; ++j) sum += (parts[j].ws + 255) & ~size_t(255);
      ws_need = std::max(ws_need, sum);
    }
    packs_of_width.push_back(packs);
  }
  const size_t ws_off = off;
  char* dev = nullptr;
  if (malloc_async(&dev, ws_off + ws_need, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("fj_submit: out of device memory for a batch");
    return FJ_ERR_OOM;
  }
  // inputs
  for (size_t i = 0; i < B.reqs.size(); ++i) {
    Request* r = B.reqs[i];
    const int64_t n = (r->graph ? r->graph : r->own_graph)->n;
    cudaMemcpyAsync(dev + base[i], r->s.data(), (size_t)n * r->k * 8, cudaMemcpyHostToDevice, st);
    char* small = dev + base[i] + (((size_t)n * r->k * 8 + 255) & ~size_t(255));
    cudaMemsetAsync(small + (size_t)r->k * 6 * 8, 0, (size_t)r->launches * 12, st);
  }
  // the packed launches; a request's part index counts its widths in the
  // order of its own launches (32, 16, ..., 1), as in an own solve.  The
  // batch's requests share a precision; tolerances and caps are their own.
  fj_opts o = B.reqs[0]->opts;
  o.flags = FJ_DEVICE_PTRS;
  std::vector<PackItem> items;
  for (const auto& packs : packs_of_width) {
    for (const auto& pr : packs) {
      items.clear();
      size_t woff = 0;
      for (int j = pr.first; j < pr.second; ++j) {
        const Part& pt = parts[j];
        Request* r = B.reqs[pt.req];
        const fj_graph* g = r->graph ? r->graph : r->own_graph;
        const int64_t n = g->n;
        char* sbase = dev + base[pt.req];
        double* dq = (double*)(sbase + (((size_t)n * r->k * 8 + 255) & ~size_t(255)));
        int Ks[64];
        const int nw = widths(r->k, Ks);
        int pidx = 0, c = 0;
        for (; pidx < nw && c != pt.col; ++pidx) c += Ks[pidx];
        PackItem it;
        it.g = g;
        it.s = (const double*)sbase + (int64_t)pt.col * n;
        it.ld = n;
        it.z = nullptr;
        it.quant = dq + (size_t)pt.col * 5;
        it.resid = dq + (size_t)r->k * 5 + pt.col;
        it.status = (int*)(dq + (size_t)r->k * 6) + 3 * pidx;
        it.ws = dev + ws_off + woff;
        it.ws_bytes = pt.ws;
        it.blocks = pt.blocks;
        it.opts = r->opts;
        it.opts.flags = FJ_DEVICE_PTRS | (r->opts.flags & FJ_QUANTITY_TOL);
        woff += (pt.ws + 255) & ~size_t(255);
        r->info.blocks = std::max(r->info.blocks, pt.blocks);
        items.push_back(it);
      }
      fj_status rc = fj_solve_packed_device(parts[pr.first].K, (int)items.size(), items.data(), st, o,
                                            dev + bars_off);
      if (rc != FJ_OK) {
        cudaFreeAsync(dev, st);
        return rc;
      }
    }
  }
  // results into each request's pinned slot buffer, then release
  for (size_t i = 0; i < B.reqs.size(); ++i) {
    Request* r = B.reqs[i];
    const int64_t n = (r->graph ? r->graph : r->own_graph)->n;
    char* small = dev + base[i] + (((size_t)n * r->k * 8 + 255) & ~size_t(255));
    cudaMemcpyAsync(S.slots[r->slot].pinned, small, (size_t)r->k * 6 * 8 + (size_t)r->launches * 12,
                    cudaMemcpyDeviceToHost, st);
    if (r->own_graph) fj_free_graph_arrays(r->own_graph, st);
    std::vector<double>().swap(r->s);
  }
  cudaFreeAsync(dev, st);
  cudaEventCreate(&B.ev);
  cudaEventRecord(B.ev, st);
  for (Request* r : B.reqs) r->ev_end = B.ev;
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
  float a = 0.f, b = 0.f;
  if (r->ev_begin && r->ev_end && cudaEventElapsedTime(&a, S.epoch, r->ev_begin) == cudaSuccess &&
      cudaEventElapsedTime(&b, S.epoch, r->ev_end) == cudaSuccess) {
    r->info.t_begin_ms = a;
    r->info.t_end_ms = b;
  }
  cudaGetLastError();
  r->info.batched = r->in_batch ? 1 : 0;
  if (r->own_graph) {
    delete r->own_graph;  // arrays were freed stream-ordered at launch time
    r->own_graph = nullptr;
  }
  if (!r->in_batch && r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  r->ev_end = nullptr;
  if (r->ev_begin) cudaEventDestroy(r->ev_begin);
  r->ev_begin = nullptr;
  finish(S, r, rc);
}

// A request that could not be started (or whose graph was bad): free what
// it holds on its slot's stream, release the slot, complete it with rc.
void abandon(Server& S, Request* r, fj_status rc) {
  cudaStream_t st = S.slots[r->slot].stream;
  S.slots[r->slot].busy = false;
  S.used -= (int64_t)r->mem_est;
  --S.admitted;
  if (r->own_graph) {
    fj_free_graph_arrays(r->own_graph, st);
    delete r->own_graph;
    r->own_graph = nullptr;
  }
  if (r->dev) {
    cudaFreeAsync(r->dev, st);
    r->dev = nullptr;
  }
  if (r->ev && !r->in_batch) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  if (r->ev_begin) cudaEventDestroy(r->ev_begin);
  r->ev_begin = nullptr;
  r->ev_end = nullptr;
  finish(S, r, rc);
  S.cv_done.notify_all();
}

bool small_request(const Server& S, const Request* r) {
  return S.pack_max_nodes > 0 && request_n(*r) <= S.pack_max_nodes;
}

// A request whose graph is resident: small ones wait for the next batch,
// others start their own solve.  Returns an error code if it could not be
// started.
fj_status on_ready(Server& S, Request* r, std::unique_lock<std::mutex>& lock) {
  if (small_request(S, r)) {
    S.ready.push_back(r);
    return FJ_OK;
  }
  lock.unlock();
  const fj_status rc = start_solve(S, r);
  lock.lock();
  if (rc == FJ_OK) S.inflight.push_back(r);
  return rc;
}

void worker_loop(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.device);
  std::unique_lock<std::mutex> lock(S.mu);
  while (true) {
    if (S.stop) break;
    bool progress = false;
    // builds that ended make their request ready; own solves that ended
    // retire (only this thread changes these lists)
    for (size_t i = 0; i < S.inflight.size();) {
      Request* r = S.inflight[i];
      if (cudaEventQuery(r->ev) != cudaSuccess) {
        ++i;
        continue;
      }
      progress = true;
      S.inflight.erase(S.inflight.begin() + i);
      if (r->building) {
        lock.unlock();
        fj_status rc = end_build(S, r);
        lock.lock();
        if (rc == FJ_OK) rc = on_ready(S, r, lock);
        if (rc != FJ_OK) abandon(S, r, rc);
        continue;
      }
      collect(S, r);
      S.slots[r->slot].busy = false;
      S.used -= (int64_t)r->mem_est;
      --S.admitted;
    }
    // batches that ended retire their requests
    for (Batch& B : S.batches) {
      if (!B.busy || cudaEventQuery(B.ev) != cudaSuccess) continue;
      progress = true;
      for (Request* r : B.reqs) {
        collect(S, r);
        S.slots[r->slot].busy = false;
        S.used -= (int64_t)r->mem_est;
        --S.admitted;
      }
      B.reqs.clear();
      cudaEventDestroy(B.ev);
      B.ev = nullptr;
      B.busy = false;
    }
    if (progress) S.cv_done.notify_all();
    // ready small requests go out as a batch on a free batch stream
    // (grouped by precision: one batch holds one precision)
    for (Batch& B : S.batches) {
      if (S.ready.empty()) break;
      if (B.busy) continue;
      const int prec = S.ready.front()->opts.precision;
      for (size_t i = 0; i < S.ready.size() && (int)B.reqs.size() < kBatchMaxRequests;) {
        if (S.ready[i]->opts.precision == prec) {
          B.reqs.push_back(S.ready[i]);
          S.ready.erase(S.ready.begin() + i);
        } else {
          ++i;
        }
      }
      for (Request* r : B.reqs) r->in_batch = true;
      B.busy = true;
      lock.unlock();
      const fj_status rc = start_batch(S, B);
      lock.lock();
      if (rc != FJ_OK) {
        for (Request* r : B.reqs) abandon(S, r, rc);
        B.reqs.clear();
        B.busy = false;
      }
      progress = true;
    }
    // admission: in arrival order; a request that does not fit yet is passed
    // over by later ones at most kMaxPassOver times
    Request* blocked = nullptr;
    for (auto it = S.pending.begin(); it != S.pending.end() && S.admitted < S.max_inflight;) {
      Request* r = *it;
      if (S.used + (int64_t)r->mem_est > S.budget && S.admitted > 0) {
        if (!blocked) blocked = r;
        if (blocked->passed >= kMaxPassOver) break;
        ++it;
        continue;
      }
      if (blocked) {
        if (blocked->passed >= kMaxPassOver) break;
        ++blocked->passed;
      }
      it = S.pending.erase(it);
      int slot = 0;
      while (S.slots[slot].busy) ++slot;
      S.slots[slot].busy = true;
      r->slot = slot;
      r->block_cap = block_cap(S, *r);
      S.used += (int64_t)r->mem_est;
      ++S.admitted;
      r->t_start = std::chrono::steady_clock::now();
      cudaEventCreate(&r->ev_begin);
      cudaEventRecord(r->ev_begin, S.slots[slot].stream);
      fj_status rc = FJ_OK;
      if (r->graph) {
        rc = on_ready(S, r, lock);
      } else {
        lock.unlock();
        rc = start_build(S, r);
        lock.lock();
        if (rc == FJ_OK) S.inflight.push_back(r);
      }
      if (rc != FJ_OK) abandon(S, r, rc);
      progress = true;
    }
    if (!progress) {
      bool busy = !S.inflight.empty() || !S.ready.empty();
      for (auto& B : S.batches) busy |= B.busy;
      if (!busy && S.pending.empty())
        S.cv_work.wait(lock);
      else
        S.cv_work.wait_for(lock, std::chrono::microseconds(20));
    }
  }
  // shutdown: drain what is on the GPU, drop what is queued
  for (Batch& B : S.batches) {
    if (!B.busy) continue;
    cudaStreamSynchronize(B.stream);
    for (Request* r : B.reqs) collect(S, r);
    B.reqs.clear();
    cudaEventDestroy(B.ev);
    B.ev = nullptr;
    B.busy = false;
  }
  for (Request* r : S.ready) {
    if (r->own_graph) {
      fj_free_graph_arrays(r->own_graph, S.slots[r->slot].stream);
      cudaStreamSynchronize(S.slots[r->slot].stream);
      delete r->own_graph;
      r->own_graph = nullptr;
    }
    if (r->ev_begin) cudaEventDestroy(r->ev_begin);
    r->ev_begin = nullptr;
    finish(S, r, FJ_ERR_ARG);
  }
  S.ready.clear();
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
      if (r->ev_begin) cudaEventDestroy(r->ev_begin);
      r->ev_begin = nullptr;
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
  for (auto& B : S->batches) {
    if (cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return nullptr;
    }
  }
  if (cudaEventCreate(&S->epoch) != cudaSuccess || cudaEventRecord(S->epoch, S->slots[0].stream) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return nullptr;
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

fj_status server_pack(Server* S, int64_t max_nodes) {
  std::lock_guard<std::mutex> lock(S->mu);
  S->pack_max_nodes = max_nodes;
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
