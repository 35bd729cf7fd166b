// fj_api.cpp - the extern "C" entry points declared in include/fj.h.
//
// A context owns a device, a stream and one grow-only workspace that every
// solve carves its vectors from, so the solve path allocates nothing once the
// workspace has reached the size of the largest problem seen.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "fj_internal.cuh"

// defined in fj_graph.cu, fj_solve.cu and fj_lcc.cu
fj_status fj_lcc_device(const fj_graph* g, cudaStream_t st, fj_graph** out);
fj_status fj_build_graph_device(int device, cudaStream_t st, int64_t n, int64_t m,
                                const int32_t* src, const int32_t* dst, const float* w,
                                bool merge_duplicates, const fj::Layout& lay, fj_graph** out,
                                int32_t* copy_src = nullptr, int32_t* copy_dst = nullptr, float* copy_w = nullptr);
fj_status fj_free_graph_device(fj_graph* g, cudaStream_t st);
fj_status fj_update_weights_device(fj_graph* g, cudaStream_t st, int64_t count, const int32_t* src,
                                   const int32_t* dst, const float* w);
size_t fj_solve_workspace_bytes(const fj_graph* g, int K, int inner_bytes, int num_sms);
fj_status fj_solve_device(const fj_graph* g, cudaStream_t st, int num_sms, int32_t k,
                          const double* s, double* z, double* quant, double* resid, int* status,
                          char* ws, size_t ws_bytes, const fj_opts& o, int* launches_out,
                          int max_blocks, const double* z0, int* grid_out);

namespace fj {
struct Server;
struct Request;
Server* server_create(int device, int num_sms);
void server_destroy(Server* S);
fj_status server_config(Server* S, int32_t max_inflight, int64_t budget, int32_t max_blocks);
fj_status server_pack(Server* S, int64_t max_nodes);
fj_status server_submit(Server* S, Request* r, uint64_t* ticket);
fj_status server_poll(Server* S, uint64_t ticket, int32_t timeout_us, fj_quant* out, fj_info* info);
Request* request_new();
void request_set_graph(Request* r, const fj_graph* g);
void request_set_edges(Request* r, int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const float* w);
void request_set_problem(Request* r, int32_t k, const double* s, int64_t n, const fj_opts& o);
void request_delete(Request* r);
constexpr int kServeMaxK = 1024;

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices];
}  // namespace

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaMallocAsync(p, bytes, st);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      g_pool[dev] = np;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void pool_trim(int device) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (device >= 0 && device < kMaxPoolDevices && g_pool[device]) cudaMemPoolTrimTo(g_pool[device], 0);
}

fj_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FJ_ERR_OOM : FJ_ERR_CUDA;
}

}  // namespace fj

using namespace fj;

struct fj_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;  // solver workspace
  size_t ws_bytes = 0;
  char* small = nullptr;  // quantities, residuals, status words
  size_t small_bytes = 0;
  double* s_dev = nullptr;  // staging of host s / z
  size_t s_bytes = 0;
  double* z_dev = nullptr;
  size_t z_bytes = 0;
  double* z0_dev = nullptr;  // staging of a host initial guess
  size_t z0_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int max_blocks = 0;  // 0: all co-resident blocks
  int grid = 0;        // > 0: exactly this many blocks (fj_set_grid)
  fj::Layout layout;   // layout of later uploads (fj_set_layout)
  std::mutex server_mu;
  fj::Server* server = nullptr;  // created by the first fj_submit / fj_serve_config
};

namespace {

fj_status grow(void** p, size_t* have, size_t need) {
  if (*have >= need) return FJ_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  size_t sz = std::max(need, (size_t)4096);
  cudaError_t e = cudaMalloc(p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("out of device memory (%zu bytes)", sz);
    return FJ_ERR_OOM;
  }
  *have = sz;
  return FJ_OK;
}

// Device address of a page-locked (registered) host array, or null for
// memory a kernel cannot read directly.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

// Grids chosen by fj_tune, per graph: (k, float64 or not) -> grid cap.
struct TunedGrid {
  int32_t k;
  int32_t fp64;
  int32_t blocks;
};
std::mutex g_tuned_mu;
std::unordered_map<const fj_graph*, std::vector<TunedGrid>> g_tuned;

int tuned_grid(const fj_graph* g, int32_t k, bool fp64) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  auto it = g_tuned.find(g);
  if (it == g_tuned.end()) return 0;
  for (const TunedGrid& t : it->second)
    if (t.k == k && t.fp64 == (int32_t)fp64) return t.blocks;
  return 0;
}

void set_tuned_grid(const fj_graph* g, int32_t k, bool fp64, int32_t blocks) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  std::vector<TunedGrid>& v = g_tuned[g];
  for (TunedGrid& t : v)
    if (t.k == k && t.fp64 == (int32_t)fp64) {
      t.blocks = blocks;
      return;
    }
  v.push_back({k, (int32_t)fp64, blocks});
}

void forget_tuned_grids(const fj_graph* g) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  g_tuned.erase(g);
}

// Launch widths for k columns: 32 at a time, then 16, 8, 4, 2, 1.
std::vector<int> decomposition(int64_t k) {
  std::vector<int> Ks;
  for (int64_t col = 0; col < k;) {
    int K = 32;
    while (K > k - col) K >>= 1;
    Ks.push_back(K);
    col += K;
  }
  return Ks;
}

fj_status status_from_bits(int bits) {
  if (bits & kErrTimeout) {
    set_error("a device-side wait timed out (solve abandoned)");
    return FJ_ERR_TIMEOUT;
  }
  if (bits & kErrNumeric) {
    set_error("NaN or Inf met in the iteration");
    return FJ_ERR_NUMERIC;
  }
  if (bits & kErrNotConverged) {
    set_error("iteration caps reached before the residual target");
    return FJ_ERR_NOT_CONVERGED;
  }
  return FJ_OK;
}

}  // namespace

// Context internals for fj_batch.cpp: the device, its SM count and the
// context's stream; and grow-only device scratch (0: solver workspace, 1:
// small outputs, 2: staged s, 3: staged z).
fj_status fj::ctx_device(fj_ctx* c, int* device, int* num_sms, cudaStream_t* st) {
  *device = c->device;
  *num_sms = c->num_sms;
  *st = c->stream;
  return FJ_OK;
}

fj_status fj::ctx_scratch(fj_ctx* c, int which, size_t bytes, char** out) {
  void** p = nullptr;
  size_t* have = nullptr;
  switch (which) {
    case 0: p = (void**)&c->ws; have = &c->ws_bytes; break;
    case 1: p = (void**)&c->small; have = &c->small_bytes; break;
    case 2: p = (void**)&c->s_dev; have = &c->s_bytes; break;
    default: p = (void**)&c->z_dev; have = &c->z_bytes; break;
  }
  fj_status rc = grow(p, have, bytes);
  if (rc != FJ_OK) return rc;
  *out = (char*)*p;
  return FJ_OK;
}

extern "C" {

void fj_default_opts(fj_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->inner_tol = 1e-5;
  o->precision = FJ_PREC_MIXED;
  o->max_iter = 20000;
  o->max_refine = 12;
  o->flags = FJ_HOST_PTRS;
}

const char* fj_last_error(void) { return g_last_error.c_str(); }

int64_t fj_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

const char* fj_version(void) { return "fj-gb300 0.1 (sm_103a)"; }

fj_status fj_create(int device, fj_ctx** out) {
  if (!out) {
    set_error("fj_create: out is NULL");
    return FJ_ERR_ARG;
  }
  *out = nullptr;
  int count = 0;
  FJ_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    set_error("fj_create: device %d not present (%d devices)", device, count);
    return FJ_ERR_ARG;
  }
  FJ_CUDA(cudaSetDevice(device));
  fj_ctx* c = new fj_ctx();
  c->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "fj_create");
  }
  c->stream = c->own;
  *out = c;
  return FJ_OK;
}

fj_status fj_destroy(fj_ctx* c) {
  if (!c) return FJ_OK;
  if (c->server) server_destroy(c->server);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->ws) cudaFree(c->ws);
  if (c->small) cudaFree(c->small);
  if (c->s_dev) cudaFree(c->s_dev);
  if (c->z_dev) cudaFree(c->z_dev);
  if (c->z0_dev) cudaFree(c->z0_dev);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own) cudaStreamDestroy(c->own);
  pool_trim(c->device);
  delete c;
  return FJ_OK;
}

fj_status fj_set_stream(fj_ctx* c, void* stream) {
  if (!c) {
    set_error("fj_set_stream: ctx is NULL");
    return FJ_ERR_ARG;
  }
  c->stream = stream ? (cudaStream_t)stream : c->own;
  return FJ_OK;
}

// Caps the persistent grid (0 = every co-resident block).  Lets several
// contexts share the GPU at once; also used by tests.
fj_status fj_set_max_blocks(fj_ctx* c, int32_t max_blocks) {
  if (!c || max_blocks < 0) {
    set_error("fj_set_max_blocks: bad argument");
    return FJ_ERR_ARG;
  }
  c->max_blocks = max_blocks;
  return FJ_OK;
}

// Runs later solves on exactly `blocks` blocks (0: size the grid by the
// work, or by fj_tune's choice for the graph).
fj_status fj_set_grid(fj_ctx* c, int32_t blocks) {
  if (!c || blocks < 0) {
    set_error("fj_set_grid: bad argument");
    return FJ_ERR_ARG;
  }
  c->grid = blocks;
  return FJ_OK;
}

fj_status fj_graph_upload(fj_ctx* c, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                          const float* w, uint32_t flags, fj_graph** out) {
  if (!c || !out) {
    set_error("fj_graph_upload: ctx or out is NULL");
    return FJ_ERR_ARG;
  }
  *out = nullptr;
  if (n < 1 || n > (int64_t)INT32_MAX - 1 || m < 0 || 2 * m > (int64_t)INT32_MAX - 64) {
    set_error("fj_graph_upload: need 1 <= n < 2^31-1 and 0 <= 2m < 2^31-64 (n=%lld, m=%lld)",
              (long long)n, (long long)m);
    return FJ_ERR_ARG;
  }
  if (m > 0 && (!src || !dst)) {
    set_error("fj_graph_upload: src/dst is NULL");
    return FJ_ERR_ARG;
  }
  if (flags & ~(FJ_DEVICE_PTRS | FJ_MERGE_DUPLICATES)) {
    set_error("fj_graph_upload: unknown flags 0x%x", flags);
    return FJ_ERR_ARG;
  }
  FJ_CUDA(cudaSetDevice(c->device));
  const bool merge = (flags & FJ_MERGE_DUPLICATES) != 0;
  if (flags & FJ_DEVICE_PTRS)
    return fj_build_graph_device(c->device, c->stream, n, m, src, dst, w, merge, c->layout, out);
  // host edge list: copy it to the device first
  int32_t *ds = nullptr, *dd = nullptr;
  float* dw = nullptr;
  const size_t eb = (size_t)std::max<int64_t>(m, 1) * 4;
  if (malloc_async(&ds, eb, c->stream) != cudaSuccess ||
      malloc_async(&dd, eb, c->stream) != cudaSuccess ||
      (w && malloc_async(&dw, eb, c->stream) != cudaSuccess)) {
    cudaGetLastError();
    if (ds) cudaFreeAsync(ds, c->stream);
    if (dd) cudaFreeAsync(dd, c->stream);
    set_error("fj_graph_upload: out of device memory for the edge list");
    return FJ_ERR_OOM;
  }
  fj_status rc = FJ_OK;
  // Page-locked (registered) host arrays are read by the validation pass
  // itself, which writes the device copy on the way; other host memory is
  // copied first.
  const void* ms = mapped_host(src);
  const void* md = mapped_host(dst);
  const void* mw = w ? mapped_host(w) : nullptr;
  if (m > 0 && ms && md && (!w || mw)) {
    rc = fj_build_graph_device(c->device, c->stream, n, m, (const int32_t*)ms, (const int32_t*)md,
                               (const float*)mw, merge, c->layout, out, ds, dd, dw);
  } else {
    if (m > 0) {
      cudaError_t e = cudaMemcpyAsync(ds, src, m * 4, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dst, m * 4, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess && w) e = cudaMemcpyAsync(dw, w, m * 4, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "fj_graph_upload copy");
    }
    if (rc == FJ_OK)
      rc = fj_build_graph_device(c->device, c->stream, n, m, ds, dd, w ? dw : nullptr, merge, c->layout, out);
  }
  cudaFreeAsync(ds, c->stream);
  cudaFreeAsync(dd, c->stream);
  if (dw) cudaFreeAsync(dw, c->stream);
  cudaStreamSynchronize(c->stream);
  return rc;
}

fj_status fj_graph_free(fj_ctx* c, fj_graph* g) {
  if (!c) {
    set_error("fj_graph_free: ctx is NULL");
    return FJ_ERR_ARG;
  }
  if (!g) return FJ_OK;
  forget_tuned_grids(g);
  FJ_CUDA(cudaSetDevice(c->device));
  return fj_free_graph_device(g, c->stream);
}

fj_status fj_set_layout(fj_ctx* c, const fj_layout* l) {
  if (!c) {
    set_error("fj_set_layout: ctx is NULL");
    return FJ_ERR_ARG;
  }
  fj::Layout lay;
  if (l) {
    if (l->chunk_len < 32 || l->chunk_len > 65536 || l->sell_max < 8 || l->sell_max > kSellMaxLenLimit) {
      set_error("fj_set_layout: need 32 <= chunk_len <= 65536 and 8 <= sell_max <= %d", kSellMaxLenLimit);
      return FJ_ERR_ARG;
    }
    lay.chunk_len = l->chunk_len;
    lay.sell_max = l->sell_max;
  }
  c->layout = lay;
  return FJ_OK;
}

fj_status fj_graph_layout(const fj_graph* g, fj_layout* out) {
  if (!g || !out) {
    set_error("fj_graph_layout: graph and out must be non-NULL");
    return FJ_ERR_ARG;
  }
  out->chunk_len = g->chunk_len;
  out->sell_max = g->sell_max;
  return FJ_OK;
}

fj_status fj_graph_update_weights(fj_ctx* c, fj_graph* g, int64_t count, const int32_t* src, const int32_t* dst,
                                  const float* w, uint32_t flags) {
  if (!c || !g || count < 0 || (count > 0 && (!src || !dst || !w)) || (flags & ~FJ_DEVICE_PTRS)) {
    set_error("fj_graph_update_weights: ctx and graph must be non-NULL, count >= 0, src/dst/w non-NULL");
    return FJ_ERR_ARG;
  }
  if (g->device != c->device) {
    set_error("fj_graph_update_weights: graph belongs to device %d, context to %d", g->device, c->device);
    return FJ_ERR_ARG;
  }
  if (count == 0) return FJ_OK;
  FJ_CUDA(cudaSetDevice(c->device));
  if (flags & FJ_DEVICE_PTRS) return fj_update_weights_device(g, c->stream, count, src, dst, w);
  int32_t *ds = nullptr, *dd = nullptr;
  float* dw = nullptr;
  if (malloc_async(&ds, (size_t)count * 4, c->stream) != cudaSuccess ||
      malloc_async(&dd, (size_t)count * 4, c->stream) != cudaSuccess ||
      malloc_async(&dw, (size_t)count * 4, c->stream) != cudaSuccess) {
    cudaGetLastError();
    if (ds) cudaFreeAsync(ds, c->stream);
    if (dd) cudaFreeAsync(dd, c->stream);
    set_error("fj_graph_update_weights: out of device memory");
    return FJ_ERR_OOM;
  }
  fj_status rc = FJ_OK;
  cudaError_t e = cudaMemcpyAsync(ds, src, (size_t)count * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dst, (size_t)count * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w, (size_t)count * 4, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess)
    rc = cuda_fail(e, "fj_graph_update_weights copy");
  else
    rc = fj_update_weights_device(g, c->stream, count, ds, dd, dw);
  cudaFreeAsync(ds, c->stream);
  cudaFreeAsync(dd, c->stream);
  cudaFreeAsync(dw, c->stream);
  cudaStreamSynchronize(c->stream);
  return rc;
}

fj_status fj_graph_lcc(fj_ctx* c, const fj_graph* g, fj_graph** out) {
  if (!c || !g || !out) {
    set_error("fj_graph_lcc: ctx, graph and out must be non-NULL");
    return FJ_ERR_ARG;
  }
  *out = nullptr;
  if (g->device != c->device) {
    set_error("fj_graph_lcc: graph belongs to device %d, context to %d", g->device, c->device);
    return FJ_ERR_ARG;
  }
  FJ_CUDA(cudaSetDevice(c->device));
  return fj_lcc_device(g, c->stream, out);
}

fj_status fj_graph_node_ids(fj_ctx* c, const fj_graph* g, int32_t* ids) {
  if (!c || !g || !ids) {
    set_error("fj_graph_node_ids: ctx, graph and ids must be non-NULL");
    return FJ_ERR_ARG;
  }
  if (!g->orig_ids) {
    for (int64_t i = 0; i < g->n; ++i) ids[i] = (int32_t)i;
    return FJ_OK;
  }
  FJ_CUDA(cudaSetDevice(c->device));
  FJ_CUDA(cudaMemcpyAsync(ids, g->orig_ids, (size_t)g->n * 4, cudaMemcpyDeviceToHost, c->stream));
  FJ_CUDA(cudaStreamSynchronize(c->stream));
  return FJ_OK;
}

fj_status fj_graph_stats(const fj_graph* g, int64_t* n, int64_t* nnz, int32_t* weighted) {
  if (!g) {
    set_error("fj_graph_stats: graph is NULL");
    return FJ_ERR_ARG;
  }
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (weighted) *weighted = g->weighted;
  return FJ_OK;
}

static fj_status solve_impl(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, const double* z0,
                            double* z, fj_quant* quant, const fj_opts* opts, fj_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!c || !g || !s || k < 1) {
    set_error("fj_solve: ctx, graph and s must be non-NULL and k >= 1");
    return FJ_ERR_ARG;
  }
  if (g->device != c->device) {
    set_error("fj_solve: graph belongs to device %d, context to %d", g->device, c->device);
    return FJ_ERR_ARG;
  }
  fj_opts o;
  fj_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.inner_tol >= 1.0 || o.max_iter < 1 ||
      o.max_refine < 1 || o.precision < 0 || o.precision > 2 ||
      (o.flags & ~(FJ_DEVICE_PTRS | FJ_MERGE_DUPLICATES | FJ_TWO_SOLVES | FJ_QUANTITY_TOL))) {
    set_error("fj_solve: invalid options");
    return FJ_ERR_ARG;
  }
  if ((o.flags & FJ_QUANTITY_TOL) && ((o.flags & FJ_TWO_SOLVES) || o.precision == FJ_PREC_FP32)) {
    set_error("fj_solve: FJ_QUANTITY_TOL needs the one-solve form and a refined precision (MIXED or FP64)");
    return FJ_ERR_ARG;
  }
  FJ_CUDA(cudaSetDevice(c->device));
  const int64_t n = g->n;
  // two-solve mode runs 2k launch columns (s_j as is, s_j centred)
  const bool paper = (o.flags & FJ_TWO_SOLVES) != 0;
  const int64_t cols = paper ? 2 * (int64_t)k : k;
  const std::vector<int> Ks = decomposition(cols);
  const int launches = (int)Ks.size();
  const int inner_bytes = o.precision == FJ_PREC_FP64 ? 8 : 4;
  size_t need = 0;
  for (int K : Ks) need = std::max(need, fj_solve_workspace_bytes(g, K, inner_bytes, c->num_sms));
  fj_status rc = grow((void**)&c->ws, &c->ws_bytes, need);
  if (rc != FJ_OK) return rc;
  const size_t small_need = (size_t)cols * 5 * 8 + (size_t)cols * 8 + (size_t)launches * 3 * 4 + 1024;
  rc = grow((void**)&c->small, &c->small_bytes, small_need);
  if (rc != FJ_OK) return rc;
  double* dq = (double*)c->small;
  double* dres = dq + (size_t)cols * 5;
  int* dstat = (int*)(dres + cols);

  const bool host = !(o.flags & FJ_DEVICE_PTRS);
  const double* sd = s;
  double* zd = z;
  const size_t vec_bytes = (size_t)n * k * 8;
  if (host) {
    rc = grow((void**)&c->s_dev, &c->s_bytes, vec_bytes);
    if (rc != FJ_OK) return rc;
    FJ_CUDA(cudaMemcpyAsync(c->s_dev, s, vec_bytes, cudaMemcpyHostToDevice, c->stream));
    sd = c->s_dev;
    if (z0) {
      rc = grow((void**)&c->z0_dev, &c->z0_bytes, vec_bytes);
      if (rc != FJ_OK) return rc;
      FJ_CUDA(cudaMemcpyAsync(c->z0_dev, z0, vec_bytes, cudaMemcpyHostToDevice, c->stream));
      z0 = c->z0_dev;
    }
    if (z) {
      rc = grow((void**)&c->z_dev, &c->z_bytes, vec_bytes);
      if (rc != FJ_OK) return rc;
      zd = c->z_dev;
    }
  }
  FJ_CUDA(cudaMemsetAsync(dstat, 0, (size_t)launches * 3 * 4, c->stream));
  FJ_CUDA(cudaEventRecord(c->ev0, c->stream));
  int done_launches = 0;
  // grid: the context's exact grid, else the one fj_tune chose for this
  // graph and k, else sized by the work; the context's cap bounds all three
  int grid = c->grid > 0 ? c->grid : tuned_grid(g, k, o.precision == FJ_PREC_FP64);
  if (grid > 0 && c->max_blocks > 0) grid = std::min(grid, c->max_blocks);
  const int grid_arg = grid > 0 ? -grid : c->max_blocks;
  int grid_used = 0;
  rc = fj_solve_device(g, c->stream, c->num_sms, k, sd, zd, dq, dres, dstat, c->ws, c->ws_bytes, o,
                       &done_launches, grid_arg, z0, &grid_used);
  if (rc != FJ_OK) return rc;
  FJ_CUDA(cudaEventRecord(c->ev1, c->stream));
  std::vector<double> hq((size_t)cols * 5), hres(cols);
  std::vector<int> hstat((size_t)launches * 3);
  FJ_CUDA(cudaMemcpyAsync(hq.data(), dq, hq.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  FJ_CUDA(cudaMemcpyAsync(hres.data(), dres, hres.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  FJ_CUDA(cudaMemcpyAsync(hstat.data(), dstat, hstat.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  if (host && z) FJ_CUDA(cudaMemcpyAsync(z, zd, vec_bytes, cudaMemcpyDeviceToHost, c->stream));
  FJ_CUDA(cudaStreamSynchronize(c->stream));
  int bits = 0, iters = 0, refines = 0;
  for (int i = 0; i < launches; ++i) {
    bits |= hstat[3 * i];
    iters = std::max(iters, hstat[3 * i + 1]);
    refines = std::max(refines, hstat[3 * i + 2]);
  }
  double worst = 0.0;
  for (int64_t j = 0; j < cols; ++j) worst = std::max(worst, hres[j]);
  if (quant && !paper) memcpy(quant, hq.data(), hq.size() * 8);
  if (quant && paper) {
    // Algorithm 1: C_I = ||L z~||^2 and C = ||z~||^2 from the column solved
    // as is, D = ||W^1/2 B q||^2 and P = ||q||^2 from the centred one
    for (int64_t j = 0; j < k; ++j) {
      const double* a = &hq[(size_t)(2 * j) * 5];
      const double* b = &hq[(size_t)(2 * j + 1) * 5];
      quant[j].C_I = a[0];
      quant[j].D = b[1];
      quant[j].P = b[2];
      quant[j].C = a[3];
      quant[j].I_dc = b[1] + a[3];
    }
  }
  rc = status_from_bits(bits);
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->iterations = iters;
    info->refinements = refines;
    info->rel_residual = worst;
    info->device_ms = ms;
    info->status = rc;
    info->columns = k;
    info->blocks = grid_used;
    info->warnings = (bits & kWarnOpinionRange) ? FJ_WARN_OPINION_RANGE : 0u;
  }
  return rc;
}

fj_status fj_solve_ex(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, double* z,
                      fj_quant* quant, const fj_opts* opts, fj_info* info) {
  return solve_impl(c, g, k, s, nullptr, z, quant, opts, info);
}

fj_status fj_solve_warm(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, const double* z0,
                        double* z, fj_quant* quant, const fj_opts* opts, fj_info* info) {
  if (!z0) {
    if (info) memset(info, 0, sizeof(*info));
    set_error("fj_solve_warm: z0 must be non-NULL");
    return FJ_ERR_ARG;
  }
  return solve_impl(c, g, k, s, z0, z, quant, opts, info);
}

fj_status fj_solve(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, double* z,
                   const fj_opts* opts, fj_info* info) {
  return fj_solve_ex(c, g, k, s, z, nullptr, opts, info);
}

fj_status fj_quantities(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, fj_quant* out,
                        const fj_opts* opts, fj_info* info) {
  if (!out) {
    set_error("fj_quantities: out is NULL");
    return FJ_ERR_ARG;
  }
  return fj_solve_ex(c, g, k, s, nullptr, out, opts, info);
}

fj_status fj_tune(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, const fj_opts* opts,
                  int32_t repeats, fj_tune_result* out) {
  if (!c || !g || !s || !out || k < 1 || repeats < 1 || repeats > 64) {
    set_error("fj_tune: ctx, graph, s and out must be non-NULL, k >= 1, 1 <= repeats <= 64");
    return FJ_ERR_ARG;
  }
  memset(out, 0, sizeof(*out));
  fj_opts o;
  fj_default_opts(&o);
  if (opts) o = *opts;
  if (o.flags & FJ_TWO_SOLVES) {
    set_error("fj_tune: FJ_TWO_SOLVES is not tuned");
    return FJ_ERR_ARG;
  }
  const bool fp64 = o.precision == FJ_PREC_FP64;
  // candidates: the default sizing, then grids of 2*SMs, SMs, SMs/2, ..., 1
  std::vector<int32_t> caps = {0};
  for (int32_t b = 2 * c->num_sms; b >= 1; b /= 2) {
    if ((int)caps.size() == FJ_TUNE_MAX) break;
    caps.push_back(b);
  }
  const int saved_cap = c->max_blocks, saved_grid = c->grid;
  c->max_blocks = 0;
  // grid 0 must mean the default sizing here, not an earlier tuning
  set_tuned_grid(g, k, fp64, 0);
  int32_t best = 0;
  double best_ms = 0.0;
  fj_status rc = FJ_OK;
  for (size_t i = 0; i < caps.size() && rc == FJ_OK; ++i) {
    c->grid = caps[i];
    std::vector<double> ms;
    for (int r = 0; r <= repeats && rc == FJ_OK; ++r) {
      fj_info info;
      rc = solve_impl(c, g, k, s, nullptr, nullptr, nullptr, &o, &info);
      if (r > 0) ms.push_back(info.device_ms);
    }
    if (rc != FJ_OK) break;
    std::sort(ms.begin(), ms.end());
    const double med = ms[ms.size() / 2];
    out->blocks[i] = caps[i];
    out->ms[i] = med;
    out->count = (int32_t)i + 1;
    if (i == 0 || med < best_ms) {
      best = caps[i];
      best_ms = med;
    }
  }
  c->max_blocks = saved_cap;
  c->grid = saved_grid;
  if (rc != FJ_OK) return rc;
  out->best = best;
  set_tuned_grid(g, k, fp64, best);
  return FJ_OK;
}

fj_status fj_tune_layout(fj_ctx* c, int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const float* w,
                         uint32_t upload_flags, int32_t k, const double* s, const fj_opts* opts, int32_t repeats,
                         fj_layout_tune_result* out) {
  if (!c || !s || !out || k < 1 || repeats < 1 || repeats > 64) {
    set_error("fj_tune_layout: ctx, s and out must be non-NULL, k >= 1, 1 <= repeats <= 64");
    return FJ_ERR_ARG;
  }
  memset(out, 0, sizeof(*out));
  fj_opts o;
  fj_default_opts(&o);
  if (opts) o = *opts;
  if (o.flags & FJ_TWO_SOLVES) {
    set_error("fj_tune_layout: FJ_TWO_SOLVES is not tuned");
    return FJ_ERR_ARG;
  }
  // candidates: chunk lengths 256..4096 entries, sliced-ELL rows of up to
  // 32 or 64 entries; the default (512, 64) first
  std::vector<fj::Layout> cand;
  cand.push_back(fj::Layout());
  for (int sm : {64, 32})
    for (int cl : {256, 512, 1024, 2048, 4096}) {
      fj::Layout l;
      l.chunk_len = cl;
      l.sell_max = sm;
      if (!(cl == kChunkLen && sm == kSellMaxLen)) cand.push_back(l);
    }
  const fj::Layout saved = c->layout;
  fj_status rc = FJ_OK;
  double best_ms = 0.0;
  for (size_t i = 0; i < cand.size() && i < FJ_LAYOUT_TUNE_MAX && rc == FJ_OK; ++i) {
    c->layout = cand[i];
    fj_graph* g = nullptr;
    rc = fj_graph_upload(c, n, m, src, dst, w, upload_flags, &g);
    if (rc != FJ_OK) break;
    std::vector<double> ms;
    for (int r = 0; r <= repeats && rc == FJ_OK; ++r) {
      fj_info info;
      rc = fj_solve_ex(c, g, k, s, nullptr, nullptr, &o, &info);
      if (r > 0) ms.push_back(info.device_ms);
    }
    fj_graph_free(c, g);
    if (rc != FJ_OK) break;
    std::sort(ms.begin(), ms.end());
    out->tried[i].chunk_len = cand[i].chunk_len;
    out->tried[i].sell_max = cand[i].sell_max;
    out->ms[i] = ms[ms.size() / 2];
    out->count = (int32_t)i + 1;
    if (i == 0 || out->ms[i] < best_ms) {
      best_ms = out->ms[i];
      out->best = out->tried[i];
    }
  }
  c->layout = saved;
  if (rc != FJ_OK) return rc;
  return fj_set_layout(c, &out->best);
}

// ------------------------------------------------------------- serving

static fj_status get_server(fj_ctx* c, fj::Server** out) {
  std::lock_guard<std::mutex> lock(c->server_mu);
  if (!c->server) {
    c->server = server_create(c->device, c->num_sms);
    if (!c->server) {
      set_error("could not start the serving worker (streams / pinned buffers)");
      return FJ_ERR_CUDA;
    }
  }
  *out = c->server;
  return FJ_OK;
}

static fj_status check_serve_args(int32_t k, const double* s, const fj_opts* opts, fj_opts* o) {
  if (k < 1 || k > kServeMaxK || !s) {
    set_error("fj_submit: need s non-NULL and 1 <= k <= %d (k=%d)", kServeMaxK, (int)k);
    return FJ_ERR_ARG;
  }
  fj_default_opts(o);
  if (opts) *o = *opts;
  if (!(o->tol > 0.0) || !(o->inner_tol > 0.0) || o->inner_tol >= 1.0 || o->max_iter < 1 || o->max_refine < 1 ||
      o->precision < 0 || o->precision > 2 || (o->flags & FJ_TWO_SOLVES) ||
      ((o->flags & FJ_QUANTITY_TOL) && o->precision == FJ_PREC_FP32)) {
    set_error("fj_submit: invalid options (FJ_TWO_SOLVES is for fj_solve_ex; FJ_QUANTITY_TOL needs MIXED or FP64)");
    return FJ_ERR_ARG;
  }
  return FJ_OK;
}

fj_status fj_serve_config(fj_ctx* c, int32_t max_inflight, int64_t mem_budget_bytes,
                          int32_t max_blocks_per_request) {
  if (!c || max_inflight < 0 || max_inflight > 256) {
    set_error("fj_serve_config: bad argument");
    return FJ_ERR_ARG;
  }
  fj::Server* S = nullptr;
  fj_status rc = get_server(c, &S);
  if (rc != FJ_OK) return rc;
  return server_config(S, max_inflight, mem_budget_bytes, max_blocks_per_request);
}

fj_status fj_serve_pack(fj_ctx* c, int64_t max_nodes) {
  if (!c || max_nodes < 0) {
    set_error("fj_serve_pack: bad argument");
    return FJ_ERR_ARG;
  }
  fj::Server* S = nullptr;
  fj_status rc = get_server(c, &S);
  if (rc != FJ_OK) return rc;
  return server_pack(S, max_nodes);
}

fj_status fj_submit(fj_ctx* c, const fj_graph* g, int32_t k, const double* s, const fj_opts* opts,
                    uint64_t* ticket) {
  if (!c || !g || !ticket) {
    set_error("fj_submit: ctx, graph and ticket must be non-NULL");
    return FJ_ERR_ARG;
  }
  if (g->device != c->device) {
    set_error("fj_submit: graph belongs to device %d, context to %d", g->device, c->device);
    return FJ_ERR_ARG;
  }
  fj_opts o;
  fj_status rc = check_serve_args(k, s, opts, &o);
  if (rc != FJ_OK) return rc;
  fj::Server* S = nullptr;
  rc = get_server(c, &S);
  if (rc != FJ_OK) return rc;
  fj::Request* r = request_new();
  request_set_graph(r, g);
  request_set_problem(r, k, s, g->n, o);
  return server_submit(S, r, ticket);
}

fj_status fj_submit_edges(fj_ctx* c, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                          const float* w, int32_t k, const double* s, const fj_opts* opts, uint64_t* ticket) {
  if (!c || !ticket || n < 1 || n > (int64_t)INT32_MAX - 1 || m < 0 || 2 * m > (int64_t)INT32_MAX - 64 ||
      (m > 0 && (!src || !dst))) {
    set_error("fj_submit_edges: bad argument (n=%lld, m=%lld)", (long long)n, (long long)m);
    return FJ_ERR_ARG;
  }
  fj_opts o;
  fj_status rc = check_serve_args(k, s, opts, &o);
  if (rc != FJ_OK) return rc;
  fj::Server* S = nullptr;
  rc = get_server(c, &S);
  if (rc != FJ_OK) return rc;
  fj::Request* r = request_new();
  request_set_edges(r, n, m, src, dst, w);
  request_set_problem(r, k, s, n, o);
  return server_submit(S, r, ticket);
}

fj_status fj_poll(fj_ctx* c, uint64_t ticket, int32_t timeout_us, fj_quant* out, fj_info* info) {
  if (!c) {
    set_error("fj_poll: ctx is NULL");
    return FJ_ERR_ARG;
  }
  fj::Server* S = nullptr;
  fj_status rc = get_server(c, &S);
  if (rc != FJ_OK) return rc;
  return server_poll(S, ticket, timeout_us, out, info);
}

}  // extern "C"
