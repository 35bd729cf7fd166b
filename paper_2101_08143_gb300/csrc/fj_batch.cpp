// fj_batch.cpp - many small problems packed into shared persistent launches.
//
// A solve of K columns on a small graph needs only a few thread blocks, and
// as its own cooperative launch it pays a launch and a whole-device grid for
// every problem.  fj_solve_batch instead cuts every problem into parts of
// 32/16/8/4/2/1 columns (as fj_solve_ex does), and packs parts of equal width
// into one cooperative launch of k_solve_packed: each part runs on its own
// block range with its own barrier, reduction slots, workspace and stopping
// test, so its results are those of a solve of the same part on that many
// blocks alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fj_internal.cuh"

fj_status fj_solve_packed_device(int K, int count, const fj::PackItem* items, cudaStream_t st, const fj_opts& o,
                                 char* bars);
int fj_pack_blocks(const fj_graph* g, int K, int cap);
fj_status fj_pack_capacity(int precision, int K, int num_sms, int* out);
size_t fj_solve_workspace_bytes_blocks(const fj_graph* g, int K, int inner_bytes, int64_t blocks);

namespace fj {

// Launch widths of k columns: 32 at a time, then 16, 8, 4, 2, 1.
static void widths(int64_t k, std::vector<int>& out) {
  out.clear();
  for (int64_t col = 0; col < k;) {
    int K = 32;
    while (K > k - col) K >>= 1;
    out.push_back(K);
    col += K;
  }
}

// Packs the parts (in order) greedily into launches of at most kPackMaxItems
// parts and `capacity` blocks; returns the index ranges [begin, end).
std::vector<std::pair<int, int>> plan_packs(const std::vector<int>& blocks, int capacity) {
  std::vector<std::pair<int, int>> packs;
  int begin = 0, used = 0;
  for (int i = 0; i < (int)blocks.size(); ++i) {
    if (i > begin && (i - begin == FJ_PACK_MAX || used + blocks[i] > capacity)) {
      packs.push_back({begin, i});
      begin = i;
      used = 0;
    }
    used += blocks[i];
  }
  if (begin < (int)blocks.size()) packs.push_back({begin, (int)blocks.size()});
  return packs;
}

}  // namespace fj

using namespace fj;

extern "C" fj_status fj_solve_batch(fj_ctx* c, int32_t count, const fj_graph* const* graphs, const int32_t* k,
                                    const double* const* s, double* const* z, fj_quant* const* quant,
                                    const fj_opts* opts, fj_info* info) {
  if (info && count > 0) memset(info, 0, sizeof(fj_info) * (size_t)count);
  if (!c || count < 1 || count > FJ_BATCH_MAX || !graphs || !k || !s) {
    set_error("fj_solve_batch: ctx, graphs, k and s must be non-NULL and 1 <= count <= %d", FJ_BATCH_MAX);
    return FJ_ERR_ARG;
  }
  fj_opts o;
  fj_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.inner_tol >= 1.0 || o.max_iter < 1 || o.max_refine < 1 ||
      o.precision < 0 || o.precision > 2 || (o.flags & ~(FJ_DEVICE_PTRS | FJ_MERGE_DUPLICATES | FJ_QUANTITY_TOL)) ||
      ((o.flags & FJ_QUANTITY_TOL) && o.precision == FJ_PREC_FP32)) {
    set_error("fj_solve_batch: invalid options (FJ_TWO_SOLVES is for fj_solve_ex; FJ_QUANTITY_TOL needs MIXED or FP64)");
    return FJ_ERR_ARG;
  }
  int device = 0, num_sms = 0;
  cudaStream_t st = nullptr;
  fj_status rc = ctx_device(c, &device, &num_sms, &st);
  if (rc != FJ_OK) return rc;
  for (int i = 0; i < count; ++i) {
    if (!graphs[i] || !s[i] || k[i] < 1 || k[i] > 1024) {
      set_error("fj_solve_batch: problem %d needs a graph, s and 1 <= k <= 1024", i);
      return FJ_ERR_ARG;
    }
    if (graphs[i]->device != device) {
      set_error("fj_solve_batch: problem %d's graph belongs to device %d, the context to %d", i,
                graphs[i]->device, device);
      return FJ_ERR_ARG;
    }
  }
  FJ_CUDA(cudaSetDevice(device));
  const bool host = !(o.flags & FJ_DEVICE_PTRS);
  const int inner = o.precision == FJ_PREC_FP64 ? 8 : 4;

  // parts: (problem, first column, width), grouped by width
  struct Part {
    int prob, col, K, blocks;
    size_t ws;
  };
  std::vector<Part> parts;
  std::vector<int64_t> col0(count + 1, 0), vec0(count + 1, 0);  // column and element offsets
  std::vector<int> ws_k;
  for (int i = 0; i < count; ++i) {
    col0[i + 1] = col0[i] + k[i];
    vec0[i + 1] = vec0[i] + graphs[i]->n * (int64_t)k[i];
  }
  const int64_t cols = col0[count];
  for (int K : {32, 16, 8, 4, 2, 1}) {
    int cap = 0;
    rc = fj_pack_capacity(o.precision, K, num_sms, &cap);
    if (rc != FJ_OK) return rc;
    for (int i = 0; i < count; ++i) {
      widths(k[i], ws_k);
      int col = 0;
      for (int w : ws_k) {
        if (w == K) {
          const int b = fj_pack_blocks(graphs[i], K, cap);
          parts.push_back({i, col, K, b, fj_solve_workspace_bytes_blocks(graphs[i], K, inner, b)});
        }
        col += w;
      }
    }
  }
  // packs: consecutive parts of one width
  struct Pack {
    int begin, end, K;
  };
  std::vector<Pack> packs;
  size_t ws_need = 0;
  for (size_t a = 0; a < parts.size();) {
    size_t b = a;
    while (b < parts.size() && parts[b].K == parts[a].K) ++b;
    int cap = 0;
    rc = fj_pack_capacity(o.precision, parts[a].K, num_sms, &cap);
    if (rc != FJ_OK) return rc;
    std::vector<int> blocks;
    for (size_t j = a; j < b; ++j) blocks.push_back(parts[j].blocks);
    for (const auto& pr : plan_packs(blocks, cap)) {
      packs.push_back({(int)a + pr.first, (int)a + pr.second, parts[a].K});
      size_t sum = 0;
      for (int j = (int)a + pr.first; j < (int)a + pr.second; ++j) sum += (parts[j].ws + 255) & ~size_t(255);
      ws_need = std::max(ws_need, sum);
    }
    a = b;
  }

  // device scratch: small outputs, barriers, staged s and z, workspace
  const size_t q_bytes = ((size_t)cols * 6 * 8 + parts.size() * 12 + 255) & ~size_t(255);
  const size_t bar_bytes = 64 * FJ_PACK_MAX;
  char* small = nullptr;
  rc = ctx_scratch(c, 1, q_bytes + bar_bytes, &small);
  if (rc != FJ_OK) return rc;
  double* dq = (double*)small;
  double* dres = dq + cols * 5;
  int* dstat = (int*)(dres + cols);
  char* bars = small + q_bytes;
  const double* sd_base = nullptr;
  double* zd_base = nullptr;
  const bool want_z = z != nullptr;
  if (host) {
    char* sd = nullptr;
    rc = ctx_scratch(c, 2, (size_t)vec0[count] * 8, &sd);
    if (rc != FJ_OK) return rc;
    for (int i = 0; i < count; ++i)
      FJ_CUDA(cudaMemcpyAsync(sd + vec0[i] * 8, s[i], (size_t)(vec0[i + 1] - vec0[i]) * 8, cudaMemcpyHostToDevice,
                              st));
    sd_base = (const double*)sd;
    if (want_z) {
      char* zd = nullptr;
      rc = ctx_scratch(c, 3, (size_t)vec0[count] * 8, &zd);
      if (rc != FJ_OK) return rc;
      zd_base = (double*)zd;
    }
  }
  char* ws = nullptr;
  rc = ctx_scratch(c, 0, ws_need, &ws);
  if (rc != FJ_OK) return rc;
  FJ_CUDA(cudaMemsetAsync(dstat, 0, parts.size() * 12, st));
  cudaEvent_t e0, e1;
  FJ_CUDA(cudaEventCreate(&e0));
  FJ_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  std::vector<PackItem> items;
  for (const Pack& pk : packs) {
    items.clear();
    size_t off = 0;
    for (int j = pk.begin; j < pk.end; ++j) {
      const Part& pt = parts[j];
      const fj_graph* g = graphs[pt.prob];
      PackItem it;
      it.g = g;
      it.ld = g->n;
      const double* sp = host ? sd_base + vec0[pt.prob] : s[pt.prob];
      it.s = sp + (int64_t)pt.col * g->n;
      double* zp = nullptr;
      if (want_z && z[pt.prob]) zp = host ? zd_base + vec0[pt.prob] : z[pt.prob];
      it.z = zp ? zp + (int64_t)pt.col * g->n : nullptr;
      it.quant = dq + (col0[pt.prob] + pt.col) * 5;
      it.resid = dres + col0[pt.prob] + pt.col;
      it.status = dstat + 3 * j;
      it.ws = ws + off;
      it.ws_bytes = pt.ws;
      it.blocks = pt.blocks;
      it.opts = o;
      off += (pt.ws + 255) & ~size_t(255);
      items.push_back(it);
    }
    rc = fj_solve_packed_device(pk.K, (int)items.size(), items.data(), st, o, bars);
    if (rc != FJ_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
  }
  cudaEventRecord(e1, st);
  std::vector<double> hq((size_t)cols * 6);
  std::vector<int> hstat(parts.size() * 3);
  cudaError_t e = cudaMemcpyAsync(hq.data(), dq, (size_t)cols * 6 * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hstat.data(), dstat, parts.size() * 12, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && host && want_z)
    for (int i = 0; i < count && e == cudaSuccess; ++i)
      if (z[i])
        e = cudaMemcpyAsync(z[i], zd_base + vec0[i], (size_t)(vec0[i + 1] - vec0[i]) * 8, cudaMemcpyDeviceToHost,
                            st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "fj_solve_batch");

  // per problem: status bits, iterations, worst residual, largest part grid
  fj_status first = FJ_OK;
  std::vector<int> bits(count, 0), iters(count, 0), refines(count, 0), blocks(count, 0);
  for (size_t j = 0; j < parts.size(); ++j) {
    const int i = parts[j].prob;
    bits[i] |= hstat[3 * j];
    iters[i] = std::max(iters[i], hstat[3 * j + 1]);
    refines[i] = std::max(refines[i], hstat[3 * j + 2]);
    blocks[i] = std::max(blocks[i], parts[j].blocks);
  }
  const double* hres = hq.data() + cols * 5;
  for (int i = 0; i < count; ++i) {
    if (quant && quant[i]) memcpy(quant[i], hq.data() + col0[i] * 5, (size_t)k[i] * 5 * 8);
    fj_status r = FJ_OK;
    if (bits[i] & kErrTimeout)
      r = FJ_ERR_TIMEOUT;
    else if (bits[i] & kErrNumeric)
      r = FJ_ERR_NUMERIC;
    else if (bits[i] & kErrNotConverged)
      r = FJ_ERR_NOT_CONVERGED;
    if (r != FJ_OK && first == FJ_OK) first = r;
    if (info) {
      double worst = 0.0;
      for (int64_t j = col0[i]; j < col0[i + 1]; ++j) worst = std::max(worst, hres[j]);
      info[i].iterations = iters[i];
      info[i].refinements = refines[i];
      info[i].rel_residual = worst;
      info[i].device_ms = ms;
      info[i].status = r;
      info[i].columns = k[i];
      info[i].blocks = blocks[i];
      info[i].warnings = (bits[i] & kWarnOpinionRange) ? FJ_WARN_OPINION_RANGE : 0u;
    }
  }
  if (first != FJ_OK) set_error("fj_solve_batch: a problem finished with status %d (see its fj_info)", (int)first);
  return first;
}
