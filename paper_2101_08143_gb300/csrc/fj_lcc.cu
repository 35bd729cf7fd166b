// fj_lcc.cu - connected components and the largest connected component.
//
// The paper evaluates its method on the largest connected component of each
// network (Sec. 5, Experiments).  fj_graph_lcc extracts it on the device:
//   1. components by minimum-label hooking with pointer jumping (in the
//      manner of Shiloach and Vishkin, 1982): parent[i] starts at i; a round
//      lets every CSR entry (i, j) whose endpoints have different roots hook
//      the larger root onto the smaller one (atomicMin), then every node
//      jumps to its root.  Rounds repeat until no entry joins two trees.  A
//      component's root is then its smallest solver id, whatever the order of
//      the atomics.
//   2. component sizes and smallest input ids; the largest component wins,
//      ties going to the one holding the smallest input id.
//   3. the induced subgraph: its nodes renumbered in increasing input id, its
//      edges (each once, in CSR order) built like an upload.
// Every device wait is a kernel boundary; the host loops are bounded.
#include <algorithm>
#include <cstring>

#include "fj_internal.cuh"

fj_status fj_build_graph_device(int device, cudaStream_t st, int64_t n, int64_t m, const int32_t* src,
                                const int32_t* dst, const float* w, bool merge_duplicates, const fj::Layout& lay,
                                fj_graph** out, int32_t* copy_src = nullptr, int32_t* copy_dst = nullptr,
                                float* copy_w = nullptr);

namespace fj {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kMaxRounds = 256;   // hooking rounds
constexpr int kJumpSteps = 64;    // pointer steps per node and launch

unsigned grid_of(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

__global__ void k_cc_init(int32_t* __restrict__ parent, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int32_t)i;
}

__device__ __forceinline__ void hook(int32_t* parent, int32_t i, int32_t j, int* joined) {
  const int32_t a = parent[i], b = parent[j];
  if (a != b) {
    const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
    atomicMin(&parent[hi], lo);
    *joined = 1;
  }
}

// One hooking round over every CSR entry: long rows a warp per chunk, short
// rows [n_long, n_nz) a thread per row.  parent[] holds roots on entry.
__global__ void k_cc_hook(const fj_graph g, int32_t* __restrict__ parent, int* __restrict__ joined) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  int any = 0;
  for (int64_t ch = tid >> 5; ch < g.n_chunks; ch += nthreads >> 5) {
    const int32_t r = g.chunk_row[ch];
    for (int32_t p = g.chunk_begin[ch] + lane; p < g.chunk_end[ch]; p += 32) hook(parent, r, g.col[p], &any);
  }
  for (int64_t r = g.n_long + tid; r < g.n_nz; r += nthreads)
    for (int32_t p = g.row_ptr[r]; p < g.row_ptr[r + 1]; ++p) hook(parent, (int32_t)r, g.col[p], &any);
  if (any) *joined = 1;
}

// Every node moves up to kJumpSteps parent links towards its root; *deeper
// is set when a node has not reached it yet.
__global__ void k_cc_jump(int32_t* __restrict__ parent, int64_t n, int* __restrict__ deeper) {
  int more = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = parent[i];
    int s = 0;
    for (; s < kJumpSteps; ++s) {
      const int32_t q = parent[p];
      if (q == p) break;
      p = q;
    }
    if (s == kJumpSteps) more = 1;
    parent[i] = p;
  }
  if (more) *deeper = 1;
}

// Per root: size and smallest input id of its component.  Most nodes share
// one root (the large component), so the lanes of a warp with equal roots
// combine first: one atomic per distinct root and warp.
__global__ void k_cc_sizes(const int32_t* __restrict__ parent, const int32_t* __restrict__ perm, int64_t n,
                           int32_t* __restrict__ size, int32_t* __restrict__ min_in) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = parent[i];
    const unsigned peers = __match_any_sync(__activemask(), r);
    const unsigned lo = __reduce_min_sync(peers, (unsigned)perm[i]);
    if (lane == __ffs(peers) - 1) {
      atomicAdd(&size[r], __popc(peers));
      atomicMin(&min_in[r], (int32_t)lo);
    }
  }
}

// best = max over roots of (size, -smallest input id), packed in 64 bits.
__global__ void k_cc_best(const int32_t* __restrict__ parent, const int32_t* __restrict__ size,
                          const int32_t* __restrict__ min_in, int64_t n, unsigned long long* __restrict__ best) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (parent[i] != (int32_t)i) continue;  // roots only
    const unsigned long long key =
        ((unsigned long long)(uint32_t)size[i] << 32) | (unsigned long long)(0xffffffffu - (uint32_t)min_in[i]);
    atomicMax(best, key);
  }
}

// keep[input id] = 1 for the nodes of the chosen component, the one whose
// smallest input id is the winner's; *root = its root (every node of it
// stores the same value).
__global__ void k_cc_mark(const int32_t* __restrict__ parent, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ min_in, int64_t n, const unsigned long long* __restrict__ best,
                          int32_t* __restrict__ keep, int32_t* __restrict__ root) {
  const uint32_t want = 0xffffffffu - (uint32_t)(*best & 0xffffffffull);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool in = (uint32_t)min_in[parent[i]] == want;
    keep[perm[i]] = in ? 1 : 0;
    if (in) *root = parent[i];
  }
}

// Block-level exclusive scan of keep[] into new ids (kept nodes only), in
// tiles of 1024 with the tile totals added by a second pass: new_id[x] for
// kept input ids x, and ids_out[new id] = x.
constexpr int kTile = 1024;

__global__ void k_tile_count(const int32_t* __restrict__ keep, int64_t n, int32_t* __restrict__ tile_sum) {
  const int64_t x = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const int v = x < n ? keep[x] : 0;
  const int c = __syncthreads_count(v);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = c;
}

__global__ void k_tile_number(const int32_t* __restrict__ keep, int64_t n, const int32_t* __restrict__ tile_sum,
                              int32_t* __restrict__ new_id, int32_t* __restrict__ ids_out) {
  __shared__ int32_t warp_sum[kTile / 32];
  __shared__ int32_t base_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 32) {  // tiles before this one, in a fixed order
    int32_t b = 0;
    for (int64_t t = lane; t < (int64_t)blockIdx.x; t += 32) b += tile_sum[t];
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(kFullMask, b, d);
    if (lane == 0) base_sh = b;
  }
  const int64_t x = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const int v = x < n ? keep[x] : 0;
  const unsigned bal = __ballot_sync(kFullMask, v);
  if (lane == 0) warp_sum[warp] = __popc(bal);
  __syncthreads();
  int32_t before = base_sh;
  for (int w = 0; w < warp; ++w) before += warp_sum[w];
  before += __popc(bal & ((1u << lane) - 1u));
  if (x < n) {
    new_id[x] = v ? before : -1;
    if (v) ids_out[before] = (int32_t)x;
  }
}

// Edge list of the component: every CSR entry (i, j) with i < j of a kept
// node, in CSR order.  The units are the chunks of the long rows (a warp
// each), then the short rows [n_long, n) (a thread each): pass 1 counts per
// unit, pass 2 writes at the unit's scanned offset.
__device__ __forceinline__ bool take(const int32_t* parent, int32_t root, int32_t i, int32_t j) {
  return j > i && parent[i] == root;
}

__global__ void k_lcc_count(const fj_graph g, const int32_t* __restrict__ parent, int32_t root,
                            int64_t* __restrict__ unit_cnt) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t ch = tid >> 5; ch < g.n_chunks; ch += nthreads >> 5) {
    const int32_t r = g.chunk_row[ch], e = g.chunk_end[ch];
    int64_t c = 0;
    for (int32_t p0 = g.chunk_begin[ch]; p0 < e; p0 += 32) {
      const int32_t p = p0 + lane;
      const bool t = p < e && take(parent, root, r, g.col[p]);
      c += __popc(__ballot_sync(kFullMask, t));
    }
    if (lane == 0) unit_cnt[ch] = c;
  }
  for (int64_t r = g.n_long + tid; r < g.n; r += nthreads) {
    int64_t c = 0;
    if (r < g.n_nz)
      for (int32_t p = g.row_ptr[r]; p < g.row_ptr[r + 1]; ++p) c += take(parent, root, (int32_t)r, g.col[p]);
    unit_cnt[g.n_chunks + r - g.n_long] = c;
  }
}

__global__ void k_lcc_write(const fj_graph g, const int32_t* __restrict__ parent, int32_t root,
                            const int64_t* __restrict__ unit_off, const int32_t* __restrict__ new_id,
                            int32_t* __restrict__ src, int32_t* __restrict__ dst, float* __restrict__ w) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t ch = tid >> 5; ch < g.n_chunks; ch += nthreads >> 5) {
    const int32_t r = g.chunk_row[ch], e = g.chunk_end[ch];
    int64_t o = unit_off[ch];
    const int32_t a = new_id[g.perm[r]];
    for (int32_t p0 = g.chunk_begin[ch]; p0 < e; p0 += 32) {
      const int32_t p = p0 + lane;
      const bool t = p < e && take(parent, root, r, g.col[p]);
      const unsigned bal = __ballot_sync(kFullMask, t);
      if (t) {
        const int64_t q = o + __popc(bal & ((1u << lane) - 1u));
        src[q] = a;
        dst[q] = new_id[g.perm[g.col[p]]];
        if (w) w[q] = g.val[p];
      }
      o += __popc(bal);
    }
  }
  for (int64_t r = g.n_long + tid; r < g.n_nz; r += nthreads) {
    int64_t o = unit_off[g.n_chunks + r - g.n_long];
    const int32_t a = new_id[g.perm[r]];
    for (int32_t p = g.row_ptr[r]; p < g.row_ptr[r + 1]; ++p) {
      const int32_t j = g.col[p];
      if (take(parent, root, (int32_t)r, j)) {
        src[o] = a;
        dst[o] = new_id[g.perm[j]];
        if (w) w[o] = g.val[p];
        ++o;
      }
    }
  }
}

// Sequential exclusive scan of row counts in tiles (host loop-free): tile
// sums, then each tile adds its predecessors' sums.
__global__ void k_row_tiles(const int64_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ tile_sum) {
  __shared__ int64_t part[32];
  int64_t v = 0;
  const int64_t x = (int64_t)blockIdx.x * kTile + threadIdx.x;
  if (x < n) v = cnt[x];
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFullMask, v, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t s = part[threadIdx.x];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFullMask, s, d);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
  }
}

__global__ void k_row_offsets(const int64_t* __restrict__ cnt, int64_t n, const int64_t* __restrict__ tile_sum,
                              int64_t* __restrict__ off, int64_t* __restrict__ total) {
  __shared__ int64_t warp_sum[kTile / 32];
  __shared__ int64_t base_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 32) {
    int64_t b = 0;
    for (int64_t t = lane; t < (int64_t)blockIdx.x; t += 32) b += tile_sum[t];
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(kFullMask, b, d);
    if (lane == 0) base_sh = b;
  }
  const int64_t x = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const int64_t v = x < n ? cnt[x] : 0;
  int64_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(kFullMask, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  int64_t before = base_sh;
  for (int w = 0; w < warp; ++w) before += warp_sum[w];
  if (x < n) off[x] = before + incl - v;
  if (x == n - 1) *total = before + incl;
}

}  // namespace
}  // namespace fj

using namespace fj;

// Called by the C ABI.  On success *out owns a new graph whose orig_ids map
// its nodes to input ids of g.
fj_status fj_lcc_device(const fj_graph* g, cudaStream_t st, fj_graph** out) {
  const int64_t n = g->n;
  int32_t *parent = nullptr, *size = nullptr, *min_in = nullptr, *keep = nullptr, *new_id = nullptr,
          *ids = nullptr, *tile32 = nullptr;
  int* flags = nullptr;  // [0] joined, [1] deeper, [2] root of the chosen component
  unsigned long long* best = nullptr;
  int64_t *row_cnt = nullptr, *row_off = nullptr, *tile64 = nullptr, *total = nullptr;
  int32_t *src = nullptr, *dst = nullptr;
  float* w = nullptr;
  const int64_t tiles = (n + kTile - 1) / kTile;
  fj_status rc = FJ_OK;
  auto cleanup = [&]() {
    void* ptrs[] = {parent, size, min_in, keep, new_id, tile32, flags, best, row_cnt, row_off, tile64, total,
                    src, dst, w};
    for (void* p : ptrs)
      if (p) cudaFreeAsync(p, st);
  };
  if (malloc_async(&parent, n * 4, st) != cudaSuccess || malloc_async(&size, n * 4, st) != cudaSuccess ||
      malloc_async(&min_in, n * 4, st) != cudaSuccess || malloc_async(&keep, n * 4, st) != cudaSuccess ||
      malloc_async(&new_id, n * 4, st) != cudaSuccess || malloc_async(&ids, n * 4, st) != cudaSuccess ||
      malloc_async(&tile32, tiles * 4, st) != cudaSuccess || malloc_async(&flags, 16, st) != cudaSuccess ||
      malloc_async(&best, 8, st) != cudaSuccess || malloc_async(&row_cnt, (n + g->n_chunks) * 8, st) != cudaSuccess ||
      malloc_async(&row_off, (n + g->n_chunks) * 8, st) != cudaSuccess ||
      malloc_async(&tile64, (tiles + g->n_chunks / kTile + 1) * 8, st) != cudaSuccess ||
      malloc_async(&total, 8, st) != cudaSuccess) {
    cudaGetLastError();
    if (ids) cudaFreeAsync(ids, st);
    cleanup();
    set_error("fj_graph_lcc: out of device memory");
    return FJ_ERR_OOM;
  }
  auto fail = [&](fj_status code) {
    cudaFreeAsync(ids, st);
    cleanup();
    return code;
  };
  // ---- 1. components
  count_launches(1);
  k_cc_init<<<grid_of(n, 256), 256, 0, st>>>(parent, n);
  int hf[2] = {0, 0};
  int round = 0;
  for (; round < kMaxRounds; ++round) {
    FJ_CUDA(cudaMemsetAsync(flags, 0, 8, st));
    count_launches(1);
    k_cc_hook<<<grid_of(std::max<int64_t>(g->n_chunks * 32, n), 256), 256, 0, st>>>(*g, parent, flags);
    for (int jumps = 0; jumps < kMaxRounds; ++jumps) {
      FJ_CUDA(cudaMemsetAsync(flags + 1, 0, 4, st));
      count_launches(1);
      k_cc_jump<<<grid_of(n, 256), 256, 0, st>>>(parent, n, flags + 1);
      FJ_CUDA(cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, st));
      FJ_CUDA(cudaStreamSynchronize(st));
      if (!hf[1]) break;
    }
    if (hf[1]) break;  // pointer chains that would not end: reported below
    if (!hf[0]) break;
  }
  if (round == kMaxRounds || hf[1]) {
    set_error("fj_graph_lcc: connected components did not settle");
    return fail(FJ_ERR_NOT_CONVERGED);
  }
  // ---- 2. the largest component
  FJ_CUDA(cudaMemsetAsync(size, 0, n * 4, st));
  FJ_CUDA(cudaMemsetAsync(min_in, 0x7f, n * 4, st));
  FJ_CUDA(cudaMemsetAsync(best, 0, 8, st));
  count_launches(3);
  k_cc_sizes<<<grid_of(n, 256), 256, 0, st>>>(parent, g->perm, n, size, min_in);
  k_cc_best<<<grid_of(n, 256), 256, 0, st>>>(parent, size, min_in, n, best);
  k_cc_mark<<<grid_of(n, 256), 256, 0, st>>>(parent, g->perm, min_in, n, best, keep, flags + 2);
  // ---- 3. nodes in increasing input id, the component's root, its edges
  count_launches(2);
  k_tile_count<<<(unsigned)tiles, kTile, 0, st>>>(keep, n, tile32);
  k_tile_number<<<(unsigned)tiles, kTile, 0, st>>>(keep, n, tile32, new_id, ids);
  unsigned long long hbest = 0;
  int32_t root = 0;
  FJ_CUDA(cudaMemcpyAsync(&hbest, best, 8, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaMemcpyAsync(&root, flags + 2, 4, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaStreamSynchronize(st));
  const int64_t n_lcc = (int64_t)(hbest >> 32);
  const int64_t units = g->n_chunks + (n - g->n_long);
  const int64_t utiles = (units + kTile - 1) / kTile;
  count_launches(3);
  k_lcc_count<<<grid_of(std::max<int64_t>(g->n_chunks * 32, n), 256), 256, 0, st>>>(*g, parent, root, row_cnt);
  k_row_tiles<<<(unsigned)utiles, kTile, 0, st>>>(row_cnt, units, tile64);
  k_row_offsets<<<(unsigned)utiles, kTile, 0, st>>>(row_cnt, units, tile64, row_off, total);
  int64_t m_lcc = 0;
  FJ_CUDA(cudaMemcpyAsync(&m_lcc, total, 8, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaStreamSynchronize(st));
  const size_t eb = (size_t)std::max<int64_t>(m_lcc, 1) * 4;
  if (malloc_async(&src, eb, st) != cudaSuccess || malloc_async(&dst, eb, st) != cudaSuccess ||
      (g->weighted && malloc_async(&w, eb, st) != cudaSuccess)) {
    cudaGetLastError();
    set_error("fj_graph_lcc: out of device memory");
    return fail(FJ_ERR_OOM);
  }
  count_launches(1);
  k_lcc_write<<<grid_of(std::max<int64_t>(g->n_chunks * 32, n), 256), 256, 0, st>>>(*g, parent, root, row_off,
                                                                                    new_id, src, dst, w);
  if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);
  // ---- 4. build it like an upload (the pairs are distinct unless g merged
  // repeated pairs, whose parallel entries are kept as such)
  fj_graph* lg = nullptr;
  fj::Layout lay;
  lay.chunk_len = g->chunk_len;
  lay.sell_max = g->sell_max;
  rc = fj_build_graph_device(g->device, st, std::max<int64_t>(n_lcc, 1), m_lcc, src, dst, w, true, lay, &lg);
  if (rc != FJ_OK) return fail(rc);
  lg->orig_ids = ids;
  cleanup();
  FJ_CUDA(cudaStreamSynchronize(st));
  *out = lg;
  return FJ_OK;
}
