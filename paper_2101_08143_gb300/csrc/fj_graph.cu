// fj_graph.cu - device construction of the CSR of I + L (Sec. 2.1).
//
// Input: an undirected edge list (src, dst, w), each edge once.  Every edge
// e = (u, v) yields two directed entries, (row u, col v) and (row v, col u),
// numbered 2e and 2e+1.  A stable LSD radix sort of the 2m entries by row
// id gives the CSR directly; inside a row, entries keep their input order,
// so the CSR (and every sum over it) is the same bits on every upload.
// Self-loops get the key n and sort past the last row, i.e. they are
// dropped (b_e = e_i - e_i = 0 contributes nothing to L).
//
// Then: row_ptr from the sorted keys, weighted degrees d_i by a merge-path
// walk (balanced over hubs), dinv = 1 / (1 + d_i), and the merge-path tile
// plan (row coordinate of every tile start) used by all later walks.
#include <algorithm>
#include <vector>

#include "fj_internal.cuh"
#include "fj_walk.cuh"

namespace fj {

constexpr int kSortThreads = 512;
constexpr int kSortItems = 16;  // items per thread per block chunk
constexpr int kSortChunk = kSortThreads * kSortItems;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

// ------------------------------------------------------------ validation

__global__ void k_validate(int64_t m, int64_t n, const int32_t* __restrict__ src,
                           const int32_t* __restrict__ dst, const float* __restrict__ w,
                           int* __restrict__ err, unsigned long long* __restrict__ first_bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    int bad = 0;
    if (u < 0 || u >= n || v < 0 || v >= n) bad |= kErrBadId;
    if (w) {
      const float x = w[e];
      if (!(x > 0.0f) || isinf(x)) bad |= kErrBadWeight;
    }
    if (bad) {
      atomicOr(err, bad);
      atomicMin(first_bad, (unsigned long long)e);
    }
  }
}

// ------------------------------------------------------------- radix sort

// One directed entry: key = row id (n for a self-loop), col, weight.
struct EntrySrc {
  const int32_t* src;  // edge list (first pass) ...
  const int32_t* dst;
  const float* w;
  const int32_t* key;  // ... or sorted arrays (later passes)
  const int32_t* col;
  const float* val;
  int32_t n;
};

template <bool FROM_EDGES>
__device__ __forceinline__ void load_entry(const EntrySrc& s, int64_t p, int32_t& key,
                                           int32_t& col, float& val) {
  if (FROM_EDGES) {
    const int64_t e = p >> 1;
    const int32_t u = s.src[e], v = s.dst[e];
    const bool side = p & 1;
    key = side ? v : u;
    col = side ? u : v;
    if (u == v) key = s.n;
    val = s.w ? s.w[e] : 1.0f;
  } else {
    key = s.key[p];
    col = s.col[p];
    val = s.val ? s.val[p] : 1.0f;
  }
}

template <bool FROM_EDGES>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(EntrySrc s, int64_t N, int shift,
                                                             int32_t* __restrict__ hist) {
  __shared__ int h[256];
  for (int i = threadIdx.x; i < 256; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  for (int i = threadIdx.x; i < kSortChunk; i += kSortThreads) {
    const int64_t p = base + i;
    if (p < N) {
      int32_t key, col;
      float val;
      load_entry<FROM_EDGES>(s, p, key, col, val);
      atomicAdd(&h[(key >> shift) & 255], 1);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += kSortThreads) hist[(int64_t)i * gridDim.x + blockIdx.x] = h[i];
}

// Stable scatter: inside a block, items are ranked in input order (rounds of
// kSortThreads items; within a round by warp, then by lane).
template <bool FROM_EDGES>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(EntrySrc s, int64_t N, int shift,
                                                                const int32_t* __restrict__ offs,
                                                                int32_t* __restrict__ okey,
                                                                int32_t* __restrict__ ocol,
                                                                float* __restrict__ oval) {
  constexpr int kW = kSortThreads / 32;
  __shared__ int base[256];
  __shared__ int tot[256];
  __shared__ int wcnt[kW][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 256; i += kSortThreads) base[i] = offs[(int64_t)i * gridDim.x + blockIdx.x];
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t cbase = (int64_t)blockIdx.x * kSortChunk;
  for (int r0 = 0; r0 < kSortChunk; r0 += kSortThreads) {
    const int64_t p = cbase + r0 + tid;
    const bool valid = p < N;
    int32_t key = 0, col = 0;
    float val = 0.f;
    if (valid) load_entry<FROM_EDGES>(s, p, key, col, val);
    const int digit = valid ? ((key >> shift) & 255) : 256;
    for (int j = lane; j < 256; j += 32) wcnt[warp][j] = 0;
    __syncwarp();
    const unsigned peers = __match_any_sync(kFull, digit);
    const int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (tid < 256) {
      int run = 0;
#pragma unroll
      for (int w = 0; w < kW; ++w) {
        const int c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      tot[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const int pos = base[digit] + wcnt[warp][digit] + rank;
      okey[pos] = key;
      ocol[pos] = col;
      if (oval) oval[pos] = val;
    }
    __syncthreads();
    if (tid < 256) base[tid] += tot[tid];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ scan

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  // sh: kScanThreads/32 ints
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(kFull, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = (lane < kScanThreads / 32) ? sh[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(kFull, s, off);
      if (lane >= off) s += y;
    }
    if (lane < kScanThreads / 32) sh[lane] = s;
  }
  __syncthreads();
  total = sh[kScanThreads / 32 - 1];
  const int before = warp > 0 ? sh[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t cnt,
                                                              int32_t* __restrict__ sums) {
  __shared__ int sh[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  int v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
    if (p < cnt) v += in[p];
  }
  int total;
  block_exclusive_scan(v, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int32_t* __restrict__ data, int64_t cnt,
                                                             const int32_t* __restrict__ offs) {
  __shared__ int sh[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    vals[i] = (base + i < cnt) ? data[base + i] : 0;
    v += vals[i];
  }
  int total;
  int run = block_exclusive_scan(v, sh, total) + (offs ? offs[blockIdx.x] : 0);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < cnt) data[base + i] = run;
    run += vals[i];
  }
}

// In-place exclusive scan of cnt int32 values (the total must fit int32).
static fj_status exclusive_scan(int32_t* data, int64_t cnt, cudaStream_t st) {
  if (cnt <= 0) return FJ_OK;
  const int64_t blocks = (cnt + kScanChunk - 1) / kScanChunk;
  if (blocks == 1) {
    k_scan_apply<<<1, kScanThreads, 0, st>>>(data, cnt, nullptr);
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
  }
  int32_t* sums = nullptr;
  FJ_CUDA(cudaMallocAsync(&sums, blocks * sizeof(int32_t), st));
  k_scan_reduce<<<(unsigned)blocks, kScanThreads, 0, st>>>(data, cnt, sums);
  fj_status rc = exclusive_scan(sums, blocks, st);
  if (rc == FJ_OK) {
    k_scan_apply<<<(unsigned)blocks, kScanThreads, 0, st>>>(data, cnt, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "k_scan_apply");
  }
  cudaFreeAsync(sums, st);
  return rc;
}

// ------------------------------------------------------------ CSR pieces

// row_ptr[r] = first sorted position whose key >= r, for r in [0, n].
__global__ void k_row_ptr(const int32_t* __restrict__ key, int64_t N, int64_t n,
                          int32_t* __restrict__ row_ptr) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kp = (p < N) ? key[p] : n;
    const int64_t kprev = (p > 0) ? key[p - 1] : -1;
    const int64_t hi = kp < n ? kp : n;
    for (int64_t r = kprev + 1; r <= hi; ++r) row_ptr[r] = (int32_t)p;
  }
}

__global__ void k_tile_rows(const int32_t* __restrict__ row_ptr, int64_t n, int64_t nnz,
                            int64_t n_tiles, int32_t* __restrict__ tile_row) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= n_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = t * kTileItems;
    if (d > n + nnz) d = n + nnz;
    tile_row[t] = (int32_t)merge_path_row(row_ptr, n, d);
  }
}

__global__ void k_dinv_unit(const int32_t* __restrict__ row_ptr, int64_t n, float* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)(row_ptr[i + 1] - row_ptr[i]);
    dinv[i] = (float)(1.0 / (1.0 + d));
  }
}

constexpr int kWalkWarps = 8;

__global__ void __launch_bounds__(kWalkWarps * 32) k_row_sums(WalkGraph g, double* __restrict__ out,
                                                              int32_t* __restrict__ wc_row,
                                                              double* __restrict__ wc_val) {
  __shared__ TileSmem sm[kWalkWarps];
  const int warp = threadIdx.x >> 5;
  const int64_t wg = (int64_t)blockIdx.x * kWalkWarps + warp;
  walk_tiles<double, 1, kRowSum>(g, nullptr, out, wc_row, wc_val, wg, &sm[warp]);
}

__global__ void k_dinv_weighted(WalkGraph g, const double* __restrict__ sums,
                                const double* __restrict__ wc_val, float* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = row_total<double, 1>(i, sums[i], g.row_ptr, wc_val, g.tiles_per_warp, 0);
    dinv[i] = (float)(1.0 / (1.0 + d));
  }
}

static unsigned grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace fj

using namespace fj;

namespace {

struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace

// Called by the C ABI (fj_api.cpp).  src/dst/w are device pointers.
fj_status fj_build_graph_device(int device, cudaStream_t st, int64_t n, int64_t m,
                                const int32_t* src, const int32_t* dst, const float* w,
                                fj_graph** out) {
  const int64_t N = 2 * m;
  // validation
  DevBuf dflags;
  dflags.st = st;
  FJ_CUDA(cudaMallocAsync(&dflags.p, 16, st));
  int* err = (int*)dflags.p;
  unsigned long long* first_bad = (unsigned long long*)((char*)dflags.p + 8);
  FJ_CUDA(cudaMemsetAsync(err, 0, 4, st));
  FJ_CUDA(cudaMemsetAsync(first_bad, 0xff, 8, st));
  if (m > 0) {
    k_validate<<<grid_for(m, 256), 256, 0, st>>>(m, n, src, dst, w, err, first_bad);
    FJ_CUDA(cudaGetLastError());
  }
  int herr = 0;
  unsigned long long hbad = 0;
  FJ_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaMemcpyAsync(&hbad, first_bad, 8, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error("fj_graph_upload: edge %llu has %s", hbad,
              (herr & kErrBadId) ? "a node id outside [0, n)" : "a weight that is not finite and > 0");
    return FJ_ERR_GRAPH;
  }

  const bool weighted = (w != nullptr);
  // ping-pong entry buffers, padded so that tile staging never reads past
  const int64_t cap = N + kPad;
  DevBuf kb[2], cb[2], vb[2];
  for (int i = 0; i < 2; ++i) {
    kb[i].st = cb[i].st = vb[i].st = st;
    if (cudaMallocAsync(&kb[i].p, cap * 4, st) != cudaSuccess ||
        cudaMallocAsync(&cb[i].p, cap * 4, st) != cudaSuccess ||
        (weighted && cudaMallocAsync(&vb[i].p, cap * 4, st) != cudaSuccess)) {
      cudaGetLastError();
      set_error("fj_graph_upload: out of device memory for %lld entries", (long long)N);
      return FJ_ERR_OOM;
    }
  }
  int bits = 1;
  while ((int64_t(1) << bits) <= n) ++bits;  // keys are in [0, n]
  const int passes = (bits + 7) / 8;
  const int64_t nblocks = (N + kSortChunk - 1) / kSortChunk;
  int cur = 0;
  if (N > 0) {
    DevBuf hist;
    hist.st = st;
    FJ_CUDA(cudaMallocAsync(&hist.p, 256 * nblocks * sizeof(int32_t), st));
    for (int pass = 0; pass < passes; ++pass) {
      EntrySrc s{src, dst, w, (int32_t*)kb[cur].p, (int32_t*)cb[cur].p, (float*)vb[cur].p, (int32_t)n};
      const int dstb = pass == 0 ? 0 : 1 - cur;
      int32_t* h = (int32_t*)hist.p;
      if (pass == 0) {
        k_radix_hist<true><<<(unsigned)nblocks, kSortThreads, 0, st>>>(s, N, 0, h);
      } else {
        k_radix_hist<false><<<(unsigned)nblocks, kSortThreads, 0, st>>>(s, N, pass * 8, h);
      }
      FJ_CUDA(cudaGetLastError());
      fj_status rc = exclusive_scan(h, 256 * nblocks, st);
      if (rc != FJ_OK) return rc;
      if (pass == 0) {
        k_radix_scatter<true><<<(unsigned)nblocks, kSortThreads, 0, st>>>(
            s, N, 0, h, (int32_t*)kb[dstb].p, (int32_t*)cb[dstb].p, (float*)vb[dstb].p);
      } else {
        k_radix_scatter<false><<<(unsigned)nblocks, kSortThreads, 0, st>>>(
            s, N, pass * 8, h, (int32_t*)kb[dstb].p, (int32_t*)cb[dstb].p, (float*)vb[dstb].p);
      }
      FJ_CUDA(cudaGetLastError());
      cur = dstb;
    }
  }

  fj_graph* g = new fj_graph();
  g->device = device;
  g->n = n;
  g->weighted = weighted ? 1 : 0;
  auto fail = [&](fj_status rc) {
    if (g->row_ptr) cudaFreeAsync(g->row_ptr, st);
    if (g->dinv) cudaFreeAsync(g->dinv, st);
    if (g->tile_row) cudaFreeAsync(g->tile_row, st);
    delete g;
    return rc;
  };
  if (cudaMallocAsync(&g->row_ptr, (n + 1) * sizeof(int32_t), st) != cudaSuccess ||
      cudaMallocAsync(&g->dinv, n * sizeof(float), st) != cudaSuccess) {
    cudaGetLastError();
    set_error("fj_graph_upload: out of device memory");
    return fail(FJ_ERR_OOM);
  }
  k_row_ptr<<<grid_for(N + 1, 256), 256, 0, st>>>((int32_t*)kb[cur].p, N, n, g->row_ptr);
  if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);
  int32_t nnz32 = 0;
  if (cudaMemcpyAsync(&nnz32, g->row_ptr + n, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(FJ_ERR_CUDA);
  g->nnz = nnz32;
  // The sorted col/val buffers become the graph's (their tail past nnz holds
  // self-loop entries or padding; zero the padding region after nnz).
  g->col = (int32_t*)cb[cur].p;
  cb[cur].p = nullptr;
  if (cudaMemsetAsync(g->col + g->nnz, 0, kPad * 4, st) != cudaSuccess) return fail(FJ_ERR_CUDA);
  if (weighted) {
    g->val = (float*)vb[cur].p;
    vb[cur].p = nullptr;
    if (cudaMemsetAsync(g->val + g->nnz, 0, kPad * 4, st) != cudaSuccess) return fail(FJ_ERR_CUDA);
  }
  auto fail2 = [&](fj_status rc) {
    if (g->col) cudaFreeAsync(g->col, st);
    if (g->val) cudaFreeAsync(g->val, st);
    return fail(rc);
  };
  // merge-path tile plan
  g->n_tiles = (n + g->nnz + kTileItems - 1) / kTileItems;
  if (cudaMallocAsync(&g->tile_row, (g->n_tiles + 1) * sizeof(int32_t), st) != cudaSuccess) {
    cudaGetLastError();
    return fail2(FJ_ERR_OOM);
  }
  k_tile_rows<<<grid_for(g->n_tiles + 1, 256), 256, 0, st>>>(g->row_ptr, n, g->nnz, g->n_tiles,
                                                             g->tile_row);
  if (cudaGetLastError() != cudaSuccess) return fail2(FJ_ERR_CUDA);
  // Jacobi preconditioner 1 / (1 + d_i)
  if (!weighted) {
    k_dinv_unit<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, g->dinv);
    if (cudaGetLastError() != cudaSuccess) return fail2(FJ_ERR_CUDA);
  } else {
    int64_t warps = g->n_tiles < 152 * 64 ? g->n_tiles : 152 * 64;
    if (warps < 1) warps = 1;
    WalkGraph wg{g->row_ptr, g->col, g->val, g->tile_row, n, g->nnz, g->n_tiles,
                 (g->n_tiles + warps - 1) / warps};
    const int64_t blocks = (warps + kWalkWarps - 1) / kWalkWarps;
    DevBuf sums, wrow, wval;
    sums.st = wrow.st = wval.st = st;
    if (cudaMallocAsync(&sums.p, n * 8, st) != cudaSuccess ||
        cudaMallocAsync(&wrow.p, blocks * kWalkWarps * 4, st) != cudaSuccess ||
        cudaMallocAsync(&wval.p, blocks * kWalkWarps * 8, st) != cudaSuccess) {
      cudaGetLastError();
      return fail2(FJ_ERR_OOM);
    }
    k_row_sums<<<(unsigned)blocks, kWalkWarps * 32, 0, st>>>(wg, (double*)sums.p, (int32_t*)wrow.p,
                                                             (double*)wval.p);
    k_dinv_weighted<<<grid_for(n, 256), 256, 0, st>>>(wg, (double*)sums.p, (double*)wval.p, g->dinv);
    if (cudaGetLastError() != cudaSuccess) return fail2(FJ_ERR_CUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail2(FJ_ERR_CUDA);
  *out = g;
  return FJ_OK;
}

fj_status fj_free_graph_device(fj_graph* g, cudaStream_t st) {
  if (!g) return FJ_OK;
  cudaFreeAsync(g->row_ptr, st);
  cudaFreeAsync(g->col, st);
  if (g->val) cudaFreeAsync(g->val, st);
  cudaFreeAsync(g->dinv, st);
  cudaFreeAsync(g->tile_row, st);
  FJ_CUDA(cudaStreamSynchronize(st));
  delete g;
  return FJ_OK;
}
