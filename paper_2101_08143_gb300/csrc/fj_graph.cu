// fj_graph.cu - device construction of the graph of I + L (Sec. 2.1).
//
// Input: an undirected edge list (src, dst, w), each edge once.  Every edge
// e = (u, v) yields two directed entries, (row u, col v) and (row v, col u),
// numbered 2e and 2e+1.  Self-loops contribute nothing to L
// (b_e = e_i - e_i = 0) and are dropped.
//
//   1. one pass over the edges validates them and counts node degrees;
//   2. nodes are renumbered by decreasing degree (a stable radix sort of
//      saturated degree keys), which fixes the solver-order row pointers and
//      the SpMV layouts: chunks of the long rows, sliced ELL for the rest,
//      and the work units;
//   3. one streaming pass writes the 2m directed entries in solver
//      numbering; a stable LSD radix sort of them by row puts every entry at
//      its CSR position, rows keeping the input order of their entries, and
//      its last pass also writes the sliced-ELL copy;
//   4. the Jacobi preconditioner 1 / (1 + d_i).
// The graph, and every sum over it, is therefore the same bits on every
// upload.  The host waits once, at the end, for the sizes and the
// validation result; invalid edges are treated as self-loops until then, so
// no kernel indexes out of range.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fj_internal.cuh"
#include "fj_walk.cuh"

namespace fj {

constexpr int kSortThreads = 512;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr int64_t kScanDirectTiles = 1024;

// ------------------------------------------------------------ validation

// csrc/cdst/cw (nullable): the edge list is read from mapped host memory
// and copied to these device arrays on the way.
//
// Degree counts: power-law graphs send millions of increments to each hub,
// which serialize on one L2 address.  Each block therefore first counts in a
// shared-memory table of kDegSlots nodes (claimed by the first node that
// hashes to a slot; the hubs, being frequent, claim theirs early), and adds
// the table to the global counts once at the end; other nodes go straight to
// the global counts.  The counts are integers, so the result is exact.
constexpr int kDegSlots = 2048;

__device__ __forceinline__ void count_endpoint(int32_t v, int32_t* skey, int32_t* scnt, int32_t* deg) {
  const unsigned slot = ((unsigned)v * 2654435761u) >> 21;  // 11 bits: kDegSlots slots
  int32_t k = *reinterpret_cast<volatile int32_t*>(&skey[slot]);
  if (k == -1) {
    k = atomicCAS(&skey[slot], -1, v);
    if (k == -1) k = v;
  }
  if (k == v)
    atomicAdd(&scnt[slot], 1);
  else
    atomicAdd(&deg[v], 1);
}

__global__ void k_validate_degree(int64_t m, int64_t n, const int32_t* __restrict__ src,
                                  const int32_t* __restrict__ dst, const float* __restrict__ w,
                                  int64_t* __restrict__ err, int32_t* __restrict__ deg,
                                  int32_t* __restrict__ csrc, int32_t* __restrict__ cdst,
                                  float* __restrict__ cw) {
  __shared__ int32_t skey[kDegSlots], scnt[kDegSlots];
  for (int i = threadIdx.x; i < kDegSlots; i += blockDim.x) {
    skey[i] = -1;
    scnt[i] = 0;
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    const float x = w ? w[e] : 1.0f;
    if (csrc) {
      csrc[e] = u;
      cdst[e] = v;
      if (w) cw[e] = x;
    }
    int bad = 0;
    if (u < 0 || u >= n || v < 0 || v >= n) bad |= kErrBadId;
    if (w) {
      if (!(x > 0.0f) || isinf(x)) bad |= kErrBadWeight;
    }
    if (bad) {
      atomicOr(reinterpret_cast<unsigned long long*>(&err[0]), (unsigned long long)bad);
      atomicMin(reinterpret_cast<unsigned long long*>(&err[1]), (unsigned long long)e);
    } else if (u != v) {
      count_endpoint(u, skey, scnt, deg);
      count_endpoint(v, skey, scnt, deg);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kDegSlots; i += blockDim.x)
    if (skey[i] >= 0 && scnt[i] > 0) atomicAdd(&deg[skey[i]], scnt[i]);
}

// ------------------------------------------------------------- radix sort

// Sort input: key = solver-order row id (n for a self-loop or an invalid
// edge), col = solver-order column, weight (null: unit weights).
struct EntrySrc {
  const int32_t* key;
  const int32_t* col;
  const float* val;
  int32_t n;
};

__device__ __forceinline__ void load_entry(const EntrySrc& s, int64_t p, int32_t& key, int32_t& col,
                                           float& val) {
  key = s.key[p];
  col = s.col[p];
  val = s.val ? s.val[p] : 1.0f;
}

// The directed entries of the edge list in solver numbering: entry 2e is
// (new(u), new(v)), entry 2e+1 is (new(v), new(u)), both of weight w_e; a
// self-loop or an invalid edge gets the key n (sorted past the last row).
__global__ void k_make_entries(int64_t m, int32_t n, const int32_t* __restrict__ src,
                               const int32_t* __restrict__ dst, const float* __restrict__ w,
                               const int32_t* __restrict__ old2new, int2* __restrict__ key2,
                               int2* __restrict__ col2, float2* __restrict__ val2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    const bool ok = u != v && u >= 0 && u < n && v >= 0 && v < n;
    const int32_t nu = ok ? old2new[u] : n, nv = ok ? old2new[v] : n;
    key2[e] = make_int2(nu, nv);
    col2[e] = ok ? make_int2(nv, nu) : make_int2(0, 0);
    if (val2) {
      const float x = w[e];
      val2[e] = make_float2(x, x);
    }
  }
}

// Where the last pass of the entry sort writes: the CSR (sorted position =
// CSR position) and, for rows past the long ones, the sliced ELL.
struct EntryDst {
  int32_t* col;
  float* val;
  const int32_t* row_ptr;
  const int64_t* cnt;  // cnt[0] = n_long
  const int64_t* slice_off;
  int32_t* sell_col;
  float* sell_val;
};

// Digits of up to kBits bits: the digit of a pass is
// (key >> shift) & (2^width - 1) with width <= kBits.
template <int kBits, int kItems>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(EntrySrc s, int64_t N, int shift, int width,
                                                             int32_t* __restrict__ hist) {
  constexpr int kD = 1 << kBits;
  constexpr int kSortChunk = kSortThreads * kItems;
  __shared__ int h[kD];
  const int D = 1 << width, mask = D - 1;
  for (int i = threadIdx.x; i < D; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  for (int i = threadIdx.x; i < kSortChunk; i += kSortThreads) {
    const int64_t p = base + i;
    if (p < N) {
      int32_t key, col;
      float val;
      load_entry(s, p, key, col, val);
      atomicAdd(&h[(key >> shift) & mask], 1);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < D; i += kSortThreads) hist[(int64_t)i * gridDim.x + blockIdx.x] = h[i];
}

// Stable scatter of one chunk of kSortThreads * kItems items.  Items are ranked in
// input order (by warp, then round, then lane), placed in shared memory in
// digit order, and written out as one contiguous run per digit, so that
// global stores are coalesced.  LAST: the sorted position is
// the entry's CSR position; write the CSR and sliced-ELL copies instead of
// the sort buffers (entries keyed n are dropped).
template <int kBits, int kItems>
struct ScatterSmem {
  int32_t key[kSortThreads * kItems];
  int32_t col[kSortThreads * kItems];
  float val[kSortThreads * kItems];
  int wcnt[kSortThreads / 32][1 << kBits];
  int run[1 << kBits];
  int start[1 << kBits];
};

template <bool LAST, int kBits, int kItems>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(EntrySrc s, int64_t N, int shift, int width,
                                                                const int32_t* __restrict__ offs,
                                                                int32_t* __restrict__ okey,
                                                                int32_t* __restrict__ ocol,
                                                                float* __restrict__ oval, EntryDst d) {
  constexpr int kW = kSortThreads / 32;
  constexpr int kD = 1 << kBits;
  constexpr int kPer = kD / 32;  // digits per lane in the scan of the counts
  static_assert(kD <= kSortThreads, "one thread per digit");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<kBits, kItems>& sm = *reinterpret_cast<ScatterSmem<kBits, kItems>*>(smem_raw);
  constexpr int kSortChunk = kSortThreads * kItems;
  constexpr int kSortItems = kItems;
  const int D = 1 << width, mask = D - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t cbase = (int64_t)blockIdx.x * kSortChunk;
  const int cnt = (int)((N - cbase) < kSortChunk ? (N - cbase) : kSortChunk);
  // warp w holds chunk items w*32*kItems + r*32 + lane (r < kItems), so the
  // input order is (warp, round, lane): each warp ranks its own items
  // against warp-private digit counters, and one block-wide pass turns the
  // counters into per-warp offsets
  for (int j = lane; j < kD; j += 32) sm.wcnt[warp][j] = 0;
  int32_t key[kSortItems], col[kSortItems];
  float val[kSortItems];
  int rank[kSortItems];
  const int wbase = warp * 32 * kSortItems;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int li = wbase + r * 32 + lane;
    key[r] = 0;
    col[r] = 0;
    val[r] = 0.f;
    if (li < cnt) load_entry(s, cbase + li, key[r], col[r], val[r]);
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = wbase + r * 32 + lane < cnt;
    const int digit = valid ? ((key[r] >> shift) & mask) : kD;
    const unsigned peers = __match_any_sync(kFull, digit);
    const int rk = __popc(peers & lt_mask);
    const int before = valid ? sm.wcnt[warp][digit] : 0;
    __syncwarp();
    if (valid && rk == 0) sm.wcnt[warp][digit] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + rk;
  }
  __syncthreads();
  if (tid < kD) {  // per digit: offsets of the warps' runs, and the total
    int acc = 0;
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      const int c = sm.wcnt[w][tid];
      sm.wcnt[w][tid] = acc;
      acc += c;
    }
    sm.run[tid] = acc;
  }
  __syncthreads();
  // chunk-local start of every digit: exclusive scan of the kD counts
  if (warp == 0) {
    int v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      v[q] = sm.run[lane * kPer + q];
      sum += v[q];
    }
    int incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += y;
    }
    int excl = incl - sum;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      sm.start[lane * kPer + q] = excl;
      excl += v[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    if (wbase + r * 32 + lane < cnt) {
      const int digit = (key[r] >> shift) & mask;
      const int pos = sm.start[digit] + sm.wcnt[warp][digit] + rank[r];
      sm.key[pos] = key[r];
      sm.col[pos] = col[r];
      sm.val[pos] = val[r];
    }
  }
  __syncthreads();
  const int64_t n_long = LAST ? d.cnt[0] : 0;
  for (int i = tid; i < cnt; i += kSortThreads) {
    const int32_t k = sm.key[i];
    const int digit = (k >> shift) & mask;
    const int64_t pos = (int64_t)offs[(int64_t)digit * gridDim.x + blockIdx.x] + (i - sm.start[digit]);
    if (LAST) {
      if (k < s.n) {
        const int32_t c = sm.col[i];
        const float v = sm.val[i];
        d.col[pos] = c;
        if (d.val) d.val[pos] = v;
        if (k >= n_long) {
          const int64_t sr = k - n_long;
          const int64_t sp = d.slice_off[sr >> 5] + 32 * (pos - d.row_ptr[k]) + (sr & 31);
          d.sell_col[sp] = c;
          if (d.sell_val) d.sell_val[sp] = v;
        }
      }
    } else {
      okey[pos] = k;
      ocol[pos] = sm.col[i];
      if (oval) oval[pos] = sm.val[i];
    }
  }
}

// ------------------------------------------------------------------ scan

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* sh, T& total) {
  // sh: kScanThreads/32 values
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T y = __shfl_up_sync(kFull, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = (lane < kScanThreads / 32) ? sh[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T y = __shfl_up_sync(kFull, s, off);
      if (lane >= off) s += y;
    }
    if (lane < kScanThreads / 32) sh[lane] = s;
  }
  __syncthreads();
  total = sh[kScanThreads / 32 - 1];
  const T before = warp > 0 ? sh[warp - 1] : T(0);
  __syncthreads();
  return before + x - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* __restrict__ in, int64_t cnt,
                                                              T* __restrict__ sums) {
  __shared__ T sh[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  T v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
    if (p < cnt) v += in[p];
  }
  T total;
  block_exclusive_scan<T>(v, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// offs: the tiles' scanned offsets, or (sums_in) their unscanned sums, which
// warp 0 adds up for the tiles before this one (few tiles only).
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(T* __restrict__ data, int64_t cnt,
                                                             const T* __restrict__ offs, bool sums_in) {
  __shared__ T sh[kScanThreads / 32];
  __shared__ T tile_off;
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  T vals[kScanItems];
  T v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    vals[i] = (base + i < cnt) ? data[base + i] : T(0);
    v += vals[i];
  }
  if (threadIdx.x < 32) {
    T o = 0;
    if (offs && sums_in) {
      for (int64_t b = threadIdx.x; b < (int64_t)blockIdx.x; b += 32) o += offs[b];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) o += __shfl_xor_sync(kFull, o, d);
    } else if (offs) {
      o = offs[blockIdx.x];
    }
    if (threadIdx.x == 0) tile_off = o;
  }
  T total;
  T run = block_exclusive_scan<T>(v, sh, total) + tile_off;
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < cnt) data[base + i] = run;
    run += vals[i];
  }
}

// In-place exclusive scan of cnt values (int32 totals must fit int32).
template <typename T>
static fj_status exclusive_scan(T* data, int64_t cnt, cudaStream_t st) {
  if (cnt <= 0) return FJ_OK;
  const int64_t blocks = (cnt + kScanChunk - 1) / kScanChunk;
  if (blocks == 1) {
    count_launches(1);
    k_scan_apply<T><<<1, kScanThreads, 0, st>>>(data, cnt, nullptr, false);
    FJ_CUDA(cudaGetLastError());
    return FJ_OK;
  }
  T* sums = nullptr;
  FJ_CUDA(malloc_async(&sums, blocks * sizeof(T), st));
  count_launches(1);
  k_scan_reduce<T><<<(unsigned)blocks, kScanThreads, 0, st>>>(data, cnt, sums);
  // up to kScanDirectTiles tiles, each block adds its predecessors' sums
  // itself; beyond that the tile sums are scanned first
  const bool direct = blocks <= kScanDirectTiles;
  fj_status rc = direct ? FJ_OK : exclusive_scan<T>(sums, blocks, st);
  if (rc == FJ_OK) {
    count_launches(1);
    k_scan_apply<T><<<(unsigned)blocks, kScanThreads, 0, st>>>(data, cnt, sums, direct);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "k_scan_apply");
  }
  cudaFreeAsync(sums, st);
  return rc;
}

// ------------------------------------------------------------ CSR pieces

__global__ void k_dinv_unit(const int32_t* __restrict__ row_ptr, int64_t n, float* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dinv[i] = __frcp_rn(1.0f + (float)(row_ptr[i + 1] - row_ptr[i]));
  }
}

// ------------------------------------------------------- solver order

// Sort key of node i: decreasing degree (saturated), payload i.
__global__ void k_degree_keys(const int32_t* __restrict__ deg, int64_t n, int32_t* __restrict__ key,
                              int32_t* __restrict__ id) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[i];
    key[i] = kDegKeyMax - (d < kDegKeyMax ? d : kDegKeyMax);
    id[i] = (int32_t)i;
  }
}

// old2new[perm[i]] = i; deg_new[i] = degree of perm[i] (into rp_new[i]).
__global__ void k_apply_perm(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg, int64_t n,
                             int32_t* __restrict__ old2new, int32_t* __restrict__ rp_new) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i == n) {
      rp_new[n] = 0;
    } else {
      const int32_t o = perm[i];
      old2new[o] = (int32_t)i;
      rp_new[i] = deg[o];
    }
  }
}

// out[0] = n_long, the number of rows with more than sell_max entries;
// out[1] = n_nz, the number of rows with at least one entry (in solver order
// both are prefixes of the rows).
__global__ void k_count_long(const int32_t* __restrict__ row_ptr, int64_t n, int64_t* __restrict__ out,
                             int32_t sell_max) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = row_ptr[i + 1] - row_ptr[i];
    const int32_t dn = (i + 1 < n) ? row_ptr[i + 2] - row_ptr[i + 1] : 0;
    if (d > sell_max && dn <= sell_max) out[0] = i + 1;
    if (d > 0 && dn == 0) out[1] = i + 1;
  }
}

// Device-side sizes of the layout (cnt[0], cnt[1] from k_count_long):
//   cnt[0] n_long, cnt[1] n_nz, cnt[2] n_slices, cnt[3] nnz
// slice_off[s] = 32 * (length of the slice's first, i.e. longest, row) and
// long_first[r] = number of chunks of long row r (both scanned afterwards);
// entries past the live counts are 0 so that scans over upper bounds work.
__global__ void k_layout_sizes(const int32_t* __restrict__ row_ptr, int64_t n, int64_t* __restrict__ cnt,
                               int64_t ns_cap, int64_t nl_cap, int64_t* __restrict__ slice_off,
                               int32_t* __restrict__ long_first, int32_t chunk_len) {
  const int64_t n_long = cnt[0];
  const int64_t n_nz = cnt[1] > n_long ? cnt[1] : n_long;
  const int64_t n_slices = (n_nz - n_long + 31) / 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= ns_cap + nl_cap + 1;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0) {
      cnt[2] = n_slices;
      cnt[3] = row_ptr[n];
    }
    if (i <= ns_cap) {
      slice_off[i] = (i < n_slices) ? 32 * (int64_t)(row_ptr[n_long + 32 * i + 1] - row_ptr[n_long + 32 * i]) : 0;
    } else {
      const int64_t r = i - ns_cap - 1;  // r in [0, nl_cap]
      long_first[r] = (r < n_long) ? (row_ptr[r + 1] - row_ptr[r] + chunk_len - 1) / chunk_len : 0;
    }
  }
}

// Work-unit cost model of the narrow walk (K <= 4), in units of 1/8 ns: a
// fixed part per unit (its dependent round trips: unit bounds, then indices,
// then gathers) plus a part per chunk entry or per slice step (one entry per
// lane).  Fitted by least squares to per-warp walk times on a power-law
// graph (n = 10^6, 10^7 entries, 4864 warps): 1.37 us + 6.5 ns per chunk
// entry, 1.05 us + 0.25 us per slice step.
constexpr int64_t kCostChunk = 8 * 1375, kCostChunkEntry = 52;
constexpr int64_t kCostSlice = 8 * 1055, kCostSliceStep = 8 * 250;

// Fills the chunk table and the work-unit costs: unit_cost[c] for chunk c,
// unit_cost[n_chunks + s] for slice s, 0 beyond (the array is sized by an
// upper bound and scanned over all of it).
// Also completes the sizes: cnt[4] = n_chunks, cnt[5] = sliced-ELL entries.
__global__ void k_units(const int32_t* __restrict__ row_ptr, int64_t* __restrict__ cnt,
                        const int32_t* __restrict__ long_first, const int64_t* __restrict__ slice_off,
                        int64_t units_cap, int32_t* __restrict__ chunk_row, int32_t* __restrict__ chunk_begin,
                        int32_t* __restrict__ chunk_end, int64_t* __restrict__ unit_cost, int32_t chunk_len) {
  const int64_t n_long = cnt[0], n_slices = cnt[2];
  const int64_t n_chunks = long_first[n_long];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt[4] = n_chunks;
    cnt[5] = slice_off[n_slices];
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_long;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = row_ptr[r], e = row_ptr[r + 1];
    for (int32_t c = long_first[r], q = 0; c < long_first[r + 1]; ++c, ++q) {
      const int32_t cb = b + q * chunk_len;
      const int32_t ce = cb + chunk_len < e ? cb + chunk_len : e;
      chunk_row[c] = (int32_t)r;
      chunk_begin[c] = cb;
      chunk_end[c] = ce;
      unit_cost[c] = kCostChunk + kCostChunkEntry * (int64_t)(ce - cb);
    }
  }
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= units_cap;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (u < n_chunks) continue;
    const int64_t s = u - n_chunks;
    unit_cost[u] = (s < n_slices) ? kCostSlice + kCostSliceStep * ((slice_off[s + 1] - slice_off[s]) >> 5) : 0;
  }
}

// Sliced ELL padding: positions past a row's length get col = the row itself
// (w (x_r - x_r) = 0 for any weight) and weight 0.  One warp per slice.
__global__ void k_sell_pad(const int32_t* __restrict__ row_ptr, int64_t n, const int64_t* __restrict__ cnt,
                           const int64_t* __restrict__ slice_off, int32_t* __restrict__ sell_col,
                           float* __restrict__ sell_val) {
  const int64_t n_long = cnt[0], n_slices = cnt[2];
  const int lane = threadIdx.x & 31;
  for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < n_slices;
       s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t row = n_long + 32 * s + lane;
    const int32_t len = row < n ? row_ptr[row + 1] - row_ptr[row] : 0;
    const int64_t off = slice_off[s];
    const int32_t slen = (int32_t)((slice_off[s + 1] - off) >> 5);
    for (int32_t p = len; p < slen; ++p) {
      sell_col[off + 32 * (int64_t)p + lane] = row < n ? (int32_t)row : 0;
      if (sell_val) sell_val[off + 32 * (int64_t)p + lane] = 0.0f;
    }
  }
}

// Weighted degrees, accumulated in float32 in a fixed order (the Jacobi
// preconditioner needs no more).  Long rows: a warp per chunk sums its
// entries (lane-strided, then an xor tree) ...
__global__ void k_chunk_wsum(const float* __restrict__ val, const int32_t* __restrict__ long_first,
                             const int64_t* __restrict__ cnt, const int32_t* __restrict__ chunk_begin,
                             const int32_t* __restrict__ chunk_end, float* __restrict__ part) {
  const int64_t n_chunks = long_first[cnt[0]];
  const int lane = threadIdx.x & 31;
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < n_chunks;
       c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t e = chunk_end[c];
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int32_t p = chunk_begin[c] + lane;
    for (; p + 96 < e; p += 128) {
      a[0] += val[p];
      a[1] += val[p + 32];
      a[2] += val[p + 64];
      a[3] += val[p + 96];
    }
    for (; p < e; p += 32) a[0] += val[p];
    float d = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(kFull, d, off);
    if (lane == 0) part[c] = d;
  }
}

// ... then a warp per long row adds its chunk sums, and a thread per short
// row walks its sliced-ELL positions in order.  dinv_i = 1 / (1 + d_i).
__global__ void k_dinv_weighted(const int32_t* __restrict__ row_ptr, int64_t n, const int64_t* __restrict__ cnt,
                                const int32_t* __restrict__ long_first, const float* __restrict__ part,
                                const int64_t* __restrict__ slice_off, const float* __restrict__ sell_val,
                                float* __restrict__ dinv) {
  const int64_t n_long = cnt[0], n_nz = cnt[1] > cnt[0] ? cnt[1] : cnt[0];
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < n_long; r += nw) {
    float d = 0.0f;
    for (int32_t c = long_first[r] + lane; c < long_first[r + 1]; c += 32) d += part[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(kFull, d, off);
    if (lane == 0) dinv[r] = __frcp_rn(1.0f + d);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - n_long;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = n_long + i;
    float d = 0.0f;
    if (row < n_nz) {
      const int32_t len = row_ptr[row + 1] - row_ptr[row];
      const float* __restrict__ v = sell_val + slice_off[i >> 5] + (i & 31);
      for (int32_t p = 0; p < len; ++p) d += v[32 * p];
    }
    dinv[row] = __frcp_rn(1.0f + d);
  }
}

// ------------------------------------------------- repeated pairs (Sec. 2.1)
//
// Without FJ_MERGE_DUPLICATES the edge list must be simple.  A pair listed
// twice gives two entries of equal column in both of its rows, so it is
// found by checking that no row repeats a column.  A hit records the pair's
// input ids (smaller first; the smallest pair wins) in err[2].

__device__ __forceinline__ void report_duplicate(int64_t* err, const int32_t* perm, int64_t r, int32_t c) {
  const uint32_t a = (uint32_t)perm[r], b = (uint32_t)perm[c];
  const unsigned long long pair =
      ((unsigned long long)(a < b ? a : b) << 32) | (unsigned long long)(a < b ? b : a);
  atomicOr(reinterpret_cast<unsigned long long*>(&err[0]), (unsigned long long)kErrDuplicate);
  atomicMin(reinterpret_cast<unsigned long long*>(&err[2]), pair);
}

// Short rows [n_long, n_nz) (at most kSellMaxLen entries): each warp takes
// the rows whose first entry falls in its share of the entries, and packs as
// many whole rows as fit into a window of 32 entries.  One match over the
// keys (row within the window, column) finds a repeat; a row of 33..64
// entries compares its two halves, then each of its second-half entries
// against the first half.
__global__ void k_dup_short(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ cnt, const int32_t* __restrict__ perm,
                            int64_t* __restrict__ err) {
  const int64_t n_long = cnt[0], n_nz = cnt[1] > cnt[0] ? cnt[1] : cnt[0];
  if (n_nz <= n_long) return;
  const int lane = threadIdx.x & 31;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t e0 = row_ptr[n_long], E = (int64_t)row_ptr[n_nz] - e0;
  // rows [ra, rb): first row whose start is >= the share's first entry
  int64_t bound = 0;
  if (lane < 2) {
    const int64_t target = e0 + (E * (w + lane)) / W;
    int64_t lo = n_long, hi = n_nz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    bound = lo;
  }
  const int64_t ra = __shfl_sync(kFull, bound, 0), rb = __shfl_sync(kFull, bound, 1);
  const unsigned long long lane_key = ~0ull - (unsigned long long)lane;  // matches no valid key
  for (int64_t r = ra; r < rb;) {
    const int32_t p0 = row_ptr[r];
    // ends of rows r .. r+31 (clamped to the warp's rows)
    const int64_t rj = r + 1 + lane;
    const int32_t end = rj <= rb ? row_ptr[rj] : INT32_MAX;
    const unsigned fit = __ballot_sync(kFull, end - p0 <= 32);  // whole rows in the window (a prefix)
    const int q = __popc(fit);
    if (q > 0) {
      const int32_t wend = __shfl_sync(kFull, end, q - 1);
      // bit b set where a row starts at window offset b > 0
      const unsigned starts =
          __reduce_or_sync(kFull, (lane < q - 1) ? (1u << (end - p0)) : 0u);
      const int32_t p = p0 + lane;
      const bool valid = p < wend;
      const int rl = __popc(starts & ((2u << lane) - 1u));
      const int32_t c = valid ? col[p] : 0;
      const unsigned long long key = valid ? (((unsigned long long)rl << 32) | (uint32_t)c) : lane_key;
      const unsigned peers = __match_any_sync(kFull, key);
      if (valid && __popc(peers) > 1 && (peers & ((1u << lane) - 1u)) == 0) report_duplicate(err, perm, r + rl, c);
      r += q;
    } else {
      // one row of 33..64 entries
      const int32_t d = row_ptr[r + 1] - p0;
      const int32_t a = col[p0 + lane];
      const bool hb = lane < d - 32;
      const int32_t bv = hb ? col[p0 + 32 + lane] : 0;
      // every lane takes part in both matches (no short-circuit around them)
      const unsigned pa = __match_any_sync(kFull, (unsigned long long)(uint32_t)a);
      const unsigned long long kb = hb ? (unsigned long long)(uint32_t)bv : lane_key;
      const unsigned pb = __match_any_sync(kFull, kb);
      bool hit_a = __popc(pa) > 1;
      const bool hit_b = hb && __popc(pb) > 1;
      for (int j = 0; j < d - 32; ++j) hit_a |= (__shfl_sync(kFull, bv, j) == a);
      if (hit_a) report_duplicate(err, perm, r, a);
      if (hit_b) report_duplicate(err, perm, r, bv);
      r += 1;
    }
  }
}

// Long rows [0, n_long): row r owns the hash segment of 2 * deg(r) slots at
// 2 * row_ptr[r] (set to -1 first); every entry inserts its column by linear
// probing from a multiplicative hash.  At most half the slots fill, so a
// probe ends at an empty slot or at its own column within the segment.
__global__ void k_dup_fill(int32_t* __restrict__ table, const int32_t* __restrict__ row_ptr,
                           const int64_t* __restrict__ cnt) {
  const int64_t total = 2 * (int64_t)row_ptr[cnt[0]];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    table[i] = -1;
}

__global__ void k_dup_long(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ cnt, const int32_t* __restrict__ chunk_row,
                           const int32_t* __restrict__ chunk_begin, const int32_t* __restrict__ chunk_end,
                           int32_t* __restrict__ table, const int32_t* __restrict__ perm,
                           int64_t* __restrict__ err) {
  const int64_t n_chunks = cnt[4];
  const int lane = threadIdx.x & 31;
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < n_chunks;
       ch += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t r = chunk_row[ch];
    const int64_t base = 2 * (int64_t)row_ptr[r];
    const uint32_t size = 2u * (uint32_t)(row_ptr[r + 1] - row_ptr[r]);
    for (int32_t p = chunk_begin[ch] + lane; p < chunk_end[ch]; p += 32) {
      const int32_t c = col[p];
      uint32_t h = (uint32_t)(((uint64_t)((uint32_t)c * 2654435761u) * size) >> 32);
      for (uint32_t probe = 0; probe < size; ++probe) {
        const int32_t prev = atomicCAS(&table[base + h], -1, c);
        if (prev == -1) break;
        if (prev == c) {
          report_duplicate(err, perm, r, c);
          break;
        }
        h = (h + 1 == size) ? 0 : h + 1;
      }
    }
  }
}

static unsigned grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

// Stable LSD radix sort of N entries by key in [0, key_max], from buffer set
// 0, in passes of digits of at most kBits bits (their widths differ by at
// most one bit), chunks of kSortThreads * kItems entries per block.  Buffers kb/cb/vb[2] must hold N + kPad
// elements (vb may be null: no val); returns the index (0/1) of the buffer
// set holding the result.  With `last`, the last pass writes the CSR and
// sliced ELL instead.  The result is the unique stable order, whatever the
// digit widths.
template <int kBits, int kItems>
static fj_status radix_passes(int32_t n, int64_t N, int bits, int32_t* kb[2], int32_t* cb[2], float* vb[2],
                              const EntryDst* last, cudaStream_t st, int* result) {
  const int passes = (bits + kBits - 1) / kBits;
  constexpr int kSortChunk = kSortThreads * kItems;
  const int64_t nblocks = (N + kSortChunk - 1) / kSortChunk;
  int cur = 0;
  *result = 0;
  if (N == 0) return FJ_OK;
  int32_t* h = nullptr;
  FJ_CUDA(malloc_async(&h, ((int64_t)1 << kBits) * nblocks * sizeof(int32_t), st));
  fj_status rc = FJ_OK;
  const size_t ssm = sizeof(ScatterSmem<kBits, kItems>);
  const EntryDst none{};
  int shift = 0;
  for (int pass = 0; pass < passes && rc == FJ_OK; ++pass) {
    // widths differ by at most one bit, the wider ones first
    const int width = bits / passes + (pass < bits % passes ? 1 : 0);
    const bool fin = last && pass == passes - 1;
    const EntrySrc s{kb[cur], cb[cur], vb[cur], n};
    const int dstb = 1 - cur;
    count_launches(2);
    k_radix_hist<kBits, kItems><<<(unsigned)nblocks, kSortThreads, 0, st>>>(s, N, shift, width, h);
    rc = exclusive_scan<int32_t>(h, ((int64_t)1 << width) * nblocks, st);
    if (rc != FJ_OK) break;
    const EntryDst& d = fin ? *last : none;
    auto launch = [&](auto kern) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
      kern<<<(unsigned)nblocks, kSortThreads, ssm, st>>>(s, N, shift, width, h, kb[dstb], cb[dstb], vb[dstb], d);
    };
    if (fin)
      launch(k_radix_scatter<true, kBits, kItems>);
    else
      launch(k_radix_scatter<false, kBits, kItems>);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "radix sort");
    cur = dstb;
    shift += width;
  }
  cudaFreeAsync(h, st);
  *result = cur;
  return rc;
}

static fj_status radix_sort(int32_t n, int64_t N, int64_t key_max, int32_t* kb[2], int32_t* cb[2], float* vb[2],
                            const EntryDst* last, cudaStream_t st, int* result) {
  int bits = 1;
  while ((int64_t(1) << bits) <= key_max) ++bits;
  // 8-bit digits, 8 items per thread: measured against 9-bit digits (one
  // pass fewer at 25-27 bits) and 12 or 16 items per thread, which were
  // slower: a wider digit or a longer chunk shortens each digit's output
  // run, and the scatter's stores lose more than the saved pass
  return radix_passes<8, 8>(n, N, bits, kb, cb, vb, last, st, result);
}

}  // namespace fj

using namespace fj;

namespace {

// Stream-ordered device allocations released at scope exit unless kept.
struct Pool {
  cudaStream_t st;
  std::vector<void*> ptrs;
  bool failed = false;
  explicit Pool(cudaStream_t s) : st(s) {}
  template <typename T>
  T* get(int64_t count) {
    void* p = nullptr;
    if (malloc_async(&p, (size_t)std::max<int64_t>(count, 1) * sizeof(T), st) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
  void keep(const void* p) {
    for (auto& q : ptrs)
      if (q == p) q = nullptr;
  }
  ~Pool() {
    for (void* p : ptrs)
      if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace

void fj_free_graph_arrays(fj_graph* g, cudaStream_t st) {
  void* arrays[] = {g->row_ptr,     g->col,       g->val,         g->dinv,      g->perm,
                    g->long_first,  g->chunk_row, g->chunk_begin, g->chunk_end, g->slice_off,
                    g->sell_col,    g->sell_val,  g->unit_prefix, g->orig_ids};
  for (void* p : arrays)
    if (p) cudaFreeAsync(p, st);
}

// Called by the C ABI (fj_api.cpp).  src/dst/w are device pointers.
// Host words of a build: [0] n_long [1] n_nz [2] n_slices [3] nnz
// [4] n_chunks [5] sliced-ELL entries [6] error bits [7] first invalid edge
// [8] first repeated pair.
constexpr int kBuildWords = 9;

// First half of a build: every kernel and, last, the copy of the sizes and
// the validation words (kBuildWords int64) to host_words, all enqueued on st.
// *pending receives the graph, whose sizes fj_build_graph_end fills in once
// that copy has completed; host_words must stay valid until then (page-locked
// memory for an asynchronous copy).
fj_status fj_build_graph_begin(int device, cudaStream_t st, int64_t n, int64_t m, const int32_t* src,
                               const int32_t* dst, const float* w, bool merge_duplicates, const Layout& lay,
                               int64_t* host_words, fj_graph** pending, int32_t* copy_src, int32_t* copy_dst,
                               float* copy_w) {
  fj_graph** out = pending;
  const int64_t N = 2 * m;
  const bool weighted = (w != nullptr);
  Pool pool(st);
  auto oom = [&]() {
    set_error("fj_graph_upload: out of device memory (n=%lld, m=%lld)", (long long)n, (long long)m);
    return FJ_ERR_OOM;
  };
  // dcnt: [0] n_long [1] n_nz [2] n_slices [3] nnz [4] n_chunks [5] sliced-ELL
  // entries [6] error bits [7] first invalid edge [8] first repeated pair
  int64_t* dcnt = pool.get<int64_t>(kBuildWords);
  int32_t* deg = pool.get<int32_t>(n);
  if (pool.failed) return oom();
  FJ_CUDA(cudaMemsetAsync(dcnt, 0, 56, st));
  FJ_CUDA(cudaMemsetAsync(dcnt + 7, 0xff, 16, st));
  FJ_CUDA(cudaMemsetAsync(deg, 0, n * sizeof(int32_t), st));

  // ---- 1. validation and degrees
  if (m > 0) {
    count_launches(1);
    k_validate_degree<<<grid_for(m, 256), 256, 0, st>>>(m, n, src, dst, w, dcnt + 6, deg, copy_src, copy_dst,
                                                         copy_w);
    FJ_CUDA(cudaGetLastError());
  }
  if (copy_src) {  // later passes read the device copy
    src = copy_src;
    dst = copy_dst;
    if (w) w = copy_w;
  }

  // ---- 2. solver order: stable sort of nodes by decreasing degree
  int32_t* kb2[2] = {pool.get<int32_t>(n + kPad), pool.get<int32_t>(n + kPad)};
  int32_t* cb2[2] = {pool.get<int32_t>(n + kPad), pool.get<int32_t>(n + kPad)};
  float* vb2[2] = {nullptr, nullptr};
  if (pool.failed) return oom();
  count_launches(1);
  k_degree_keys<<<grid_for(n, 256), 256, 0, st>>>(deg, n, kb2[0], cb2[0]);
  FJ_CUDA(cudaGetLastError());
  int cur2 = 0;
  fj_status rc = radix_sort((int32_t)n, n, kDegKeyMax, kb2, cb2, vb2, nullptr, st, &cur2);
  if (rc != FJ_OK) return rc;
  int32_t* perm = cb2[cur2];

  fj_graph* g = new fj_graph();
  memset(g, 0, sizeof(*g));
  g->device = device;
  g->n = n;
  g->weighted = weighted ? 1 : 0;
  g->chunk_len = lay.chunk_len;
  g->sell_max = lay.sell_max;
  auto fail = [&](fj_status code) {
    fj_free_graph_arrays(g, st);
    delete g;
    return code;
  };
  // perm is kept: the pool must not free it
  g->perm = perm;
  pool.keep(perm);
  int32_t* old2new = pool.get<int32_t>(n);
  if (malloc_async(&g->row_ptr, (n + 1) * sizeof(int32_t), st) != cudaSuccess || !old2new) {
    cudaGetLastError();
    g->row_ptr = nullptr;
    return fail(oom());
  }
  count_launches(1);
  k_apply_perm<<<grid_for(n + 1, 256), 256, 0, st>>>(perm, deg, n, old2new, g->row_ptr);
  rc = exclusive_scan<int32_t>(g->row_ptr, n + 1, st);
  if (rc != FJ_OK) return fail(rc);

  // ---- 3. layout of long rows, slices, chunk table and work units, from
  // the degrees alone.  Sizes stay on the device; buffers use upper bounds:
  // in decreasing-degree order a slice's first row is no longer than any row
  // of the slice before it, so the sliced ELL holds at most
  // nnz + 32 * sell_max entries.
  const int64_t nl_cap = std::min<int64_t>(n, N / (lay.sell_max + 1));
  const int64_t ns_cap = (n + 31) / 32;
  const int64_t nc_cap = nl_cap + N / lay.chunk_len + 1;
  const int64_t units_cap = nc_cap + ns_cap;
  const int64_t sell_cap = N + 32 * (int64_t)lay.sell_max;
  if (malloc_async(&g->col, (N + kPad) * 4, st) != cudaSuccess ||
      (weighted && malloc_async(&g->val, (N + kPad) * 4, st) != cudaSuccess) ||
      malloc_async(&g->slice_off, (ns_cap + 1) * 8, st) != cudaSuccess ||
      malloc_async(&g->long_first, (nl_cap + 1) * 4, st) != cudaSuccess ||
      malloc_async(&g->sell_col, (sell_cap + kPad) * 4, st) != cudaSuccess ||
      (weighted && malloc_async(&g->sell_val, (sell_cap + kPad) * 4, st) != cudaSuccess) ||
      malloc_async(&g->chunk_row, nc_cap * 4, st) != cudaSuccess ||
      malloc_async(&g->chunk_begin, nc_cap * 4, st) != cudaSuccess ||
      malloc_async(&g->chunk_end, nc_cap * 4, st) != cudaSuccess ||
      malloc_async(&g->unit_prefix, (units_cap + 1) * 8, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(oom());
  }
  // the padding past nnz is read by batched loads (never used)
  cudaMemsetAsync(g->col + N, 0, kPad * 4, st);
  if (weighted) cudaMemsetAsync(g->val + N, 0, kPad * 4, st);
  count_launches(2);
  k_count_long<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, dcnt, lay.sell_max);
  k_layout_sizes<<<grid_for(ns_cap + nl_cap + 2, 256), 256, 0, st>>>(g->row_ptr, n, dcnt, ns_cap, nl_cap,
                                                                    g->slice_off, g->long_first, lay.chunk_len);
  rc = exclusive_scan<int64_t>(g->slice_off, ns_cap + 1, st);
  if (rc == FJ_OK) rc = exclusive_scan<int32_t>(g->long_first, nl_cap + 1, st);
  if (rc != FJ_OK) return fail(rc);
  count_launches(2);
  k_units<<<grid_for(std::max(nl_cap, units_cap + 1), 256), 256, 0, st>>>(
      g->row_ptr, dcnt, g->long_first, g->slice_off, units_cap, g->chunk_row, g->chunk_begin, g->chunk_end,
      g->unit_prefix, lay.chunk_len);
  k_sell_pad<<<grid_for(ns_cap * 32, 256), 256, 0, st>>>(g->row_ptr, n, dcnt, g->slice_off, g->sell_col,
                                                         g->sell_val);
  if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);
  rc = exclusive_scan<int64_t>(g->unit_prefix, units_cap + 1, st);
  if (rc != FJ_OK) return fail(rc);

  // ---- 4. entries, sorted by solver-order row, straight to the CSR and the
  // sliced ELL
  {
    const int64_t cap = N + kPad;
    int32_t* kb[2];
    int32_t* cb[2];
    float* vb[2] = {nullptr, nullptr};
    Pool sort_pool(st);
    for (int i = 0; i < 2; ++i) {
      kb[i] = sort_pool.get<int32_t>(cap);
      cb[i] = sort_pool.get<int32_t>(cap);
      if (weighted) vb[i] = sort_pool.get<float>(cap);
    }
    if (sort_pool.failed) return fail(oom());
    if (m > 0) {
      count_launches(1);
      k_make_entries<<<grid_for(m, 256), 256, 0, st>>>(m, (int32_t)n, src, dst, w, old2new,
                                                        reinterpret_cast<int2*>(kb[0]),
                                                        reinterpret_cast<int2*>(cb[0]),
                                                        reinterpret_cast<float2*>(vb[0]));
      if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);
    }
    EntryDst ed{g->col, g->val, g->row_ptr, dcnt, g->slice_off, g->sell_col, g->sell_val};
    int cur = 0;
    rc = radix_sort((int32_t)n, N, n, kb, cb, vb, &ed, st, &cur);
    if (rc != FJ_OK) return fail(rc);
  }

  // ---- 5. Jacobi preconditioner
  if (malloc_async(&g->dinv, n * sizeof(float), st) != cudaSuccess) {
    cudaGetLastError();
    return fail(oom());
  }
  count_launches(1);
  if (!weighted) {
    k_dinv_unit<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, g->dinv);
  } else {
    float* cpart = pool.get<float>(nc_cap);
    if (!cpart) return fail(oom());
    count_launches(1);
    k_chunk_wsum<<<grid_for(nc_cap * 32, 256), 256, 0, st>>>(g->val, g->long_first, dcnt, g->chunk_begin,
                                                             g->chunk_end, cpart);
    k_dinv_weighted<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, dcnt, g->long_first, cpart, g->slice_off,
                                                      g->sell_val, g->dinv);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);

  // ---- 6. repeated pairs
  if (!merge_duplicates && N > 0) {
    int32_t* table = pool.get<int32_t>(2 * N);
    if (!table) return fail(oom());
    count_launches(3);
    k_dup_fill<<<grid_for(2 * N, 256), 256, 0, st>>>(table, g->row_ptr, dcnt);
    k_dup_long<<<grid_for(nc_cap * 32, 256), 256, 0, st>>>(g->row_ptr, g->col, dcnt, g->chunk_row,
                                                           g->chunk_begin, g->chunk_end, table, g->perm,
                                                           dcnt + 6);
    k_dup_short<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, g->col, dcnt, g->perm, dcnt + 6);
    if (cudaGetLastError() != cudaSuccess) return fail(FJ_ERR_CUDA);
  }

  // ---- sizes and the validation result to the host (the build's one round
  // trip, completed by fj_build_graph_end)
  if (cudaMemcpyAsync(host_words, dcnt, kBuildWords * sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return fail(FJ_ERR_CUDA);
  *out = g;
  return FJ_OK;
}

// Second half: checks the validation words and fills in the sizes, or frees
// the graph (stream-ordered on st) and reports the bad input.
fj_status fj_build_graph_end(fj_graph* g, const int64_t* hc, cudaStream_t st, fj_graph** out) {
  *out = nullptr;
  auto fail = [&](fj_status code) {
    fj_free_graph_arrays(g, st);
    delete g;
    return code;
  };
  if (hc[6] & (kErrBadId | kErrBadWeight)) {
    set_error("fj_graph_upload: edge %llu has %s", (unsigned long long)hc[7],
              (hc[6] & kErrBadId) ? "a node id outside [0, n)" : "a weight that is not finite and > 0");
    return fail(FJ_ERR_GRAPH);
  }
  if (hc[6] & kErrDuplicate) {
    const unsigned long long pr = (unsigned long long)hc[8];
    set_error("fj_graph_upload: the pair (%u, %u) is listed more than once (FJ_MERGE_DUPLICATES adds the "
              "weights of repeated pairs)",
              (unsigned)(pr >> 32), (unsigned)(pr & 0xffffffffu));
    return fail(FJ_ERR_GRAPH);
  }
  g->n_long = hc[0];
  g->n_nz = std::max(hc[1], hc[0]);
  g->n_slices = hc[2];
  g->nnz = hc[3];
  g->n_chunks = hc[4];
  g->sell_nnz = hc[5];
  g->n_units = g->n_chunks + g->n_slices;
  *out = g;
  return FJ_OK;
}

// Both halves with the host waiting in between.
fj_status fj_build_graph_device(int device, cudaStream_t st, int64_t n, int64_t m, const int32_t* src,
                                const int32_t* dst, const float* w, bool merge_duplicates, const Layout& lay,
                                fj_graph** out, int32_t* copy_src, int32_t* copy_dst, float* copy_w) {
  int64_t hc[kBuildWords];
  fj_graph* g = nullptr;
  *out = nullptr;
  fj_status rc = fj_build_graph_begin(device, st, n, m, src, dst, w, merge_duplicates, lay, hc, &g, copy_src,
                                      copy_dst, copy_w);
  if (rc != FJ_OK) return rc;
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fj_free_graph_arrays(g, st);
    delete g;
    return cuda_fail(e, "fj_graph_upload");
  }
  return fj_build_graph_end(g, hc, st, out);
}

fj_status fj_free_graph_device(fj_graph* g, cudaStream_t st) {
  if (!g) return FJ_OK;
  fj_free_graph_arrays(g, st);
  FJ_CUDA(cudaStreamSynchronize(st));
  delete g;
  return FJ_OK;
}

// ------------------------------------------------------- weight updates
//
// New weights for existing edges of a resident graph (the FJ model on a
// changed graph, Sec. 3.1): the entries of each updated pair are found in
// both of its rows and rewritten in the CSR and the sliced ELL, then the
// Jacobi preconditioner is recomputed by the kernels and summation order of
// the build.  A pair listed several times (FJ_MERGE_DUPLICATES) has several
// entries per row; the update rewrites the first, which belongs to the
// first listing of the pair.

namespace fj {

__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[perm[i]] = (int32_t)i;
}

// Sliced-ELL weights of a graph built without weights: 1 for entries, 0 for
// the padding (as the build writes them).
__global__ void k_sell_unit_vals(const int32_t* __restrict__ row_ptr, int64_t n, int64_t n_long, int64_t n_slices,
                                 const int64_t* __restrict__ slice_off, float* __restrict__ sell_val) {
  const int lane = threadIdx.x & 31;
  for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < n_slices;
       s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t row = n_long + 32 * s + lane;
    const int32_t len = row < n ? row_ptr[row + 1] - row_ptr[row] : 0;
    const int64_t off = slice_off[s];
    const int32_t slen = (int32_t)((slice_off[s + 1] - off) >> 5);
    for (int32_t p = 0; p < slen; ++p) sell_val[off + 32 * (int64_t)p + lane] = p < len ? 1.0f : 0.0f;
  }
}

__global__ void k_fill_f32(float* __restrict__ a, int64_t count, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// One warp per update u: pair (src[u], dst[u]) in input ids gets weight
// w[u].  With apply == false it only checks (ids, weight, that the pair is
// an edge) and records the first bad update in err ([0] bits, [1] index);
// with apply == true it writes both directed entries.
__global__ void k_update_weights(int64_t count, int64_t n, const int32_t* __restrict__ src,
                                 const int32_t* __restrict__ dst, const float* __restrict__ w,
                                 const int32_t* __restrict__ inv, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col, float* __restrict__ val, int64_t n_long,
                                 const int64_t* __restrict__ slice_off, float* __restrict__ sell_val, bool apply,
                                 unsigned long long* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < count;
       u += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t a = src[u], b = dst[u];
    const float wn = w[u];
    unsigned long long bad = 0;
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) bad = kErrBadId;
    else if (!(wn > 0.0f) || !isfinite(wn)) bad = kErrBadWeight;
    for (int dir = 0; dir < 2 && !bad; ++dir) {
      const int32_t r = inv[dir ? b : a], c = inv[dir ? a : b];
      const int32_t e = row_ptr[r + 1];
      int32_t first = -1;
      for (int32_t base = row_ptr[r]; base < e; base += 32) {
        const int32_t p = base + lane;
        const unsigned hit = __ballot_sync(kFull, p < e && col[p] == c);
        if (hit) {
          first = base + __ffs(hit) - 1;
          break;
        }
      }
      if (first < 0) {
        bad = kErrDuplicate;  // (reused bit) the pair is not an edge
      } else if (apply && lane == 0) {
        val[first] = wn;
        if (r >= n_long) {
          const int64_t sr = r - n_long;
          sell_val[slice_off[sr >> 5] + 32 * (int64_t)(first - row_ptr[r]) + (sr & 31)] = wn;
        }
      }
    }
    if (bad && lane == 0) {
      atomicOr(&err[0], bad);
      atomicMin(&err[1], (unsigned long long)u);
    }
  }
}

}  // namespace fj

// Called by the C ABI (fj_api.cpp): src/dst/w are device pointers of count
// updates.  On FJ_ERR_GRAPH nothing was changed.
fj_status fj_update_weights_device(fj_graph* g, cudaStream_t st, int64_t count, const int32_t* src,
                                   const int32_t* dst, const float* w) {
  if (count == 0) return FJ_OK;
  const int64_t n = g->n, N = g->nnz;
  Pool pool(st);
  int32_t* inv = pool.get<int32_t>(n);
  unsigned long long* err = pool.get<unsigned long long>(2);
  int64_t* dcnt = pool.get<int64_t>(2);
  if (!inv || !err || !dcnt) {
    set_error("fj_graph_update_weights: out of device memory");
    return FJ_ERR_OOM;
  }
  const unsigned long long init[2] = {0ull, ~0ull};
  FJ_CUDA(cudaMemcpyAsync(err, init, sizeof(init), cudaMemcpyHostToDevice, st));
  count_launches(2);
  k_inverse_perm<<<grid_for(n, 256), 256, 0, st>>>(g->perm, n, inv);
  k_update_weights<<<grid_for(count * 32, 256), 256, 0, st>>>(count, n, src, dst, w, inv, g->row_ptr, g->col,
                                                               g->val, g->n_long, g->slice_off, g->sell_val,
                                                               false, err);
  FJ_CUDA(cudaGetLastError());
  unsigned long long herr[2];
  FJ_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaStreamSynchronize(st));
  if (herr[0]) {
    set_error("fj_graph_update_weights: update %llu %s", herr[1],
              (herr[0] & kErrBadId)       ? "has a node id outside [0, n) or a self-loop"
              : (herr[0] & kErrBadWeight) ? "has a weight that is not finite and > 0"
                                          : "names a pair that is not an edge of the graph");
    return FJ_ERR_GRAPH;
  }
  if (!g->weighted) {
    // a graph built without weights gets its weight arrays (all ones)
    const int64_t sell_cap = N + 32 * (int64_t)g->sell_max;
    float* val = nullptr;
    float* sell_val = nullptr;
    if (malloc_async(&val, (N + kPad) * 4, st) != cudaSuccess ||
        malloc_async(&sell_val, (sell_cap + kPad) * 4, st) != cudaSuccess) {
      cudaGetLastError();
      if (val) cudaFreeAsync(val, st);
      set_error("fj_graph_update_weights: out of device memory for the weights");
      return FJ_ERR_OOM;
    }
    count_launches(3);
    k_fill_f32<<<grid_for(N, 256), 256, 0, st>>>(val, N, 1.0f);
    FJ_CUDA(cudaMemsetAsync(val + N, 0, kPad * 4, st));
    k_fill_f32<<<grid_for(sell_cap + kPad, 256), 256, 0, st>>>(sell_val, sell_cap + kPad, 0.0f);
    k_sell_unit_vals<<<grid_for(g->n_slices * 32, 256), 256, 0, st>>>(g->row_ptr, n, g->n_long, g->n_slices,
                                                                      g->slice_off, sell_val);
    FJ_CUDA(cudaGetLastError());
    g->val = val;
    g->sell_val = sell_val;
    g->weighted = 1;
  }
  count_launches(1);
  k_update_weights<<<grid_for(count * 32, 256), 256, 0, st>>>(count, n, src, dst, w, inv, g->row_ptr, g->col,
                                                               g->val, g->n_long, g->slice_off, g->sell_val,
                                                               true, err);
  // the preconditioner, as the build computes it
  const int64_t hc[2] = {g->n_long, g->n_nz};
  FJ_CUDA(cudaMemcpyAsync(dcnt, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
  float* cpart = pool.get<float>(std::max<int64_t>(g->n_chunks, 1));
  if (!cpart) {
    set_error("fj_graph_update_weights: out of device memory");
    return FJ_ERR_OOM;
  }
  count_launches(2);
  k_chunk_wsum<<<grid_for(std::max<int64_t>(g->n_chunks, 1) * 32, 256), 256, 0, st>>>(
      g->val, g->long_first, dcnt, g->chunk_begin, g->chunk_end, cpart);
  k_dinv_weighted<<<grid_for(n, 256), 256, 0, st>>>(g->row_ptr, n, dcnt, g->long_first, cpart, g->slice_off,
                                                    g->sell_val, g->dinv);
  FJ_CUDA(cudaGetLastError());
  FJ_CUDA(cudaStreamSynchronize(st));
  return FJ_OK;
}
