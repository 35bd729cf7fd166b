// fj_walk.cuh - load-balanced CSR row reductions ("walks") for libfj.
//
// The off-diagonal part of (I + L) x is t_i = sum_j w_ij (x_i - x_j), the
// incidence form L = sum_e w_e b_e b_e^T of Sec. 2.1 evaluated row by row.
// Power-law rows (hubs of 10^5..10^7 entries) make a row-per-thread or
// row-per-warp split badly unbalanced, so every reduction over CSR rows here
// walks the merge path of (row ends, nonzeros): the n + nnz path items are
// cut into tiles of kTileItems items, each warp owns a contiguous run of
// tiles, and inside a tile the items are split evenly between "walkers".
//
// A walker is K consecutive lanes handling K right-hand sides of one path
// segment (K = 1: 32 walkers of one lane; K = 32: one walker of 32 lanes, so
// every gathered row x_j is one coalesced 128-byte line).  Rows that cross
// walker, tile or warp boundaries are combined deterministically:
//   * walkers of one tile: a segmented shuffle scan keyed by row id;
//   * tiles of one warp: the running carry stays in registers;
//   * warps: each warp publishes its final carry; the consumer of row i adds
//     the carries of the warps that end inside row i, in warp order.
// The result is bit-reproducible for a fixed graph and launch shape.
#pragma once

#include <type_traits>

#include "fj_df64.cuh"
#include "fj_internal.cuh"

namespace fj {

constexpr unsigned kFull = 0xffffffffu;

// Per-warp shared staging for one tile.
struct TileSmem {
  int32_t re[kTileItems + 1];  // row_ptr[r0+1 .. r1+1]
  int32_t col[kTileItems];
  float val[kTileItems];
};

// Narrow right-hand sides (K * sizeof(T) <= 8) also stage the gathered
// neighbour values x_j and the row values x_r of the tile, so that all of a
// tile's gathers are in flight at once and the walk itself touches only
// shared memory.
template <typename T, int K>
struct StagesX {
  static constexpr bool value = K * sizeof(T) <= 8;
};

template <typename T, int K>
struct TileSmemX {
  int32_t re[kTileItems + 1];  // row_ptr[r0+1 .. r1+1]
  float val[kTileItems];
  T xj[kTileItems * K];        // x[col[k0 + j]]
  T xr[(kTileItems + 1) * K];  // x[r0 + j]
};

template <typename T, int K>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return StagesX<T, K>::value ? sizeof(TileSmemX<T, K>) : sizeof(TileSmem);
}

// Unsigned 32-bit division by a run-time invariant d >= 1 with one multiply
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Sec. 4): q = (t + ((a - t) >> 1)) >> (l - 1),
// t = umulhi(m, a), l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
  uint32_t d, m, s;  // s = l - 1 (d >= 2); d == 1 is handled apart
  __host__ void init(uint32_t div) {
    d = div;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < div) ++l;
    m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - div)) / div + 1);
    s = l ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t a) const {
    if (d == 1) return a;
    const uint32_t t = __umulhi(m, a);
    return (t + ((a - t) >> 1)) >> s;
  }
};

struct WalkGraph {
  const int32_t* row_ptr;
  const int32_t* col;
  const float* val;  // nullptr: unit weights
  const int32_t* tile_row;
  int64_t n;
  int64_t nnz;
  int64_t n_tiles;
  int64_t tiles_per_warp;
  FastDiv items_per_warp;  // kTileItems * tiles_per_warp (n + nnz < 2^32)
};

inline void set_tiles_per_warp(WalkGraph& g, int64_t tpw) {
  g.tiles_per_warp = tpw;
  g.items_per_warp.init((uint32_t)(tpw * kTileItems));
}

enum WalkMode { kRowSum = 0, kLap = 1 };

// Asynchronous 4/8-byte copies global -> shared (no registers held while
// in flight); cp.async.wait_all makes the executing thread's copies visible.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Wide walks (K >= 8) prefetch the x rows of the next kPrefetch<T> nonzeros
// of each walker into this much shared memory per warp.
constexpr int kGatherBytesPerWarp = 4096;
template <typename T>
struct Prefetch {
  static constexpr int value = kGatherBytesPerWarp / (32 * (int)sizeof(T));  // nonzeros per walker
};

// Walks tiles [wg*tpw, (wg+1)*tpw) of the merge path.
//   kRowSum: out[r] = sum of row r's weights (K must be 1, x unused)
//   kLap:    out[r*K+c] = sum_j w_rj (x[r*K+c] - x[j*K+c]); returns this
//            lane's part of sum over entries of w (x_r - x_j)^2.
// Rows wholly inside the warp's run are final in out[]; the run's last row
// is published in wc_row[wg] / wc_val[wg*K + c] (carry of that row).
template <typename T, int K, int MODE>
__device__ __forceinline__ T walk_tiles(const WalkGraph& g, const T* __restrict__ x,
                                        T* __restrict__ out, int32_t* __restrict__ wc_row,
                                        T* __restrict__ wc_val, int64_t wg, void* smem,
                                        T* __restrict__ gbuf = nullptr) {
  constexpr bool kStageX = (MODE == kLap) && StagesX<T, K>::value;
  // wide walks: x rows of upcoming nonzeros prefetched into gbuf (per walker)
  constexpr bool kPre = (MODE == kLap) && !kStageX && K >= 8;
  constexpr int PD = Prefetch<T>::value;
  TileSmem* sm = reinterpret_cast<TileSmem*>(smem);
  TileSmemX<T, K>* smx = reinterpret_cast<TileSmemX<T, K>*>(smem);
  int32_t* s_re = kStageX ? smx->re : sm->re;
  float* s_val = kStageX ? smx->val : sm->val;
  constexpr int G = 32 / K;           // walkers per warp
  constexpr int IPW = kTileItems / G;  // items per walker per tile
  const int lane = threadIdx.x & 31;
  const int gw = lane / K;  // walker index
  const int c = lane % K;   // right-hand side handled by this lane
  const int64_t total = g.n + g.nnz;
  const int64_t t_begin = wg * g.tiles_per_warp;
  int64_t t_end = t_begin + g.tiles_per_warp;
  if (t_end > g.n_tiles) t_end = g.n_tiles;
  T quad = num<T>(0.f);
  if (t_begin >= t_end) return quad;

  // tile row coordinates of 32 tiles at a time live in one register per lane
  int32_t trow = g.tile_row[t_begin + (lane < t_end - t_begin + 1 ? lane : 0)];
  int64_t tbase = t_begin;
  int32_t carry_row = __shfl_sync(kFull, trow, 0);
  T carry = num<T>(0.f);
  for (int64_t t = t_begin; t < t_end; ++t) {
    if (t + 1 - tbase >= 32) {  // refill the coordinate window
      tbase = t;
      const int64_t q = t + lane;
      trow = g.tile_row[q <= t_end ? q : t_end];
    }
    const int32_t r0 = __shfl_sync(kFull, trow, (int)(t - tbase));
    const int32_t r1 = __shfl_sync(kFull, trow, (int)(t + 1 - tbase));
    const int64_t d0 = t * kTileItems;
    int64_t d1 = d0 + kTileItems;
    if (d1 > total) d1 = total;
    const int32_t k0 = (int32_t)(d0 - r0);
    const int32_t k1 = (int32_t)(d1 - r1);
    const int32_t rlast = (r1 < g.n - 1) ? r1 : (int32_t)(g.n - 1);
    const int nre = rlast - r0 + 1;
    const int nk = k1 - k0;
    __syncwarp();
    // Staging in two waves, each issuing all of its global loads before any
    // shared-memory store (a store between loads would serialise them):
    // wave 1 row ends, columns and weights; wave 2 the gathers x[col], x[r].
    constexpr int kPer = (kTileItems + 31) / 32;
    int32_t cj[kPer];
    {
      int32_t rev[kPer + 1];
      float wv[kPer];
#pragma unroll
      for (int u = 0; u <= kPer; ++u) {
        const int j = lane + 32 * u;
        rev[u] = (j < nre) ? g.row_ptr[r0 + 1 + j] : 0;
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = lane + 32 * u;
        cj[u] = (j < nk) ? g.col[k0 + j] : 0;
        wv[u] = (g.val && j < nk) ? g.val[k0 + j] : 1.0f;
      }
#pragma unroll
      for (int u = 0; u <= kPer; ++u) {
        const int j = lane + 32 * u;
        if (j < nre) s_re[j] = rev[u];
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = lane + 32 * u;
        if (j < nk) {
          s_val[j] = wv[u];
          if (!kStageX) sm->col[j] = cj[u];
        }
      }
    }
    if (kStageX) {
      T xg[kPer][K];
      T xrv[kPer + 1];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = lane + 32 * u;
#pragma unroll
        for (int cc = 0; cc < K; ++cc) xg[u][cc] = (j < nk) ? x[(int64_t)cj[u] * K + cc] : num<T>(0.f);
      }
      // x of the tile's rows: nre * K consecutive values
#pragma unroll
      for (int u = 0; u <= kPer; ++u) {
        const int e = lane + 32 * u;
        xrv[u] = (e < nre * K) ? x[(int64_t)r0 * K + e] : num<T>(0.f);
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = lane + 32 * u;
        if (j < nk) {
#pragma unroll
          for (int cc = 0; cc < K; ++cc) smx->xj[j * K + cc] = xg[u][cc];
        }
      }
#pragma unroll
      for (int u = 0; u <= kPer; ++u) {
        const int e = lane + 32 * u;
        if (e < nre * K) smx->xr[e] = xrv[u];
      }
      // rows beyond 32 * (kPer + 1) / K of a tile (only when K > 1)
      for (int e = lane + 32 * (kPer + 1); e < nre * K; e += 32) smx->xr[e] = x[(int64_t)r0 * K + e];
    }
    __syncwarp();

    const int len = (int)(d1 - d0);
    int dl = gw * IPW;
    if (dl > len) dl = len;
    int de = dl + IPW;
    if (de > len) de = len;
    // merge-path split of local diagonal dl inside the tile
    int lo = dl - nk;
    if (lo < 0) lo = 0;
    int hi = r1 - r0;
    if (hi > dl) hi = dl;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((s_re[mid - 1] - k0) + mid <= dl)
        lo = mid;
      else
        hi = mid - 1;
    }
    int rl = lo;       // local row
    int k = dl - lo;   // local nonzero index
    T xr = num<T>(0.f);
    T xr_nx = num<T>(0.f);  // wide walks: x of the next row, loaded one row ahead
    if (MODE == kLap && r0 + rl < g.n)
      xr = kStageX ? smx->xr[rl * K + c] : x[(int64_t)(r0 + rl) * K + c];
    if (kPre && r0 + rl + 1 < g.n) xr_nx = x[(int64_t)(r0 + rl + 1) * K + c];
    T acc = num<T>(0.f);
    bool femit = false;
    T fval = num<T>(0.f);
    const int frl = rl;
    // Two halves of PD/2 nonzeros: one being read, the next one in flight.
    constexpr int HB = PD / 2;
    int cbase = -1;  // local index of the first nonzero of the half being read
    int cur = 0;     // which half is being read
    T* wbuf = gbuf + gw * PD * K;
    auto issue_half = [&](int base, int half) {
#pragma unroll 4
      for (int i = 0; i < HB; ++i) {
        if (base + i < nk) {
          const T* src = x + (int64_t)sm->col[base + i] * K + c;
          if constexpr (sizeof(T) == 4)
            cp_async4(&wbuf[(half * HB + i) * K + c], src);
          else
            cp_async8(&wbuf[(half * HB + i) * K + c], src);
        }
      }
      cp_async_commit_group();
    };
    for (int it = dl; it < de; ++it) {
      const int rend = s_re[rl] - k0;
      if (k < rend) {
        const float w = g.val ? s_val[k] : 1.0f;
        if (MODE == kRowSum) {
          acc += num<T>(w);
        } else {
          if (kPre) {  // walker-uniform; each lane reads and copies only its own column
            if (cbase < 0) {
              cbase = k;
              cur = 0;
              issue_half(k, 0);
              issue_half(k + HB, 1);
              cp_async_wait_one();
            } else if (k >= cbase + HB) {
              cbase += HB;
              cur ^= 1;
              issue_half(cbase + HB, cur ^ 1);
              cp_async_wait_one();
            }
          }
          const T xj = kStageX ? smx->xj[k * K + c]
                               : (kPre ? wbuf[(cur * HB + (k - cbase)) * K + c] : x[(int64_t)sm->col[k] * K + c]);
          const T df = xr - xj;
          const T tw = mul_w(df, w);
          acc += tw;
          quad += tw * df;
        }
        ++k;
      } else {
        if (!femit) {
          femit = true;
          fval = acc;
        } else {
          out[(int64_t)(r0 + rl) * K + c] = acc;
        }
        acc = num<T>(0.f);
        ++rl;
        if (kPre) {
          xr = xr_nx;
          if (r0 + rl + 1 < g.n) xr_nx = x[(int64_t)(r0 + rl + 1) * K + c];
        } else if (MODE == kLap && r0 + rl < g.n) {
          xr = kStageX ? smx->xr[rl * K + c] : x[(int64_t)(r0 + rl) * K + c];
        }
      }
    }
    if (kPre && cbase >= 0) cp_async_wait_all();  // the buffer is reused by the next tile
    int32_t crow = r0 + rl;
    T cval = acc;
    if (gw == 0) {
      if (femit)
        fval += carry;
      else
        cval += carry;
    }
    T scan = cval;
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
      const T v = shfl_up_v(scan, off * K);
      const int32_t kr = __shfl_up_sync(kFull, crow, off * K);
      if (gw >= off && kr == crow) scan += v;
    }
    const T prev = shfl_up_v(scan, K);
    if (femit) out[(int64_t)(r0 + frl) * K + c] = fval + (gw > 0 ? prev : num<T>(0.f));
    carry = shfl_v(scan, (G - 1) * K + c);
    carry_row = __shfl_sync(kFull, crow, (G - 1) * K + c);
  }
  if (lane == 0) wc_row[wg] = carry_row;
  if (lane < K) wc_val[wg * K + lane] = carry;
  return quad;
}

// ------------------------------------------------------------ sliced ELL
//
// Narrow right-hand sides (K <= 4) use the sliced-ELL layout: each lane owns
// one row of a 32-row slice and walks it entry by entry, so every load of
// col/val is one coalesced 128-byte line, the K values of x_j come in one
// vector load, and a row's sum is accumulated by one lane in entry order.
// Long rows are cut into chunks processed by a whole warp (lanes stride over
// the chunk, then a fixed xor-tree reduction).  A row with several chunks is
// finished by the warp that completes its last chunk: chunk sums go to
// part[], a per-row counter counts finished chunks, and the last finisher
// adds the row's chunk sums in chunk order.  Every row sum is therefore the
// same bits whichever warp computes which unit.

struct SellGraph {
  const int32_t* row_ptr;  // solver-order CSR (long rows)
  const int32_t* col;
  const float* val;
  const int32_t* long_first;
  const int32_t* chunk_row;
  const int32_t* chunk_begin;
  const int32_t* chunk_end;
  const int64_t* slice_off;
  const int32_t* sell_col;
  const float* sell_val;
  const int64_t* unit_prefix;
  int64_t n;
  int64_t n_long;
  int64_t n_nz;  // rows [n_nz, n) have no entries: their sums are 0
  int64_t n_chunks;
  int64_t n_slices;
  int64_t n_units;
};

template <typename T, int K>
__device__ __forceinline__ void load_k(const T* __restrict__ p, T (&v)[K]) {
  if constexpr (std::is_same<T, df64>::value) {
    if constexpr (K % 2 == 0) {
#pragma unroll
      for (int cc = 0; cc < K; cc += 2) {
        const float4 q = reinterpret_cast<const float4*>(p)[cc / 2];
        v[cc] = df_make(q.x, q.y);
        v[cc + 1] = df_make(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int cc = 0; cc < K; ++cc) {
        const float2 q = reinterpret_cast<const float2*>(p)[cc];
        v[cc] = df_make(q.x, q.y);
      }
    }
  } else if constexpr (K * sizeof(T) == 16 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (K * sizeof(T) == 16 && sizeof(T) == 8) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else if constexpr (K * sizeof(T) == 8 && sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
#pragma unroll
    for (int cc = 0; cc < K; ++cc) v[cc] = p[cc];
  }
}

// First work unit of warp w of W when units are split by cumulative cost.
__device__ __forceinline__ int64_t sell_unit_start(const SellGraph& g, int64_t w, int64_t W) {
  const int64_t total = g.unit_prefix[g.n_units];
  const int64_t target = (w * total + W - 1) / W;  // ceil(w * total / W)
  int64_t lo = 0, hi = g.n_units;  // first u with prefix[u] >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (g.unit_prefix[mid] < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// out[r*K+c] = sum_j w_rj (x[r*K+c] - x[j*K+c]) for every row of units
// [u0, u1); quad[c] accumulates this lane's share of sum w (x_r - x_j)^2.
template <typename T, int K>
__device__ __forceinline__ void sell_walk(const SellGraph& g, const T* __restrict__ x, T* __restrict__ out,
                                          T* __restrict__ part, int* __restrict__ cnt, int64_t u0,
                                          int64_t u1, T (&quad)[K]) {
  const int lane = threadIdx.x & 31;
  // entries in flight per lane between two dependent round trips
  constexpr int kB = (K * sizeof(T) <= 4) ? 8 : 4;
  for (int64_t u = u0; u < u1; ++u) {
    if (u < g.n_chunks) {
      const int32_t r = g.chunk_row[u];
      const int32_t b = g.chunk_begin[u], e = g.chunk_end[u];
      T xr[K], acc[K];
      load_k<T, K>(x + (int64_t)r * K, xr);
#pragma unroll
      for (int cc = 0; cc < K; ++cc) acc[cc] = num<T>(0.f);
      // batches of kB entries per lane: all index loads, then all gathers
      for (int32_t p0 = b; p0 < e; p0 += 32 * kB) {
        int32_t j[kB];
        float w[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) {
          const int32_t p = p0 + 32 * q + lane;
          j[q] = p < e ? g.col[p] : r;
          w[q] = (p < e && g.val) ? g.val[p] : (p < e ? 1.0f : 0.0f);
        }
        T xj[kB][K];
#pragma unroll
        for (int q = 0; q < kB; ++q) load_k<T, K>(x + (int64_t)j[q] * K, xj[q]);
#pragma unroll
        for (int q = 0; q < kB; ++q) {
#pragma unroll
          for (int cc = 0; cc < K; ++cc) {
            const T df = xr[cc] - xj[q][cc];
            const T tw = mul_w(df, w[q]);
            acc[cc] += tw;
            quad[cc] += tw * df;
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < K; ++cc) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[cc] += shfl_xor_v(acc[cc], off);
      }
      T mine = acc[0];
#pragma unroll
      for (int cc = 1; cc < K; ++cc)
        if (lane == cc) mine = acc[cc];
      const int32_t f = g.long_first[r];
      const int32_t nch = g.long_first[r + 1] - f;
      if (nch == 1) {
        if (lane < K) out[(int64_t)r * K + lane] = mine;
      } else {
        if (lane < K) {
          part[u * K + lane] = mine;
          __threadfence();
        }
        __syncwarp();
        int done = 0;
        if (lane == 0) done = atomicAdd(&cnt[r], 1) == nch - 1;
        done = __shfl_sync(kFull, done, 0);
        if (done) {
          __threadfence();
          T tot[K];
#pragma unroll
          for (int cc = 0; cc < K; ++cc) tot[cc] = num<T>(0.f);
          for (int32_t q = f + lane; q < f + nch; q += 32) {
#pragma unroll
            for (int cc = 0; cc < K; ++cc) tot[cc] += ldcg_v(&part[(int64_t)q * K + cc]);
          }
#pragma unroll
          for (int cc = 0; cc < K; ++cc) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) tot[cc] += shfl_xor_v(tot[cc], off);
          }
          T t = tot[0];
#pragma unroll
          for (int cc = 1; cc < K; ++cc)
            if (lane == cc) t = tot[cc];
          if (lane < K) out[(int64_t)r * K + lane] = t;
          if (lane == 0) cnt[r] = 0;
        }
      }
    } else {
      const int64_t s = u - g.n_chunks;
      const int64_t off = g.slice_off[s];
      const int32_t len = (int32_t)((g.slice_off[s + 1] - off) >> 5);
      const int64_t row = g.n_long + 32 * s + lane;
      if (row < g.n) {
        T xr[K], acc[K];
        load_k<T, K>(x + row * K, xr);
#pragma unroll
        for (int cc = 0; cc < K; ++cc) acc[cc] = num<T>(0.f);
        const int32_t* __restrict__ cp = g.sell_col + off + lane;
        const float* __restrict__ vp = g.sell_val ? g.sell_val + off + lane : nullptr;
        // batches of kB entries: all index loads, then all gathers
        for (int32_t p0 = 0; p0 < len; p0 += kB) {
          int32_t j[kB];
          float w[kB];
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            const bool in = p0 + q < len;
            j[q] = in ? cp[32 * (p0 + q)] : (int32_t)row;
            w[q] = in ? (vp ? vp[32 * (p0 + q)] : 1.0f) : 0.0f;
          }
          T xj[kB][K];
#pragma unroll
          for (int q = 0; q < kB; ++q) load_k<T, K>(x + (int64_t)j[q] * K, xj[q]);
#pragma unroll
          for (int q = 0; q < kB; ++q) {
#pragma unroll
            for (int cc = 0; cc < K; ++cc) {
              const T df = xr[cc] - xj[q][cc];
              const T tw = mul_w(df, w[q]);
              acc[cc] += tw;
              quad[cc] += tw * df;
            }
          }
        }
#pragma unroll
        for (int cc = 0; cc < K; ++cc) out[row * K + cc] = acc[cc];
      }
    }
  }
}

// ----------------------------------------------------- wide (K >= 8)
//
// 8, 16 or 32 right-hand sides: lanes hold columns.  A warp is SUB = 32/K
// sub-groups of K lanes; every gathered row x_j is one K-wide coalesced load.
// Work units are the same as for narrow K (long-row chunks, 32-row slices):
//   chunk: the sub-groups stride over the chunk's entries, kWB entries per
//          sub-group in flight, then an xor tree across sub-groups; chunks
//          of one row are finished as in chunk_walk;
//   slice: sub-group sg owns the RB = 32/SUB consecutive rows
//          [rs + sg*RB, rs + (sg+1)*RB); their entries are one contiguous run
//          of the CSR, summed in batches of kWB entries that run across row
//          ends.  The rows' end offsets sit in lane registers (one shuffle per
//          row end) and their x values are staged in shared memory first.
constexpr int kWB = 8;

template <typename T, int K>
__device__ __forceinline__ void wide_unit(const SellGraph& g, const T* __restrict__ x, T* __restrict__ out,
                                          T* __restrict__ part, int* __restrict__ cnt, int64_t u, T& quad,
                                          T* __restrict__ sxr) {
  constexpr int SUB = 32 / K;
  constexpr int RB = 32 / SUB;  // rows per sub-group in a slice
  const int lane = threadIdx.x & 31;
  const int sg = lane / K, c = lane % K;
  const unsigned smask = (K == 32) ? kFull : (((1u << K) - 1u) << (sg * K));
  if (u < g.n_chunks) {
    const int32_t r = g.chunk_row[u];
    const int32_t b = g.chunk_begin[u], e = g.chunk_end[u];
    const T xr = x[(int64_t)r * K + c];
    T acc = num<T>(0.f);
    for (int32_t p0 = b + sg; p0 < e; p0 += SUB * kWB) {
      int32_t j[kWB];
      float w[kWB];
#pragma unroll
      for (int t = 0; t < kWB; ++t) {
        const int32_t p = p0 + t * SUB;
        const bool in = p < e;
        j[t] = in ? g.col[p] : r;
        w[t] = in ? (g.val ? g.val[p] : 1.0f) : 0.0f;
      }
      T xj[kWB];
#pragma unroll
      for (int t = 0; t < kWB; ++t) xj[t] = x[(int64_t)j[t] * K + c];
#pragma unroll
      for (int t = 0; t < kWB; ++t) {
        const T df = xr - xj[t];
        const T tw = mul_w(df, w[t]);
        acc += tw;
        quad += tw * df;
      }
    }
#pragma unroll
    for (int off = K; off < 32; off <<= 1) acc += shfl_xor_v(acc, off);
    const int32_t f = g.long_first[r];
    const int32_t nch = g.long_first[r + 1] - f;
    if (nch == 1) {
      if (sg == 0) out[(int64_t)r * K + c] = acc;
      return;
    }
    if (sg == 0) {
      part[u * K + c] = acc;
      __threadfence();
    }
    __syncwarp();
    int done = 0;
    if (lane == 0) done = atomicAdd(&cnt[r], 1) == nch - 1;
    done = __shfl_sync(kFull, done, 0);
    if (!done) return;
    __threadfence();
    T tot = num<T>(0.f);
    for (int32_t q = f + sg; q < f + nch; q += SUB) tot += ldcg_v(&part[(int64_t)q * K + c]);
#pragma unroll
    for (int off = K; off < 32; off <<= 1) tot += shfl_xor_v(tot, off);
    if (sg == 0) out[(int64_t)r * K + c] = tot;
    if (lane == 0) cnt[r] = 0;
    return;
  }
  // slice: rows [ra, rb) of this sub-group; row i of the slice is owned by
  // sub-group i / RB, whose lanes are [i / RB * K, ...) = the lanes that
  // hold the row ends of its rows (RB == K).
  constexpr bool kStageXr = 32 * K * (int)sizeof(T) <= kGatherBytesPerWarp;
  const int64_t s = u - g.n_chunks;
  const int64_t rs = g.n_long + 32 * s;
  const int64_t ra = rs + (int64_t)sg * RB;
  int64_t rb = ra + RB;
  if (rb > g.n_nz) rb = g.n_nz;
  // lane l of the warp holds row_ptr[rs + l + 1], the end of row rs + l
  const int64_t rr = rs + lane;
  const int32_t rend_l = (rr < g.n_nz) ? g.row_ptr[rr + 1] : 0;
  if (kStageXr) {  // x of the slice's 32 rows: row i at sxr[i*K + c]
    __syncwarp();
    for (int i = sg; i < 32; i += SUB) {
      const int64_t row = rs + i;
      sxr[i * K + c] = (row < g.n) ? x[row * K + c] : num<T>(0.f);
    }
    __syncwarp();
  }
  const int il = (int)((ra < rb ? ra : rs) - rs);
  const int ie = (int)((ra < rb ? rb - 1 : rs) - rs);
  int32_t cend = __shfl_sync(kFull, rend_l, il);
  const int32_t pend = __shfl_sync(kFull, rend_l, ie);
  if (ra >= rb) return;
  int32_t p = g.row_ptr[ra];
  int64_t cur = ra;  // current row
  T xr = kStageXr ? sxr[(cur - rs) * K + c] : x[cur * K + c];
  T acc = num<T>(0.f);
  while (true) {
    // rows without entries end at once
    while (cur < rb && p >= cend) {
      out[cur * K + c] = acc;
      acc = num<T>(0.f);
      ++cur;
      if (cur < rb) {
        cend = __shfl_sync(smask, rend_l, (int)(cur - rs));
        xr = kStageXr ? sxr[(cur - rs) * K + c] : x[cur * K + c];
      }
    }
    if (cur >= rb) break;
    int32_t j[kWB];
    float w[kWB];
#pragma unroll
    for (int t = 0; t < kWB; ++t) {
      const bool in = p + t < pend;
      j[t] = in ? g.col[p + t] : 0;
      w[t] = in ? (g.val ? g.val[p + t] : 1.0f) : 0.0f;
    }
    T xj[kWB];
#pragma unroll
    for (int t = 0; t < kWB; ++t) xj[t] = x[(int64_t)j[t] * K + c];
#pragma unroll
    for (int t = 0; t < kWB; ++t) {
      if (p < pend) {
        while (p >= cend) {  // row end inside the batch
          out[cur * K + c] = acc;
          acc = num<T>(0.f);
          ++cur;
          cend = __shfl_sync(smask, rend_l, (int)(cur - rs));
          xr = kStageXr ? sxr[(cur - rs) * K + c] : x[cur * K + c];
        }
        const T df = xr - xj[t];
        const T tw = mul_w(df, w[t]);
        acc += tw;
        quad += tw * df;
        ++p;
      }
    }
  }
}

// Adds to `own` (the value written for row i by the warp holding its row
// end) the carries of the warps whose runs end inside row i, in warp order.
template <typename T, int K>
__device__ __forceinline__ T row_total(int64_t i, T own, const int32_t* __restrict__ row_ptr,
                                       const T* __restrict__ wc_val, const FastDiv& ipw, int c) {
  const uint32_t a = (uint32_t)i + (uint32_t)row_ptr[i];
  const uint32_t b = (uint32_t)i + (uint32_t)row_ptr[i + 1];
  const uint32_t wa = ipw.div(a);
  const uint32_t wb = ipw.div(b);
  for (uint32_t w = wa; w < wb; ++w) own += wc_val[(int64_t)w * K + c];
  return own;
}

}  // namespace fj
