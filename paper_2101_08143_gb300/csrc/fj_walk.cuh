// fj_walk.cuh - CSR row reductions ("walks") for libfj.
//
// The off-diagonal part of (I + L) x is t_i = sum_j w_ij (x_i - x_j), the
// incidence form L = sum_e w_e b_e b_e^T of Sec. 2.1 evaluated row by row,
// and the walks also return sum over CSR entries of w_ij (x_i - x_j)^2
// (= 2 x^T L x).  Nodes are in degree-descending order; rows of more than
// kSellMaxLen entries are cut into chunks of at most kChunkLen entries, the
// rest form 32-row slices.  Chunks, then slices, are the work units:
//   K <= 4 columns  sliced ELL, one lane per row (sell_walk);
//   K >= 8 columns  lanes as columns, each gathered row x_j one K-wide
//                   coalesced load (wide_unit).
// Every row sum is accumulated in entry order by one lane or combined in a
// fixed order, so results are bit-reproducible.
#pragma once

#include "fj_df64.cuh"
#include "fj_internal.cuh"

namespace fj {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------ sliced ELL
//
// Narrow right-hand sides (K <= 4) use the sliced-ELL layout: each lane owns
// one row of a 32-row slice and walks it entry by entry, so every load of
// col/val is one coalesced 128-byte line, the K values of x_j come in one
// vector load, and a row's sum is accumulated by one lane in entry order.
// Long rows are cut into chunks processed by a whole warp (lanes stride over
// the chunk, then a fixed xor-tree reduction).  A row of one chunk is
// written directly; a row of several chunks leaves one partial sum per chunk
// in part[], and the phase after the walk's barrier adds them in chunk order
// (row_t).  Every row sum is therefore the same bits whichever warp computes
// which unit, with no fence or atomic inside the walk.

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

// Streaming store of a walk's row sum (read once, by the next phase).
__device__ __forceinline__ void st_row(float* p, float v) { st_cs(p, v); }
__device__ __forceinline__ void st_row(double* p, double v) { st_cs(p, v); }
__device__ __forceinline__ void st_row(df64* p, df64 v) { st_cs(reinterpret_cast<float2*>(p), make_float2(v.hi, v.lo)); }

// First work unit of range w of W when units are split by cumulative cost:
// the unit boundary nearest to w/W of the total (monotone in w, 0 for w = 0,
// n_units for w = W).
__device__ __forceinline__ int64_t sell_unit_start(const SellGraph& g, int64_t w, int64_t W) {
  const int64_t total = g.unit_prefix[g.n_units];
  const int64_t target = (w * total + W / 2) / W;  // round(w * total / W)
  int64_t lo = 0, hi = g.n_units;  // first u with prefix[u] >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (g.unit_prefix[mid] < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo > 0 && target - g.unit_prefix[lo - 1] < g.unit_prefix[lo] - target) --lo;
  return lo;
}

// out[r*K+c] = sum_j w_rj (x[r*K+c] - x[j*K+c]) for every row of units
// [u0, u1); quad[c] accumulates this lane's share of sum w (x_r - x_j)^2.
// The graph and the row sums are streamed (evict-first) and the gathers of x
// are plain loads, so that x stays in L2 while the graph streams past it.
template <typename T, int K, int kB>
__device__ __forceinline__ void sell_walk(const SellGraph& g, const T* __restrict__ x, T* __restrict__ out,
                                          T* __restrict__ part, int64_t u0,
                                          int64_t u1, T (&quad)[K]) {
  const int lane = threadIdx.x & 31;
  // kB: entries in flight per lane between two dependent round trips
  // bounds of unit u: a chunk's row and entry range, or a slice's offsets;
  // those of the next unit are loaded while the current one runs
  auto bounds = [&](int64_t u, int32_t& r, int64_t& lo, int64_t& hi) {
    if (u < g.n_chunks) {
      r = g.chunk_row[u];
      lo = g.chunk_begin[u];
      hi = g.chunk_end[u];
    } else {
      const int64_t s = u - g.n_chunks;
      r = 0;
      lo = g.slice_off[s];
      hi = g.slice_off[s + 1];
    }
  };
  int32_t r_next = 0;
  int64_t lo_next = 0, hi_next = 0;
  if (u0 < u1) bounds(u0, r_next, lo_next, hi_next);
  for (int64_t u = u0; u < u1; ++u) {
    const int32_t r_cur = r_next;
    const int64_t lo_cur = lo_next, hi_cur = hi_next;
    if (u + 1 < u1) bounds(u + 1, r_next, lo_next, hi_next);
    if (u < g.n_chunks) {
      const int32_t r = r_cur;
      const int32_t b = (int32_t)lo_cur, e = (int32_t)hi_cur;
      const int32_t nch = g.long_first[r + 1] - g.long_first[r];
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
          j[q] = p < e ? ld_ro(g.col + p) : r;
          w[q] = (p < e && g.val) ? ld_ro(g.val + p) : (p < e ? 1.0f : 0.0f);
        }
        T xj[kB][K];
#pragma unroll
        for (int q = 0; q < kB; ++q)
          load_k<T, K>(x + (int64_t)j[q] * K, xj[q]);
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
      // a row of one chunk is final; chunks of longer rows leave partial
      // sums, which the next phase adds up in chunk order (row_t)
      if (lane < K) (nch == 1 ? out[(int64_t)r * K + lane] : part[u * K + lane]) = mine;
    } else {
      const int64_t s = u - g.n_chunks;
      const int64_t off = lo_cur;
      const int32_t len = (int32_t)((hi_cur - off) >> 5);
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
            j[q] = in ? ld_ro(cp + 32 * (p0 + q)) : (int32_t)row;
            w[q] = in ? (vp ? ld_ro(vp + 32 * (p0 + q)) : 1.0f) : 0.0f;
          }
          T xj[kB][K];
#pragma unroll
          for (int q = 0; q < kB; ++q)
            load_k<T, K>(x + (int64_t)j[q] * K, xj[q]);
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
        for (int cc = 0; cc < K; ++cc) st_row(out + row * K + cc, acc[cc]);
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
//          sub-group in flight, then an xor tree across sub-groups; chunk
//          partials of multi-chunk rows are left for row_t, as for narrow K;
//   slice: sub-group sg owns the RB = 32/SUB consecutive rows
//          [rs + sg*RB, rs + (sg+1)*RB); their entries are one contiguous run
//          of the CSR, summed in batches of kWB entries that run across row
//          ends.  The rows' end offsets sit in lane registers (one shuffle per
//          row end) and their x values are staged in shared memory first.
constexpr int kWB = 8;

// Shared memory per warp for the slice rows' own values x_r (32 rows of K
// values, when they fit).
constexpr int kWideStageBytes = 4096;

template <typename T, int K>
__device__ __forceinline__ void wide_unit(const SellGraph& g, const T* __restrict__ x, T* __restrict__ out,
                                          T* __restrict__ part, int64_t u, T& quad,
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
      for (int t = 0; t < kWB; ++t)
        xj[t] = x[(int64_t)j[t] * K + c];
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
    const int32_t nch = g.long_first[r + 1] - g.long_first[r];
    if (sg == 0) (nch == 1 ? out[(int64_t)r * K + c] : part[u * K + c]) = acc;
    return;
  }
  // slice: rows [ra, rb) of this sub-group; row i of the slice is owned by
  // sub-group i / RB, whose lanes are [i / RB * K, ...) = the lanes that
  // hold the row ends of its rows (RB == K).
  constexpr bool kStageXr = 32 * K * (int)sizeof(T) <= kWideStageBytes;
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
    for (int t = 0; t < kWB; ++t)
      xj[t] = x[(int64_t)j[t] * K + c];
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

// Row i of the walk's output: out[i*K+c] as written by the walk, or for a
// row of several chunks the sum of its chunk partials in chunk order, or 0
// for a row without entries.  Valid after the barrier that ends the walk.
template <typename T, int K>
__device__ __forceinline__ T row_t(const SellGraph& g, const T* __restrict__ out, const T* __restrict__ part,
                                   int64_t i, int64_t idx, int c) {
  if (i >= g.n_nz) return num<T>(0.f);
  if (i < g.n_long) {
    const int32_t f = g.long_first[i], l = g.long_first[i + 1];
    if (l - f > 1) {
      T s = part[(int64_t)f * K + c];
      for (int32_t q = f + 1; q < l; ++q) s += part[(int64_t)q * K + c];
      return s;
    }
  }
  return out[idx];
}

}  // namespace fj
