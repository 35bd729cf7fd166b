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

#include "fj_internal.cuh"

namespace fj {

constexpr unsigned kFull = 0xffffffffu;

// Per-warp shared staging for one tile.
struct TileSmem {
  int32_t re[kTileItems + 1];  // row_ptr[r0+1 .. r1+1]
  int32_t col[kTileItems];
  float val[kTileItems];
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
};

enum WalkMode { kRowSum = 0, kLap = 1 };

// Walks tiles [wg*tpw, (wg+1)*tpw) of the merge path.
//   kRowSum: out[r] = sum of row r's weights (K must be 1, x unused)
//   kLap:    out[r*K+c] = sum_j w_rj (x[r*K+c] - x[j*K+c]); returns this
//            lane's part of sum over entries of w (x_r - x_j)^2.
// Rows wholly inside the warp's run are final in out[]; the run's last row
// is published in wc_row[wg] / wc_val[wg*K + c] (carry of that row).
template <typename T, int K, int MODE>
__device__ __forceinline__ T walk_tiles(const WalkGraph& g, const T* __restrict__ x,
                                        T* __restrict__ out, int32_t* __restrict__ wc_row,
                                        T* __restrict__ wc_val, int64_t wg, TileSmem* sm) {
  constexpr int G = 32 / K;           // walkers per warp
  constexpr int IPW = kTileItems / G;  // items per walker per tile
  const int lane = threadIdx.x & 31;
  const int gw = lane / K;  // walker index
  const int c = lane % K;   // right-hand side handled by this lane
  const int64_t total = g.n + g.nnz;
  const int64_t t_begin = wg * g.tiles_per_warp;
  int64_t t_end = t_begin + g.tiles_per_warp;
  if (t_end > g.n_tiles) t_end = g.n_tiles;
  T quad = T(0);
  if (t_begin >= t_end) return quad;

  int32_t carry_row = g.tile_row[t_begin];
  T carry = T(0);
  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t d0 = t * kTileItems;
    int64_t d1 = d0 + kTileItems;
    if (d1 > total) d1 = total;
    const int64_t r0 = g.tile_row[t];
    const int64_t r1 = g.tile_row[t + 1];
    const int32_t k0 = (int32_t)(d0 - r0);
    const int32_t k1 = (int32_t)(d1 - r1);
    const int64_t rlast = (r1 < g.n - 1) ? r1 : (g.n - 1);
    const int nre = (int)(rlast - r0 + 1);
    const int nk = k1 - k0;
    __syncwarp();
    for (int j = lane; j < nre; j += 32) sm->re[j] = g.row_ptr[r0 + 1 + j];
    for (int j = lane; j < nk; j += 32) {
      sm->col[j] = g.col[k0 + j];
      if (g.val) sm->val[j] = g.val[k0 + j];
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
    int hi = (int)(r1 - r0);
    if (hi > dl) hi = dl;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((sm->re[mid - 1] - k0) + mid <= dl)
        lo = mid;
      else
        hi = mid - 1;
    }
    int64_t r = r0 + lo;
    int k = dl - lo;  // local nonzero index
    T xr = T(0);
    if (MODE == kLap && r < g.n) xr = x[r * K + c];
    T acc = T(0);
    bool femit = false;
    T fval = T(0);
    const int64_t frow = r;
    for (int it = dl; it < de; ++it) {
      const int rend = sm->re[r - r0] - k0;
      if (k < rend) {
        const float w = g.val ? sm->val[k] : 1.0f;
        if (MODE == kRowSum) {
          acc += T(w);
        } else {
          const int32_t j = sm->col[k];
          const T df = xr - x[(int64_t)j * K + c];
          const T tw = T(w) * df;
          acc += tw;
          quad += tw * df;
        }
        ++k;
      } else {
        if (!femit) {
          femit = true;
          fval = acc;
        } else {
          out[r * K + c] = acc;
        }
        acc = T(0);
        ++r;
        if (MODE == kLap && r < g.n) xr = x[r * K + c];
      }
    }
    int32_t crow = (int32_t)r;
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
      const T v = __shfl_up_sync(kFull, scan, off * K);
      const int32_t kr = __shfl_up_sync(kFull, crow, off * K);
      if (gw >= off && kr == crow) scan += v;
    }
    const T prev = __shfl_up_sync(kFull, scan, K);
    if (femit) out[frow * K + c] = fval + (gw > 0 ? prev : T(0));
    carry = __shfl_sync(kFull, scan, (G - 1) * K + c);
    carry_row = __shfl_sync(kFull, crow, (G - 1) * K + c);
  }
  if (lane == 0) wc_row[wg] = carry_row;
  if (lane < K) wc_val[wg * K + lane] = carry;
  return quad;
}

// Adds to `own` (the value written for row i by the warp holding its row
// end) the carries of the warps whose runs end inside row i, in warp order.
template <typename T, int K>
__device__ __forceinline__ T row_total(int64_t i, T own, const int32_t* __restrict__ row_ptr,
                                       const T* __restrict__ wc_val, int64_t tiles_per_warp,
                                       int c) {
  const int64_t a = i + row_ptr[i];
  const int64_t b = i + row_ptr[i + 1];
  const int64_t wa = (a / kTileItems) / tiles_per_warp;
  const int64_t wb = (b / kTileItems) / tiles_per_warp;
  for (int64_t w = wa; w < wb; ++w) own += wc_val[w * K + c];
  return own;
}

}  // namespace fj
