// fj_solve.cu - persistent Jacobi-PCG solve of (I + L) q = s_bar and the five
// FJ quantities (Eq. FJmodel02, Sec. 3.2, Algorithm 1).
//
// One cooperative launch runs the whole solve for K right-hand sides:
//
//   setup     mu = 1^T s / n, s_bar = s - mu 1               (Alg. 1, step 2)
//             and a power of two 2^-e per column with max |s_bar| 2^-e in
//             [1, 2): the system is linear, so the solve runs on the scaled
//             s_bar exactly and q, z and the quantities are scaled back
//   refine    repeat: r64 = s_bar - (I+L) q        (float64 residual walk)
//               inner Jacobi-PCG on (I+L) e = r64 in the inner precision,
//               q += e                                 (iterative refinement)
//   output    z = q + mu 1 (Omega 1 = 1, Sec. 2.2), and from the last
//             residual pass: P = ||q||^2, C = ||q + mu 1||^2
//             = P + 2 mu 1^T q + n mu^2, C_I = ||s_bar - q||^2,
//             D = 1/2 sum_CSR w (q_i - q_j)^2 (= ||W^1/2 B q||^2,
//             Lemma PropA), I_dc = D + C.
//
// The refinement ("float64") arithmetic is double-float for float32 inner
// iterations and plain float64 for float64 inner iterations.
//
// The inner solver is the Chronopoulos-Gear form of preconditioned CG: both
// inner products of an iteration come out of one grid-wide reduction, so an
// iteration costs two grid barriers (vector update | SpMV walk; a third for
// the 8-32 column walks, whose work-unit sums are added after the walk).  The
// SpMV reduction (w, u) is taken as u^T u + 1/2 sum_CSR w (u_i - u_j)^2,
// which the walks produce without waiting for split rows to be combined.
//
// All reductions are two-level and in a fixed order (per block, then over
// blocks), and every block evaluates the same scalars, so control flow is
// identical in all blocks and results are bit-reproducible.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "fj_internal.cuh"
#include "fj_walk.cuh"

namespace fj {

constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxBlocksPerSM = 4;
constexpr int kMaxDevices = 64;

enum Slot {
  S_SUM = 0,  // column sums of s
  S_MAX,      // max s (max-reduced)
  S_NMIN,     // -min s (max-reduced)
  S_BB,       // ||s_bar||^2 (scaled)
  S_GAM,      // (r, u)
  S_RR,       // (r, r) inner
  S_UU,       // (u, u)
  S_EQ,       // 1/2 sum_CSR w (u_i - u_j)^2 times 2 (raw walk sum)
  S_RR64,     // ||r64||^2
  S_P,        // ||q||^2
  S_QS,       // 1^T q
  S_CI,       // ||s_bar - q||^2
  S_D,        // raw walk sum of w (q_i - q_j)^2 over CSR entries
  NSLOT
};

enum Mode { kModeMixed = 0, kModeFP64 = 1, kModeFP32 = 2 };

template <typename VI>
struct SolveParams {
  using VR = typename Refine<VI>::type;  // refinement arithmetic
  SellGraph sg;  // work units: long-row chunks and 32-row slices
  const int32_t* perm;  // solver node -> input id
  VI* hub_part;         // [n_chunks][K] chunk sums of multi-chunk rows
  VR* hub_part64;
  double* quad_u;       // [n_units][K] edge sums per work unit (K >= 8)
  unsigned long long* unit_counter;  // next work unit of the wide walks
  const float* dinv;
  // problem (column c of this launch: s + c*ld)
  const double* s;
  int64_t ld;
  double* z_out;  // nullable, same layout as s
  double* quant;  // [K][5]
  double* resid;  // [K]
  int* status;    // [0] err bits, [1] iterations, [2] refinements
  // row-major n x K workspace; the refinement state is in VR
  VR* sbar;
  VR* q;
  VR* t64;
  VI* x;
  VI* r;
  VI* u;
  VI* p;
  VI* d;
  VI* t;
  double* part;  // [blocks][NSLOT][K]
  Barrier* bar;
  // options
  double tol;
  double inner_tol;
  int max_iter;
  int max_refine;
  int mode;
  int qtol;  // tol bounds each quantity's relative error (FJ_QUANTITY_TOL)
  double qtol_frac;   // part of tol the certified bound may use
  double first_goal;  // quantity mode: the first inner solve's reduction
  // two-solve mode (Algorithm 1 as printed): launch columns come in pairs
  // (2j: s_j solved as is, 2j+1: s_j centred), source column = c >> col_shift
  int paper;
  int col_shift;
  // warm start: initial guess z0 (same layout as s) or null
  const double* z0;
  // bounded waits: a grid barrier gives up after timeout_ns; withhold > 0
  // makes block 0 skip its arrival at barrier number `withhold` (the
  // failure-detection test's stuck block)
  uint64_t timeout_ns;
  unsigned withhold;
};

// Barrier of one problem's nb blocks (bid = this block's index among them;
// the whole grid, or one problem's block range of a packed launch) with a
// bounded wait.  The counter only grows: barrier number e of a solve
// completes when it reaches e * nb.  Arrival is
// one release-reduction per block (publishing the block's writes, ordered
// before it by __syncthreads); the wait polls with acquire loads.  Returns
// false once any block has given up (error bit kErrTimeout), after which every
// later barrier returns at once so that all blocks leave the kernel.
__device__ __forceinline__ bool grid_sync(Barrier* bar, int* status, unsigned& epoch, uint64_t timeout_ns,
                                          unsigned withhold, int bid, int nb) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = (ld_volatile_i32(status) & kErrTimeout) == 0;
    if (nb > 1 && ok) {
      ++epoch;
      const unsigned target = epoch * (unsigned)nb;
      if (!(epoch == withhold && bid == 0))
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
      if (ld_acquire_u32(&bar->count) < target) {
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u32(&bar->count) < target) {
          if ((++spins & 255u) == 0) {
            if ((ld_volatile_i32(status) & kErrTimeout) || global_ns() - t0 > timeout_ns) {
              atomicOr(status, kErrTimeout);
              ok = 0;
              break;
            }
          }
        }
      }
    }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Block-level sums (or maxima, kMax) of NS per-thread values (thread column
// c = tid % K), stored as this block's partials for the given slots.
template <int K, int NS, bool kMax = false>
__device__ __forceinline__ void block_store(const double (&v)[NS], const int (&slots)[NS],
                                            double* part, double* red /*[NS][kWarps][K]*/, int bid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // red aliases the walks' shared staging
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    double x = v[j];
#pragma unroll
    for (int off = 16; off >= K; off >>= 1) {
      const double y = __shfl_xor_sync(kFull, x, off);
      x = kMax ? fmax(x, y) : x + y;
    }
    if (lane < K) red[(j * kWarps + warp) * K + lane] = x;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NS * K; e += kThreads) {
    const int j = e / K, c = e % K;
    double s = kMax ? -INFINITY : 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const double y = red[(j * kWarps + w) * K + c];
      s = kMax ? fmax(s, y) : s + y;
    }
    part[((int64_t)bid * NSLOT + slots[j]) * K + c] = s;
  }
  __syncthreads();
}

// After a barrier: res[slot][c] = sum (or max, kMax) over blocks of the
// partials, in block order, identically in every block.
template <int K, int NS, bool kMax = false>
__device__ __forceinline__ void grid_reduce(const int (&slots)[NS], const double* part,
                                            double* res /*[NSLOT][K]*/, int nb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = warp; e < NS * K; e += kWarps) {
    const int slot = slots[e / K], c = e % K;
    double s = kMax ? -INFINITY : 0.0;
    for (int b = lane; b < nb; b += 32) {
      const double y = __ldcg(&part[((int64_t)b * NSLOT + slot) * K + c]);
      s = kMax ? fmax(s, y) : s + y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double y = __shfl_xor_sync(kFull, s, off);
      s = kMax ? fmax(s, y) : s + y;
    }
    if (lane == 0) res[slot * K + c] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Largest residual norm eps = ||s_bar - (I+L) q|| at which every quantity
// evaluated at the iterate is certified within relative error t of its
// value at the exact solution.  (I + L) has no eigenvalue below 1, so the
// error e = (I+L)^-1 r has ||e|| <= eps and e^T L e <= r^T (I+L)^-1 r <=
// eps^2.  Each of C_I, D, P, C is ||a||^2 for a vector a that moves with the
// iterate by e, the centred e, or W^1/2 B e (Sec. 3.2 definitions), so it is
// off by at most eps (2 ||a|| + eps); I_dc = D + C by the sum of two such
// terms.  A relative error of at most t needs dev <= t (x - dev), i.e.
// dev <= t' x with t' = t / (1 + t): the positive root of
// eps^2 + 2 a eps = t' x, written stably.  Zero quantities bound nothing.
__device__ __forceinline__ double quantity_eps(double CI, double D, double Pq, double C, double t) {
  const double tp = t / (1.0 + t);
  double best = INFINITY;
  const double xs[4] = {CI, D, Pq, C};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double x = xs[j];
    if (x > 0.0) {
      const double a = sqrt(x);
      best = fmin(best, tp * x / (a + sqrt(a * a + tp * x)));
    }
  }
  const double I = D + C;  // 2 eps^2 + 2 (a_D + a_C) eps = t' I
  if (I > 0.0) {
    const double b = sqrt(fmax(D, 0.0)) + sqrt(fmax(C, 0.0));
    best = fmin(best, tp * I / (b + sqrt(b * b + 2.0 * tp * I)));
  }
  return best;
}

// SpMM walk for K >= 8: the warps of the whole grid take work units one at a
// time from one counter, in unit order (hub chunks first, then slices by
// falling degree), so the walk ends with at most one unit per warp in flight.
// The counter only grows: a walk starting at value `base` hands out units
// base + [0, n_units) and ends at base + n_units + (number of warps), each
// warp having drawn exactly one value past the end.  Each unit's edge sum
// sum w (x_r - x_j)^2 is stored per unit and column (quad_u); unit_sum adds
// them up after the walk's barrier in a fixed partition, so the result does
// not depend on which warp took which unit.
template <typename T, int K>
__device__ __forceinline__ void wide_walk(const SellGraph& g, const T* __restrict__ x, T* __restrict__ out,
                                          T* __restrict__ part,
                                          unsigned long long* counter, unsigned long long base,
                                          double* __restrict__ quad_u, T* __restrict__ sxr) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(counter, 1ull) - base;
    const int64_t u = (int64_t)__shfl_sync(kFull, k, 0);
    if (u >= g.n_units) break;
    T q = num<T>(0.f);
    wide_unit<T, K>(g, x, out, part, u, q, sxr);
    double qd = to_double(q);
#pragma unroll
    for (int off = K; off < 32; off <<= 1) qd += __shfl_xor_sync(kFull, qd, off);
    if (lane < K) quad_u[u * K + lane] = qd;
  }
}

// This thread's share of the block's sum of quad_u over units [ub0, ub1):
// column c = tid % K, group tid / K takes a fixed contiguous sub-range.
template <int K>
__device__ __forceinline__ double unit_sum(const double* __restrict__ quad_u, int64_t ub0, int64_t ub1) {
  constexpr int G = kThreads / K;
  const int c = threadIdx.x % K, gi = threadIdx.x / K;
  const int64_t len = ub1 - ub0;
  const int64_t a = ub0 + len * gi / G, b = ub0 + len * (gi + 1) / G;
  double s = 0.0;
  for (int64_t u = a; u < b; ++u) s += __ldcg(&quad_u[u * K + c]);
  return s;
}

// A lane holding partial sums for all K columns hands them to block_store,
// which sums lanes of equal column lane % K: lane c < K gets the warp total of
// column c, every other lane 0.
template <typename T, int K>
__device__ __forceinline__ double lane_share(T (&v)[K]) {
  const int lane = threadIdx.x & 31;
  double mine = 0.0;
#pragma unroll
  for (int cc = 0; cc < K; ++cc) {
    double x = to_double(v[cc]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
    if (lane == cc) mine = x;
  }
  return mine;
}

// The whole solve of one problem on nb blocks; bid = this block's index
// among them.  Every grid-wide step (barriers, reductions, work splits) is
// over those nb blocks only, so a problem's results depend on nb alone, not
// on the launch it runs in.
template <typename VI, int K>
__device__ __forceinline__ void solve_body(const SolveParams<VI>& P, const int bid, const int nb) {
  using VR = typename SolveParams<VI>::VR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw);  // [7][kWarps][K], aliases the staging
  __shared__ double res[NSLOT * K];
  __shared__ double alpha[K], beta[K], gam_prev[K], alpha_prev[K], rr_goal[K], mu[K], bb[K];
  __shared__ double sc[K], isc[K];  // 2^-e and 2^e of each column
  __shared__ int ex[K];             // e
  __shared__ int active[K], first[K], done[K], inner_ok[K];
  __shared__ int ctl_any_active, ctl_stop;
  __shared__ int64_t n_multi_sh;

  const int warp = threadIdx.x >> 5;
  const int64_t n = P.sg.n;
  const int64_t NK = n * K;
  const int64_t gtid = (int64_t)bid * kThreads + threadIdx.x;
  const int64_t gstride = (int64_t)nb * kThreads;
  const int c = threadIdx.x % K;
  // per-warp staging of the wide walks' row values
  VI* my_sxr = reinterpret_cast<VI*>(smem_raw + warp * kWideStageBytes);
  VR* my_sxr64 = reinterpret_cast<VR*>(my_sxr);
  int* status = P.status;
  const bool fp32_mode = P.mode == kModeFP32;
  unsigned epoch = 0;  // barriers passed (used by thread 0)
  auto sync = [&]() { return grid_sync(P.bar, status, epoch, P.timeout_ns, P.withhold, bid, nb); };
  // every K walks the same work units (sliced ELL for K <= 4, lanes as
  // columns for K >= 8), so all row sums are complete after a walk
  constexpr bool kWide = K >= 8;
  // narrow walks: entries in flight per lane (8 for rows of up to 8 bytes in
  // the float32-inner kernels; 4 otherwise, which keeps the float64-inner
  // kernels from spilling)
  constexpr int kInnerBatch = (sizeof(VI) == 4 && K <= 2) ? 8 : 4;
  constexpr int kResidBatch = (sizeof(VI) == 4 && K == 1) ? 8 : 4;
  // narrow kernels stream the vectors of the update pass (evict-first), so
  // that the walk's gathered vector stays in L2; the wide kernels keep
  // plain loads and stores, which measured faster there
  constexpr bool kStream = K <= 4;
  auto vld = [](const VI* a) -> VI {
    if constexpr (kStream) return ld_cs(a);
    else return *a;
  };
  auto vst = [](VI* a, VI v) {
    if constexpr (kStream) st_cs(a, v);
    else *a = v;
  };

  // K <= 4: this warp's share of the work units, split by cost;
  // K >= 8: the units whose edge sums this block adds up (even split)
  int64_t u0 = 0, u1 = 0;
  unsigned long long unit_base = 0;  // unit counter at the start of the next wide walk
  if constexpr (kWide) {
    u0 = P.sg.n_units * (int64_t)bid / nb;
    u1 = P.sg.n_units * (int64_t)(bid + 1) / nb;
  } else {
    // range wr of W: consecutive ranges (units of similar kind) go to
    // different blocks, so that every SM gets a mix of hub chunks and slices
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)nb * kWarps;
    const int64_t wr = (int64_t)warp * nb + bid;
    int64_t v = 0;
    if (lane < 2) v = sell_unit_start(P.sg, wr + lane, W);
    u0 = __shfl_sync(kFull, v, 0);
    u1 = __shfl_sync(kFull, v, 1);
  }
  const unsigned long long unit_step = (unsigned long long)P.sg.n_units + (unsigned long long)nb * kWarps;

  // ---------------------------------------------------------------- setup
  {
    // the opinions' sum and range, and whether any lies outside the [0, 1]
    // of Sec. 2.2
    double acc = 0.0, mx = -INFINITY, nmn = -INFINITY;
    bool outside = false;
    for (int64_t idx = gtid; idx < NK; idx += gstride) {
      const double x = P.s[(int64_t)(c >> P.col_shift) * P.ld + idx / K];
      acc += x;
      mx = fmax(mx, x);
      nmn = fmax(nmn, -x);
      outside |= !(x >= 0.0 && x <= 1.0);
    }
    if (threadIdx.x == 0) {
      // rows [0, n_multi) hold every row of several chunks: the rows of
      // degree >= kDegKeyMax come first (in input order among themselves),
      // then rows by falling degree, so "degree >= kDegKeyMax or several
      // chunks" holds on a prefix.  The narrow kernels add these rows'
      // chunk partials warp-wide in the passes after the walks.
      int64_t lo = 0, hi = kWide ? 0 : P.sg.n_long;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (P.sg.row_ptr[mid + 1] - P.sg.row_ptr[mid] >= kDegKeyMax ||
            P.sg.long_first[mid + 1] - P.sg.long_first[mid] >= 2)
          lo = mid + 1;
        else
          hi = mid;
      }
      n_multi_sh = lo;
    }
    if (__syncthreads_or(outside) && threadIdx.x == 0) atomicOr(status, kWarnOpinionRange);
    const double v[1] = {acc};
    const int sl[1] = {S_SUM};
    block_store<K, 1>(v, sl, P.part, red, bid);
    const double vm[2] = {mx, nmn};
    const int slm[2] = {S_MAX, S_NMIN};
    block_store<K, 2, true>(vm, slm, P.part, red, bid);
  }
  if (!sync()) return;
  {
    const int sl[1] = {S_SUM};
    grid_reduce<K, 1>(sl, P.part, res, nb);
    const int slm[2] = {S_MAX, S_NMIN};
    grid_reduce<K, 2, true>(slm, P.part, res, nb);
    if (threadIdx.x < K) {
      const int cc = threadIdx.x;
      // a column solved as is (two-solve mode, even columns) keeps mu = 0
      const double m = (P.paper && !(cc & 1)) ? 0.0 : res[S_SUM * K + cc] / (double)n;
      mu[cc] = m;
      // max |s_bar| = max(max s - mu, mu - min s); its binary exponent e
      // (clamped so that 2^-e and 2^e stay normal) scales the column
      const double bound = fmax(res[S_MAX * K + cc] - m, res[S_NMIN * K + cc] + m);
      int e = 0;
      if (bound > 0.0 && isfinite(bound)) e = max(-1020, min(1020, ilogb(bound)));
      ex[cc] = e;
      sc[cc] = ldexp(1.0, -e);
      isc[cc] = ldexp(1.0, e);
      done[cc] = 0;
    }
    __syncthreads();
  }

  // refinement residual walk: t64 = L q (off-diagonal part of (I + L) q) and
  // this block's part of sum w (q_i - q_j)^2, then the barrier
  auto residual_walk = [&]() -> bool {
    double quad;
    if constexpr (kWide) {
      wide_walk<VR, K>(P.sg, P.q, P.t64, P.hub_part64, P.unit_counter, unit_base, P.quad_u, my_sxr64);
      unit_base += unit_step;
      if (!sync()) return false;
      quad = unit_sum<K>(P.quad_u, u0, u1);
    } else {
      VR qd[K];
#pragma unroll
      for (int cc = 0; cc < K; ++cc) qd[cc] = num<VR>(0.0f);
      sell_walk<VR, K, kResidBatch>(P.sg, P.q, P.t64, P.hub_part64, u0, u1, qd);
      quad = lane_share<VR, K>(qd);
    }
    const double v[1] = {quad};
    const int sl[1] = {S_D};
    block_store<K, 1>(v, sl, P.part, red, bid);
    return sync();
  };

  // warm start: q = (z0 - mu 1) 2^-e (its residual walk opens the loop)
  const bool warm = P.z0 != nullptr;
  if (warm) {
    for (int64_t idx = gtid; idx < NK; idx += gstride)
      P.q[idx] = from_double<VR>((P.z0[(int64_t)(c >> P.col_shift) * P.ld + P.perm[idx / K]] - mu[c]) * sc[c]);
    if (!sync()) return;
  }

  int iters = 0, refines = 0;
  bool init = true;
  bool need_walk = warm;  // q changed since the last residual walk
  while (true) {
    if (need_walk && !residual_walk()) return;
    // ---------------------------------------------- refinement residual pass
    // r64 = s_bar - q - t64 (t64 = off-diagonal part of L q, from the walk)
    // plus the quantity partials and the start of the next inner solve.
    {
      // float64-accurate sums in VR; the inner-solve sums in VI
      const VR zero = num<VR>(0.0f);
      VR a_rr64 = zero, a_p = zero, a_qs = zero, a_ci = zero;
      double a_bb = 0, a_gam = 0, a_rr = 0, a_uu = 0;
      const double m = mu[c], scale = sc[c];
      const bool lz_col = P.paper && !(c & 1);
      // after a residual walk, rows of several chunks (narrow kernels) get
      // their row sums warp-wide first, as in the vector update
      const bool walked = !init || warm;
      const int64_t n_multi = walked ? n_multi_sh : 0;
      auto elem = [&](int64_t idx, int64_t i, bool given, VR lq_given) {
        VR sb, qv, lq;
        if (init) {
          const double sbd = (P.s[(int64_t)(c >> P.col_shift) * P.ld + P.perm[i]] - m) * scale;
          sb = from_double<VR>(sbd);
          P.sbar[idx] = sb;
          a_bb += sbd * sbd;
          if (warm) {
            qv = P.q[idx];
            lq = given ? lq_given : row_t<VR, K>(P.sg, P.t64, P.hub_part64, i, idx, c);
          } else {
            P.q[idx] = zero;
            qv = zero;
            lq = zero;
          }
        } else {
          sb = P.sbar[idx];
          qv = P.q[idx];
          lq = given ? lq_given : row_t<VR, K>(P.sg, P.t64, P.hub_part64, i, idx, c);
        }
        const VR r64 = (sb - qv) - lq;
        a_rr64 += r64 * r64;
        a_p += qv * qv;
        a_qs += qv;
        // C_I = ||s_bar - q||^2, or ||L z~||^2 for a column solved as is
        // in two-solve mode (lq = off-diagonal part of (I + L) q = L q)
        const VR dq = lz_col ? lq : sb - qv;
        a_ci += dq * dq;
        const VI rv = to_inner<VI>(r64);
        const VI uv = P.dinv[i] * rv;
        vst(P.x + idx, VI(0));
        vst(P.r + idx, rv);
        P.u[idx] = uv;
        a_gam += (double)(rv * uv);
        a_rr += (double)(rv * rv);
        a_uu += (double)(uv * uv);
      };
      if constexpr (!kWide) {
        const int lane = threadIdx.x & 31;
        for (int64_t i = (int64_t)bid * kWarps + warp; i < n_multi; i += (int64_t)nb * kWarps) {
          const int32_t f = P.sg.long_first[i], l = P.sg.long_first[i + 1];
          VR ts[K];
#pragma unroll
          for (int cc = 0; cc < K; ++cc) ts[cc] = zero;
          if (l - f == 1) {  // a row of one chunk: the walk wrote its sum
#pragma unroll
            for (int cc = 0; cc < K; ++cc)
              if (lane == 0) ts[cc] = P.t64[i * K + cc];
          }
          for (int32_t q = f + lane; l - f > 1 && q < l; q += 32) {
#pragma unroll
            for (int cc = 0; cc < K; ++cc) ts[cc] += P.hub_part64[(int64_t)q * K + cc];
          }
#pragma unroll
          for (int cc = 0; cc < K; ++cc) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) ts[cc] += shfl_xor_v(ts[cc], off);
          }
          VR lq = ts[0];
#pragma unroll
          for (int cc = 1; cc < K; ++cc)
            if (lane == cc) lq = ts[cc];
          if (lane < K) elem(i * K + lane, i, true, lq);
        }
      }
      for (int64_t idx = gtid + n_multi * K; idx < NK; idx += gstride) elem(idx, idx / K, false, zero);
      const double v[7] = {to_double(a_rr64), to_double(a_p), to_double(a_qs), to_double(a_ci),
                           a_gam, a_rr, a_uu};
      const int sl[7] = {S_RR64, S_P, S_QS, S_CI, S_GAM, S_RR, S_UU};
      block_store<K, 7>(v, sl, P.part, red, bid);
      if (init) {
        const double vb[1] = {a_bb};
        const int sb[1] = {S_BB};
        block_store<K, 1>(vb, sb, P.part, red, bid);
      }
    }
    if (!sync()) return;
    {
      const int sl[7] = {S_RR64, S_P, S_QS, S_CI, S_GAM, S_RR, S_UU};
      grid_reduce<K, 7>(sl, P.part, res, nb);
      if (init) {
        const int sb[1] = {S_BB};
        grid_reduce<K, 1>(sb, P.part, res, nb);
      }
      if (!init || warm) {
        const int sd[1] = {S_D};
        grid_reduce<K, 1>(sd, P.part, res, nb);
      }
    }
    if (threadIdx.x == 0) ctl_stop = 0;
    __syncthreads();
    if (threadIdx.x < K) {
      const int cc = threadIdx.x;
      if (init) bb[cc] = res[S_BB * K + cc];
      const double rr64 = res[S_RR64 * K + cc];
      const double rel = bb[cc] > 0.0 ? sqrt(rr64 / bb[cc]) : 0.0;
      if (!finite(rr64)) atomicOr(status, kErrNumeric);
      // quantities of the current iterate (final after the last pass),
      // scaled back: squares by 2^2e, 1^T q by 2^e
      if (bid == 0) {
        const int e2 = 2 * ex[cc];
        const double m = mu[cc];
        const double D = (init && !warm) ? 0.0 : ldexp(0.5 * res[S_D * K + cc], e2);
        const double Pq = ldexp(res[S_P * K + cc], e2);
        const double C = Pq + 2.0 * m * ldexp(res[S_QS * K + cc], ex[cc]) + (double)n * m * m;
        P.quant[cc * 5 + 0] = ldexp(res[S_CI * K + cc], e2);
        P.quant[cc * 5 + 1] = D;
        P.quant[cc * 5 + 2] = Pq;
        P.quant[cc * 5 + 3] = C;
        P.quant[cc * 5 + 4] = D + C;
        P.resid[cc] = rel;
      }
      bool conv = (bb[cc] == 0.0) || (rel <= P.tol);
      // residual-norm reduction the next inner solve should reach
      double need = (rr64 > 0.0) ? 0.5 * P.tol * sqrt(bb[cc] / rr64) : 1.0;
      if (P.qtol) {
        // certified per-quantity rule, with part of tol kept as margin for
        // rounding; the first pass (q = 0 or z0) only sets the first inner
        // solve's goal
        if (init) {
          need = P.first_goal;
          conv = bb[cc] == 0.0;
        } else {
          const int e2 = 2 * ex[cc];
          const double m = mu[cc];
          const double Pq = ldexp(res[S_P * K + cc], e2);
          const double eps_goal =
              quantity_eps(ldexp(res[S_CI * K + cc], e2), ldexp(0.5 * res[S_D * K + cc], e2), Pq,
                           Pq + 2.0 * m * ldexp(res[S_QS * K + cc], ex[cc]) + (double)n * m * m,
                           P.qtol_frac * P.tol);
          const double eps = ldexp(sqrt(rr64), ex[cc]);
          conv = bb[cc] == 0.0 || eps <= eps_goal;
          need = (eps > 0.0) ? 0.5 * fmin(eps_goal / eps, 1.0) : 1.0;
        }
      }
      if (fp32_mode && !init) conv = inner_ok[cc] || bb[cc] == 0.0;  // one inner solve only
      if (!done[cc] && conv) done[cc] = 1;
      // next inner solve for columns not done
      const double rr = res[S_RR * K + cc];
      double goal = P.inner_tol;
      if (P.mode == kModeFP64) goal = need;
      else if (need > goal || (P.qtol && init)) goal = need;
      if (fp32_mode) goal = P.tol;
      rr_goal[cc] = goal * goal * rr;
      active[cc] = !done[cc] && rr > rr_goal[cc];
      inner_ok[cc] = !active[cc];
      first[cc] = 1;
    }
    __syncthreads();
    if (!init) ++refines;
    if (threadIdx.x == 0) {
      int all_done = 1, any = 0;
      for (int j = 0; j < K; ++j) {
        all_done &= done[j];
        any |= active[j];
      }
      int stop = all_done || (ld_volatile_i32(status) & (kErrNumeric | kErrTimeout));
      if (!init && refines >= P.max_refine) stop = 1;
      if (!init && fp32_mode) stop = 1;
      if (iters >= P.max_iter) stop = 1;
      ctl_stop = stop;
      ctl_any_active = any;
    }
    __syncthreads();
    init = false;
    if (ctl_stop) break;

    // ------------------------------------------------------ inner PCG loop
    while (ctl_any_active && iters < P.max_iter) {
      // SpMV walk: t = off-diagonal part of (I + L) u, and the edge part of
      // (u, (I+L) u).
      {
        double qv;
        if constexpr (kWide) {
          wide_walk<VI, K>(P.sg, P.u, P.t, P.hub_part, P.unit_counter, unit_base, P.quad_u, my_sxr);
          unit_base += unit_step;
          if (!sync()) return;
          qv = unit_sum<K>(P.quad_u, u0, u1);
        } else {
          VI quad[K];
#pragma unroll
          for (int cc = 0; cc < K; ++cc) quad[cc] = VI(0);
          sell_walk<VI, K, kInnerBatch>(P.sg, P.u, P.t, P.hub_part, u0, u1, quad);
          qv = lane_share<VI, K>(quad);
        }
        const double v[1] = {qv};
        const int sl[1] = {S_EQ};
        block_store<K, 1>(v, sl, P.part, red, bid);
      }
      if (!sync()) return;
      {
        const int sl[1] = {S_EQ};
        grid_reduce<K, 1>(sl, P.part, res, nb);
      }
      if (threadIdx.x < K) {
        const int cc = threadIdx.x;
        if (active[cc]) {
          const double gam = res[S_GAM * K + cc];
          // (u, (I+L) u) = u^T u + u^T L u, u^T L u = 1/2 sum over CSR entries
          const double delta = res[S_UU * K + cc] + 0.5 * res[S_EQ * K + cc];
          double a, b;
          if (first[cc]) {
            b = 0.0;
            a = gam / delta;
          } else {
            b = gam / gam_prev[cc];
            a = gam / (delta - b * gam / alpha_prev[cc]);
          }
          if (!finite(a) || !finite(b) || gam == 0.0) {
            if (!(gam == 0.0)) atomicOr(status, kErrNumeric);
            a = 0.0;
            b = 0.0;
            active[cc] = 0;
          }
          alpha[cc] = a;
          beta[cc] = b;
          gam_prev[cc] = gam;
          alpha_prev[cc] = a;
        } else {
          alpha[cc] = 0.0;
          beta[cc] = 0.0;
        }
      }
      __syncthreads();
      // vector update: p = u + beta p, d = w + beta d, x += alpha p,
      // r -= alpha d, u = M r; partials (r,u), (r,r), (u,u).
      {
        double a_gam = 0, a_rr = 0, a_uu = 0;
        const VI al = (VI)alpha[c], be = (VI)beta[c];
        const bool fst = first[c] != 0;
        VI l_gam = 0, l_rr = 0, l_uu = 0;
        VI* __restrict__ vp = P.p;
        VI* __restrict__ vd = P.d;
        VI* __restrict__ vx = P.x;
        VI* __restrict__ vr = P.r;
        VI* __restrict__ vu = P.u;
        const VI* __restrict__ vt = P.t;
        const float* __restrict__ vdinv = P.dinv;
        // the new u is the next walk's gathered vector: stored normally (it
        // stays in L2), the other vectors streamed in the narrow kernels
        auto update = [&](int64_t idx, int64_t i, VI uv, VI tv, VI pv, VI dv, VI xv, VI rv, VI di, VI al_, VI be_) {
          const VI wv = uv + tv;
          const VI pn = uv + be_ * pv;
          const VI dn = wv + be_ * dv;
          const VI xn = xv + al_ * pn;
          const VI rn = rv - al_ * dn;
          const VI un = di * rn;
          vst(vp + idx, pn);
          vst(vd + idx, dn);
          vst(vx + idx, xn);
          vst(vr + idx, rn);
          vu[idx] = un;
          l_gam += rn * un;
          l_rr += rn * rn;
          l_uu += un * un;
        };
        // rows of several chunks (narrow kernels): one warp per row adds its
        // chunk sums (lanes stride over the chunks, then the xor tree) and
        // lane c updates the row's column c
        const int64_t n_multi = n_multi_sh;
        if constexpr (!kWide) {
          const int lane = threadIdx.x & 31;
          for (int64_t i = (int64_t)bid * kWarps + warp; i < n_multi; i += (int64_t)nb * kWarps) {
            const int32_t f = P.sg.long_first[i], l = P.sg.long_first[i + 1];
            VI ts[K];
#pragma unroll
            for (int cc = 0; cc < K; ++cc) ts[cc] = VI(0);
            if (l - f == 1) {  // a row of one chunk: the walk wrote its sum
#pragma unroll
              for (int cc = 0; cc < K; ++cc)
                if (lane == 0) ts[cc] = vt[i * K + cc];
            }
            for (int32_t q = f + lane; l - f > 1 && q < l; q += 32) {
#pragma unroll
              for (int cc = 0; cc < K; ++cc) ts[cc] += P.hub_part[(int64_t)q * K + cc];
            }
#pragma unroll
            for (int cc = 0; cc < K; ++cc) {
#pragma unroll
              for (int off = 16; off > 0; off >>= 1) ts[cc] += shfl_xor_v(ts[cc], off);
            }
            VI tv = ts[0];
#pragma unroll
            for (int cc = 1; cc < K; ++cc)
              if (lane == cc) tv = ts[cc];
            if (lane < K) {
              const int64_t idx = i * K + lane;
              update(idx, i, vld(vu + idx), tv, fst ? VI(0) : vld(vp + idx), fst ? VI(0) : vld(vd + idx),
                     vld(vx + idx), vld(vr + idx), vdinv[i], al, be);
            }
          }
        }
        // kV elements per thread per round, all loads issued before use
        constexpr int kV = 2;
        for (int64_t base = gtid + (kWide ? 0 : n_multi * K); base < NK; base += kV * gstride) {
          VI uv[kV], tv[kV], pv[kV], dv[kV], xv[kV], rv[kV], di[kV];
#pragma unroll
          for (int e = 0; e < kV; ++e) {
            const int64_t idx = base + e * gstride;
            if (idx < NK) {
              const int64_t i = idx / K;
              uv[e] = vld(vu + idx);
              tv[e] = row_t<VI, K>(P.sg, vt, P.hub_part, i, idx, c);
              pv[e] = fst ? VI(0) : vld(vp + idx);
              dv[e] = fst ? VI(0) : vld(vd + idx);
              xv[e] = vld(vx + idx);
              rv[e] = vld(vr + idx);
              di[e] = kStream ? ld_ro(vdinv + i) : vdinv[i];
            }
          }
#pragma unroll
          for (int e = 0; e < kV; ++e) {
            const int64_t idx = base + e * gstride;
            if (idx < NK) update(idx, idx / K, uv[e], tv[e], pv[e], dv[e], xv[e], rv[e], di[e], al, be);
          }
        }
        a_gam = (double)l_gam;
        a_rr = (double)l_rr;
        a_uu = (double)l_uu;
        const double v[3] = {a_gam, a_rr, a_uu};
        const int sl[3] = {S_GAM, S_RR, S_UU};
        block_store<K, 3>(v, sl, P.part, red, bid);
      }
      if (!sync()) return;
      {
        const int sl[3] = {S_GAM, S_RR, S_UU};
        grid_reduce<K, 3>(sl, P.part, res, nb);
      }
      ++iters;
      if (threadIdx.x < K) {
        const int cc = threadIdx.x;
        first[cc] = 0;
        const double rr = res[S_RR * K + cc];
        if (!finite(rr)) {
          atomicOr(status, kErrNumeric);
          active[cc] = 0;
        }
        if (active[cc] && rr <= rr_goal[cc]) {
          active[cc] = 0;
          inner_ok[cc] = 1;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int any = 0;
        for (int j = 0; j < K; ++j) any |= active[j];
        if (ld_volatile_i32(status) & (kErrNumeric | kErrTimeout)) any = 0;
        ctl_any_active = any;
      }
      __syncthreads();
    }

    // q += x in the refinement arithmetic, then the residual walk t64 = L q
    // and sum w (q_i - q_j)^2
    for (int64_t idx = gtid; idx < NK; idx += gstride) P.q[idx] = add_inner(P.q[idx], P.x[idx]);
    if (!sync()) return;
    need_walk = true;
  }

  // ---------------------------------------------------------------- output
  if (P.z_out && !(P.paper && (c & 1))) {
    for (int64_t idx = gtid; idx < NK; idx += gstride)
      P.z_out[(int64_t)(c >> P.col_shift) * P.ld + P.perm[idx / K]] = to_double(P.q[idx]) * isc[c] + mu[c];
  }
  if (bid == 0 && threadIdx.x == 0) {
    int all_done = 1;
    for (int j = 0; j < K; ++j) all_done &= done[j];
    if (!all_done) atomicOr(status, kErrNotConverged);
    status[1] = iters;
    status[2] = refines;
  }
}

template <typename VI, int K>
__global__ void __launch_bounds__(kThreads, 2) k_solve(const __grid_constant__ SolveParams<VI> P) {
  solve_body<VI, K>(P, blockIdx.x, gridDim.x);
}

// Several independent problems in one cooperative launch (small graphs
// packed together): problem p runs on blocks [first_block[p],
// first_block[p + 1]) with its own barrier, reduction slots, workspace and
// convergence control.
constexpr int kPackMax = FJ_PACK_MAX;
template <typename VI>
struct PackParams {
  int count;
  int first_block[kPackMax + 1];
  SolveParams<VI> prob[kPackMax];
};
// kernel parameters are limited to 32764 bytes
static_assert(sizeof(PackParams<float>) <= 32000 && sizeof(PackParams<double>) <= 32000,
              "packed launch parameters too large");

template <typename VI, int K>
__global__ void __launch_bounds__(kThreads, 2) k_solve_packed(const __grid_constant__ PackParams<VI> PP) {
  int p = 0;  // block-uniform
  while (p + 1 < PP.count && (int)blockIdx.x >= PP.first_block[p + 1]) ++p;
  const int b0 = PP.first_block[p];
  solve_body<VI, K>(PP.prob[p], (int)blockIdx.x - b0, PP.first_block[p + 1] - b0);
}

// ------------------------------------------------------------------ host

// Limit of every grid-barrier wait, and the test hook's withheld barrier
// (fj_debug_barrier).
constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // 4 s
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
std::atomic<int> g_withhold{0};

// Dynamic shared memory of the solve kernels (reduction scratch, or the
// wide walks' staging).
template <typename VI, int K>
static size_t solve_dyn_smem() {
  const size_t red_bytes = (size_t)7 * kWarps * K * sizeof(double);
  const size_t stage = (K <= 4) ? 0 : (size_t)kWarps * kWideStageBytes;
  return std::max(red_bytes, stage);
}

// Co-resident blocks per SM of k_solve<VI, K> and k_solve_packed<VI, K> on
// the current device (the attribute and the occupancy query once per device
// and instantiation; the two kernels share the body and its resources, and
// the smaller of the two counts is returned).
template <typename VI, int K>
static fj_status solve_blocks_per_sm(int* out) {
  static std::mutex setup_mu;
  static int per_sm_of[kMaxDevices] = {};
  int device = 0;
  FJ_CUDA(cudaGetDevice(&device));
  if (device < 0 || device >= kMaxDevices) {
    set_error("device %d out of range", device);
    return FJ_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(setup_mu);
  if (per_sm_of[device] == 0) {
    const size_t dyn = solve_dyn_smem<VI, K>();
    int a = 0, b = 0;
    FJ_CUDA(cudaFuncSetAttribute(k_solve<VI, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    FJ_CUDA(cudaFuncSetAttribute(k_solve_packed<VI, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    FJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_solve<VI, K>, kThreads, dyn));
    FJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_solve_packed<VI, K>, kThreads, dyn));
    const int per_sm = std::min(std::min(a, b), kMaxBlocksPerSM);
    per_sm_of[device] = per_sm > 0 ? per_sm : -1;
  }
  if (per_sm_of[device] < 1) {
    set_error("solver kernel does not fit on an SM");
    return FJ_ERR_CUDA;
  }
  *out = per_sm_of[device];
  return FJ_OK;
}

// Blocks a solve of K columns on g asks for when sized by its work: about 16
// path items per thread.
static int64_t work_blocks(const fj_graph* g, int K) {
  const int64_t work = g->n * K + g->nnz * K;
  const int64_t want = (work + kThreads * 16 - 1) / (kThreads * 16);
  return want < 1 ? 1 : want;
}

// Fills the parameters of one problem (K columns of s on g, on `blocks`
// blocks) and carves its workspace from ws.
template <typename VI, int K>
static fj_status fill_params(SolveParams<VI>& P, const fj_graph* g, const double* s, int64_t ld, double* z,
                             double* quant, double* resid, int* status, char* ws, size_t ws_bytes,
                             const fj_opts& o, int mode, int blocks, bool paper, const double* z0) {
  const int64_t n = g->n;
  const int64_t NK = n * K;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = ws + off;
    off += (bytes + 255) & ~size_t(255);
    return (void*)p;
  };
  P.sg = SellGraph{g->row_ptr,   g->col,       g->val,      g->long_first, g->chunk_row,
                   g->chunk_begin, g->chunk_end, g->slice_off, g->sell_col,   g->sell_val,
                   g->unit_prefix, n,            g->n_long,   g->n_nz,       g->n_chunks,
                   g->n_slices,    g->n_units};
  P.perm = g->perm;
  P.dinv = g->dinv;
  P.s = s;
  P.ld = ld;
  P.z_out = z;
  P.quant = quant;
  P.resid = resid;
  P.status = status;
  using VR = typename SolveParams<VI>::VR;
  static_assert(sizeof(VR) == 8, "refinement values are 8 bytes");
  P.sbar = (VR*)take(NK * 8);
  P.q = (VR*)take(NK * 8);
  P.t64 = (VR*)take(NK * 8);
  P.x = (VI*)take(NK * sizeof(VI));
  P.r = (VI*)take(NK * sizeof(VI));
  P.u = (VI*)take(NK * sizeof(VI));
  P.p = (VI*)take(NK * sizeof(VI));
  P.d = (VI*)take(NK * sizeof(VI));
  P.t = (VI*)take(NK * sizeof(VI));
  P.part = (double*)take((size_t)blocks * NSLOT * K * 8);
  P.hub_part = (VI*)take(std::max<int64_t>(g->n_chunks, 1) * K * sizeof(VI));
  P.hub_part64 = (VR*)take(std::max<int64_t>(g->n_chunks, 1) * K * 8);
  P.quad_u = (double*)take(std::max<int64_t>(g->n_units, 1) * K * 8);
  P.bar = (Barrier*)take(64);  // the barrier, then the unit counter
  P.unit_counter = (unsigned long long*)((char*)P.bar + 32);
  if (off > ws_bytes) {
    set_error("internal: workspace too small (%zu > %zu)", off, ws_bytes);
    return FJ_ERR_OOM;
  }
  P.tol = o.tol;
  P.inner_tol = o.inner_tol;
  P.max_iter = o.max_iter;
  P.max_refine = o.max_refine;
  P.mode = mode;
  P.qtol = (o.flags & FJ_QUANTITY_TOL) ? 1 : 0;
  // the bound may use 90% of tol; the rest covers rounding of the residual
  // and of the quantity sums (~1e-14 relative)
  P.qtol_frac = 0.9;
  // first inner solve of the quantity rule: 3% of inner_tol (3e-7 by
  // default, about the accuracy a float32 iteration attains on these
  // systems), so that the first residual check needs at most one short
  // second solve; float64 mode: a tenth of tol
  P.first_goal = mode == kModeFP64 ? 0.1 * o.tol : std::max(0.03 * o.inner_tol, 0.1 * o.tol);
  P.paper = paper ? 1 : 0;
  P.z0 = z0;
  P.col_shift = paper ? 1 : 0;
  P.timeout_ns = g_wait_ns.load(std::memory_order_relaxed);
  P.withhold = (unsigned)g_withhold.load(std::memory_order_relaxed);
  return FJ_OK;
}

template <typename VI, int K>
static fj_status launch_one(const fj_graph* g, cudaStream_t st, int num_sms, const double* s,
                            int64_t ld, double* z, double* quant, double* resid, int* status,
                            char* ws, size_t ws_bytes, const fj_opts& o, int mode, int max_blocks,
                            bool paper, const double* z0, int* grid_out) {
  int per_sm = 0;
  fj_status rc = solve_blocks_per_sm<VI, K>(&per_sm);
  if (rc != FJ_OK) return rc;
  // grid: enough blocks for the work, at most what is co-resident; a
  // negative max_blocks asks for exactly -max_blocks blocks instead
  int64_t want = work_blocks(g, K);
  int64_t cap = (int64_t)per_sm * num_sms;
  if (max_blocks < 0)
    want = -(int64_t)max_blocks;
  else if (max_blocks > 0 && cap > max_blocks)
    cap = max_blocks;
  const int blocks = (int)std::min(want, cap);
  if (grid_out && *grid_out < blocks) *grid_out = blocks;
  SolveParams<VI> P;
  rc = fill_params<VI, K>(P, g, s, ld, z, quant, resid, status, ws, ws_bytes, o, mode, blocks, paper, z0);
  if (rc != FJ_OK) return rc;
  FJ_CUDA(cudaMemsetAsync(P.bar, 0, 64, st));
  void* args[] = {&P};
  FJ_CUDA(cudaLaunchCooperativeKernel((void*)k_solve<VI, K>, dim3(blocks), dim3(kThreads), args,
                                      solve_dyn_smem<VI, K>(), st));
  count_launches(1);
  return FJ_OK;
}

// One packed launch of `count` problems of K columns each (PackItem i: graph,
// its columns, outputs, workspace, blocks).  Every problem's barrier and
// unit counter sit in `bars` (count x 64 bytes, zeroed here).
template <typename VI, int K>
static fj_status launch_packed(int count, const PackItem* it, cudaStream_t st, const fj_opts& o, int mode,
                               char* bars) {
  PackParams<VI> PP;
  PP.count = count;
  PP.first_block[0] = 0;
  for (int i = 0; i < count; ++i) {
    fj_status rc = fill_params<VI, K>(PP.prob[i], it[i].g, it[i].s, it[i].ld, it[i].z, it[i].quant,
                                      it[i].resid, it[i].status, it[i].ws, it[i].ws_bytes, it[i].opts, mode,
                                      it[i].blocks, false, nullptr);
    if (rc != FJ_OK) return rc;
    PP.prob[i].bar = (Barrier*)(bars + 64 * i);
    PP.prob[i].unit_counter = (unsigned long long*)(bars + 64 * i + 32);
    PP.first_block[i + 1] = PP.first_block[i] + it[i].blocks;
  }
  FJ_CUDA(cudaMemsetAsync(bars, 0, (size_t)64 * count, st));
  void* args[] = {&PP};
  FJ_CUDA(cudaLaunchCooperativeKernel((void*)k_solve_packed<VI, K>, dim3(PP.first_block[count]), dim3(kThreads),
                                      args, solve_dyn_smem<VI, K>(), st));
  count_launches(1);
  return FJ_OK;
}

}  // namespace fj

using namespace fj;

// Failure-detection test hook: the limit of later solves' barrier waits, and
// a barrier at which block 0 of later multi-block solves does not arrive.
extern "C" fj_status fj_debug_barrier(int64_t wait_ns, int32_t withhold) {
  if (wait_ns > 60000000000ll || (wait_ns > 0 && wait_ns < 100000) || withhold < 0) {
    set_error("fj_debug_barrier: need wait_ns <= 0 (default) or in [1e5, 6e10], withhold >= 0");
    return FJ_ERR_ARG;
  }
  g_wait_ns.store(wait_ns > 0 ? (uint64_t)wait_ns : kDefaultWaitNs, std::memory_order_relaxed);
  g_withhold.store(withhold, std::memory_order_relaxed);
  return FJ_OK;
}

// Workspace bytes of one problem of K columns solved on at most `blocks`
// blocks.
size_t fj_solve_workspace_bytes_blocks(const fj_graph* g, int K, int inner_bytes, int64_t blocks) {
  const int64_t NK = g->n * (int64_t)K;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  add(NK * 8);
  add(NK * 8);
  add(NK * 8);
  for (int i = 0; i < 6; ++i) add(NK * inner_bytes);
  add((size_t)blocks * NSLOT * K * 8);
  add(std::max<int64_t>(g->n_chunks, 1) * K * inner_bytes);
  add(std::max<int64_t>(g->n_chunks, 1) * K * 8);
  add(std::max<int64_t>(g->n_units, 1) * K * 8);
  add(64);
  return b;
}

// Workspace bytes one launch of K columns needs (on any grid).
size_t fj_solve_workspace_bytes(const fj_graph* g, int K, int inner_bytes, int num_sms) {
  return fj_solve_workspace_bytes_blocks(g, K, inner_bytes, (int64_t)num_sms * kMaxBlocksPerSM);
}

// Runs the solve for columns [0, k) of s (column-major, leading dim n, all
// device pointers) in launches of K = 32, 16, ..., 1 columns.
// quant: device [k][5]; resid: device [k]; status: device int[3 * launches].
// max_blocks > 0 caps each launch's grid, < 0 asks for exactly -max_blocks
// blocks (at most the co-resident count), 0 sizes it by the work.
// *grid_out (if given) is raised to the largest grid launched.
fj_status fj_solve_device(const fj_graph* g, cudaStream_t st, int num_sms, int32_t k,
                          const double* s, double* z, double* quant, double* resid, int* status,
                          char* ws, size_t ws_bytes, const fj_opts& o, int* launches_out,
                          int max_blocks, const double* z0, int* grid_out) {
  int mode = o.precision == FJ_PREC_FP64 ? kModeFP64 : (o.precision == FJ_PREC_FP32 ? kModeFP32 : kModeMixed);
  // two-solve mode: 2k launch columns (s_j as is, s_j centred), quant and
  // resid per launch column; every launch starts at an even column
  const bool paper = (o.flags & FJ_TWO_SOLVES) != 0;
  const int cols = paper ? 2 * k : k;
  int col = 0, li = 0;
  while (col < cols) {
    const int left = cols - col;
    int K = 32;
    while (K > left) K >>= 1;
    const int64_t src_col = paper ? col / 2 : col;
    const double* sc = s + src_col * g->n;
    double* zc = z ? z + src_col * g->n : nullptr;
    const double* z0c = z0 ? z0 + src_col * g->n : nullptr;
    double* qc = quant + (int64_t)col * 5;
    double* rc = resid + col;
    int* stc = status + 3 * li;
    fj_status rcode;
#define FJ_LAUNCH(KK)                                                                                  \
  if (mode == kModeFP64)                                                                               \
    rcode = launch_one<double, KK>(g, st, num_sms, sc, g->n, zc, qc, rc, stc, ws, ws_bytes, o, mode,   \
                                   max_blocks, paper, z0c, grid_out);                                  \
  else                                                                                                 \
    rcode = launch_one<float, KK>(g, st, num_sms, sc, g->n, zc, qc, rc, stc, ws, ws_bytes, o, mode,    \
                                  max_blocks, paper, z0c, grid_out);
    switch (K) {
      case 32: FJ_LAUNCH(32) break;
      case 16: FJ_LAUNCH(16) break;
      case 8: FJ_LAUNCH(8) break;
      case 4: FJ_LAUNCH(4) break;
      case 2: FJ_LAUNCH(2) break;
      default: FJ_LAUNCH(1) break;
    }
#undef FJ_LAUNCH
    if (rcode != FJ_OK) return rcode;
    col += K;
    ++li;
  }
  *launches_out = li;
  return FJ_OK;
}

// Packed solves: blocks a problem of K columns on g takes in a packed launch
// (sized by its work, at most `cap`), and the blocks one packed launch may
// use in all (every block co-resident).
int fj_pack_blocks(const fj_graph* g, int K, int cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(work_blocks(g, K), cap));
}

fj_status fj_pack_capacity(int precision, int K, int num_sms, int* out) {
  int per_sm = 0;
  fj_status rc = FJ_OK;
#define FJ_PER_SM(KK)                                                                     \
  rc = precision == FJ_PREC_FP64 ? solve_blocks_per_sm<double, KK>(&per_sm)               \
                                 : solve_blocks_per_sm<float, KK>(&per_sm);
  switch (K) {
    case 32: FJ_PER_SM(32) break;
    case 16: FJ_PER_SM(16) break;
    case 8: FJ_PER_SM(8) break;
    case 4: FJ_PER_SM(4) break;
    case 2: FJ_PER_SM(2) break;
    default: FJ_PER_SM(1) break;
  }
#undef FJ_PER_SM
  if (rc != FJ_OK) return rc;
  *out = per_sm * num_sms;
  return FJ_OK;
}

// Runs `count` (1 <= count <= FJ_PACK_MAX) problems of K columns each in one
// cooperative launch on st, in the precision of o (each problem's own
// tolerances and caps come with its item).  The sum of the items' blocks
// must not exceed fj_pack_capacity.  bars: device scratch of 64 * count
// bytes.
fj_status fj_solve_packed_device(int K, int count, const PackItem* items, cudaStream_t st, const fj_opts& o,
                                 char* bars) {
  if (count < 1 || count > kPackMax) {
    set_error("internal: %d problems in one packed launch (1..%d)", count, kPackMax);
    return FJ_ERR_ARG;
  }
  const int mode = o.precision == FJ_PREC_FP64 ? kModeFP64 : (o.precision == FJ_PREC_FP32 ? kModeFP32 : kModeMixed);
#define FJ_PACK(KK)                                                                   \
  return mode == kModeFP64 ? launch_packed<double, KK>(count, items, st, o, mode, bars) \
                           : launch_packed<float, KK>(count, items, st, o, mode, bars);
  switch (K) {
    case 32: FJ_PACK(32)
    case 16: FJ_PACK(16)
    case 8: FJ_PACK(8)
    case 4: FJ_PACK(4)
    case 2: FJ_PACK(2)
    default: FJ_PACK(1)
  }
#undef FJ_PACK
}

// ------------------------------------------------- allocation-free solve
//
// fj_solve_fixed runs the same solve kernel as fj_solve_ex, but takes all of
// its scratch (solver vectors, reduction slots, status words, quantities)
// from one fixed array compiled into the library instead of allocating it.
// It exists for callers that must not allocate device memory during a solve:
// code driving a latency-critical loop (cudaMalloc and cudaFree can
// synchronize the whole device), and programs whose device memory is owned
// by another allocator.  The array is FJ_FIXED_SCRATCH_BYTES per device, is
// created when the library's solver code is loaded on a device and stays
// until the process exits.

namespace {

static __device__ __align__(256) unsigned char g_fixed_scratch[FJ_FIXED_SCRATCH_BYTES];

constexpr int kFixedMaxDevices = 64;
std::mutex g_fixed_mu;
void* g_fixed_addr[kFixedMaxDevices];  // device address of g_fixed_scratch, per device

// Host code cannot use g_fixed_scratch's name as a device address: look the
// address up once per device, with that device current.
fj_status fixed_scratch_address(int device, char** out) {
  if (device < 0 || device >= kFixedMaxDevices) {
    set_error("fj_solve_fixed: device %d out of range", device);
    return FJ_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_fixed_mu);
  if (!g_fixed_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fj_solve_fixed: cudaGetSymbolAddress");
    g_fixed_addr[device] = p;
  }
  *out = (char*)g_fixed_addr[device];
  return FJ_OK;
}

}  // namespace

extern "C" fj_status fj_solve_fixed(const fj_graph* g, void* stream, int32_t k, const double* s, double* z,
                                    fj_quant* quant, const fj_opts* opts, fj_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!g || !s || k < 1 || k > 32) {
    set_error("fj_solve_fixed: graph and s must be non-NULL and 1 <= k <= 32 (k=%d)", (int)k);
    return FJ_ERR_ARG;
  }
  fj_opts o;
  fj_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.inner_tol >= 1.0 || o.max_iter < 1 ||
      o.max_refine < 1 || o.precision < 0 || o.precision > 2 || (o.flags & FJ_TWO_SOLVES) ||
      ((o.flags & FJ_QUANTITY_TOL) && o.precision == FJ_PREC_FP32)) {
    set_error("fj_solve_fixed: invalid options (FJ_TWO_SOLVES is for fj_solve_ex; FJ_QUANTITY_TOL needs MIXED or FP64)");
    return FJ_ERR_ARG;
  }
  FJ_CUDA(cudaSetDevice(g->device));
  // s and z are read and written by the kernel directly: they must be device
  // (or managed) memory of the graph's device (the query allocates nothing)
  for (const void* ptr : {(const void*)s, (const void*)z}) {
    if (!ptr) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
      cudaGetLastError();
      a.type = cudaMemoryTypeUnregistered;
    }
    if (!((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == g->device)) {
      set_error("fj_solve_fixed: s and z must be device memory of device %d (opts->flags is ignored)",
                g->device);
      return FJ_ERR_ARG;
    }
  }
  int num_sms = 0;
  FJ_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, g->device));
  // launches of 32/16/8/4/2/1 columns, as in fj_solve_ex
  int Ks[6], launches = 0;
  for (int col = 0; col < k;) {
    int K = 32;
    while (K > k - col) K >>= 1;
    Ks[launches++] = K;
    col += K;
  }
  const int inner_bytes = o.precision == FJ_PREC_FP64 ? 8 : 4;
  size_t ws_need = 0;
  for (int i = 0; i < launches; ++i)
    ws_need = std::max(ws_need, fj_solve_workspace_bytes(g, Ks[i], inner_bytes, num_sms));
  // scratch layout: quantities [k][5] | residuals [k] | status [launches][3] | solver workspace
  const size_t head = 4096;
  if (ws_need > FJ_FIXED_SCRATCH_BYTES - head) {
    set_error("fj_solve_fixed: this solve needs %zu bytes of scratch, the fixed area holds %zu; use "
              "fj_solve_ex",
              ws_need + head, (size_t)FJ_FIXED_SCRATCH_BYTES);
    return FJ_ERR_ARG;
  }
  char* base = nullptr;
  fj_status rc = fixed_scratch_address(g->device, &base);
  if (rc != FJ_OK) return rc;
  double* dq = (double*)base;
  double* dres = dq + 32 * 5;
  int* dstat = (int*)(dres + 32);
  cudaStream_t st = (cudaStream_t)stream;
  FJ_CUDA(cudaMemsetAsync(dstat, 0, sizeof(int) * 3 * 6, st));
  fj_opts od = o;
  od.flags = FJ_DEVICE_PTRS | (o.flags & FJ_QUANTITY_TOL);
  int done = 0, grid = 0;
  rc = fj_solve_device(g, st, num_sms, k, s, z, dq, dres, dstat, base + head, FJ_FIXED_SCRATCH_BYTES - head, od,
                       &done, 0, nullptr, &grid);
  if (rc != FJ_OK) return rc;
  double hq[32 * 5], hres[32];
  int hstat[3 * 6];
  FJ_CUDA(cudaMemcpyAsync(hq, dq, sizeof(double) * 5 * k, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaMemcpyAsync(hres, dres, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaMemcpyAsync(hstat, dstat, sizeof(int) * 3 * launches, cudaMemcpyDeviceToHost, st));
  FJ_CUDA(cudaStreamSynchronize(st));
  int bits = 0, iters = 0, refines = 0;
  for (int i = 0; i < launches; ++i) {
    bits |= hstat[3 * i];
    iters = std::max(iters, hstat[3 * i + 1]);
    refines = std::max(refines, hstat[3 * i + 2]);
  }
  if (quant) memcpy(quant, hq, sizeof(double) * 5 * k);
  rc = FJ_OK;
  if (bits & kErrTimeout) {
    set_error("a device-side wait timed out (solve abandoned)");
    rc = FJ_ERR_TIMEOUT;
  } else if (bits & kErrNumeric) {
    set_error("NaN or Inf met in the iteration");
    rc = FJ_ERR_NUMERIC;
  } else if (bits & kErrNotConverged) {
    set_error("iteration caps reached before the residual target");
    rc = FJ_ERR_NOT_CONVERGED;
  }
  if (info) {
    double worst = 0.0;
    for (int j = 0; j < k; ++j) worst = std::max(worst, hres[j]);
    info->iterations = iters;
    info->refinements = refines;
    info->rel_residual = worst;
    info->status = rc;
    info->columns = k;
    info->blocks = grid;
    info->warnings = (bits & kWarnOpinionRange) ? FJ_WARN_OPINION_RANGE : 0u;
  }
  return rc;
}
