// fj_internal.cuh - shared device/host definitions of libfj (not installed).
//
// Data layout of one graph in device memory.  Nodes are renumbered in order
// of decreasing degree ("solver order"; perm maps back to input ids), which
// puts the hubs first and lets rows of similar length share a slice.
//   row_ptr/col/val  CSR of the off-diagonal part of L in solver order,
//                    each row's entries in input-edge order
//   dinv             1 / (1 + d_i), the Jacobi preconditioner
//   rows [0, n_long) with more than kSellMaxLen entries ("long rows") are cut
//                    into chunks of at most kChunkLen entries
//   rows [n_long, n_nz) are stored as sliced ELL (rows [n_nz, n) have no
//                    entries): slices of 32 consecutive rows,
//                    column-major inside a slice (entry p of the slice's lane
//                    l at slice_off + 32 p + l), padded with col = own row
//   unit_prefix      cumulative cost of the work units (chunks, then slices)
//                    used to split every SpMV evenly over the warps
// The diagonal 1 + d_i of I + L is never stored: (I + L) x is evaluated as
// x_i + sum_j w_ij (x_i - x_j), the edge form of L = B^T W B (Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fj.h"

namespace fj {

// Extra elements after the sort buffers and col/val (batched loads past the
// last entry stay inside the allocation).
constexpr int kPad = 64;
// Default layout: rows with at most kSellMaxLen entries go to sliced ELL;
// longer rows are processed warp-wide in chunks of at most kChunkLen
// entries.  Both are per graph (fj_set_layout, fj_tune_layout); the sliced
// ELL threshold is at most kSellMaxLenLimit (the repeated-pair check of short
// rows handles rows of up to 64 entries).
constexpr int kSellMaxLen = 64;
constexpr int kChunkLen = 512;
constexpr int kSellMaxLenLimit = 64;
struct Layout {
  int32_t chunk_len = kChunkLen;
  int32_t sell_max = kSellMaxLen;
};
// Degree keys of the reordering sort saturate here (16-bit keys: two radix
// passes).  Rows are ordered by falling degree, except that rows of degree
// >= kDegKeyMax come first and keep their input order among themselves; so
// the rows of several chunks (degree > chunk length) form a prefix together
// with those.
constexpr int kDegKeyMax = 65535;

// Error bits raised by device code.
enum : int {
  kErrBadId = 1,
  kErrBadWeight = 2,
  kErrTimeout = 4,
  kErrNumeric = 8,
  kErrNotConverged = 16,
  kErrDuplicate = 32,
  kWarnOpinionRange = 64,  // not an error: some s_i outside [0, 1]
};

struct Barrier {
  unsigned count;
  unsigned gen;
};

}  // namespace fj

struct fj_graph {
  int device;
  int64_t n;
  int64_t nnz;
  int weighted;
  // CSR in solver order
  int32_t* row_ptr;
  int32_t* col;
  float* val;
  float* dinv;
  int32_t* perm;  // perm[i] = input id of solver node i
  int32_t* orig_ids;  // for an extracted component: node id in the parent graph (else null)
  // long rows [0, n_long) in chunks; rows [n_nz, n) have no entries
  int64_t n_long;
  int64_t n_nz;
  int64_t n_chunks;
  int32_t* long_first;   // [n_long + 1] first chunk of each long row
  int32_t* chunk_row;    // [n_chunks]
  int32_t* chunk_begin;  // [n_chunks]
  int32_t* chunk_end;    // [n_chunks]
  // sliced ELL of rows [n_long, n)
  int64_t n_slices;
  int64_t sell_nnz;
  int64_t* slice_off;  // [n_slices + 1]
  int32_t* sell_col;
  float* sell_val;  // absent for unit weights
  // work units: chunks, then slices
  int64_t n_units;
  int64_t* unit_prefix;  // [n_units + 1]
  // layout parameters the graph was built with
  int32_t chunk_len;
  int32_t sell_max;
};

namespace fj {

// ------------------------------------------------------------------ device

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Streaming loads and stores (the .cs cache operator: lines allocated with
// evict-first priority in L1 and L2).  The SpMV walks stream the graph (col,
// val: read once per walk) and gather the iterate x; streaming the graph and
// the vectors of the update pass keeps the gathered rows of x, loaded and
// stored normally, in L2 while everything else passes through.

// Read-only data of the whole kernel (the graph): non-coherent path.
__device__ __forceinline__ int32_t ld_ro(const int32_t* a) {
  int32_t v;
  asm volatile("ld.global.cs.nc.b32 %0, [%1];" : "=r"(v) : "l"(a));
  return v;
}
__device__ __forceinline__ float ld_ro(const float* a) {
  float v;
  asm volatile("ld.global.cs.nc.f32 %0, [%1];" : "=f"(v) : "l"(a));
  return v;
}

// Data written by the kernel itself (vectors): coherent loads and stores.
__device__ __forceinline__ void ld_cs(const float* a, float& v) {
  asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(v) : "l"(a));
}
__device__ __forceinline__ void ld_cs(const double* a, double& v) {
  asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(a));
}
__device__ __forceinline__ void ld_cs(const float2* a, float2& v) {
  asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(a));
}
__device__ __forceinline__ void ld_cs(const float4* a, float4& v) {
  asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a));
}
__device__ __forceinline__ void ld_cs(const double2* a, double2& v) {
  asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(a));
}
template <typename T>
__device__ __forceinline__ T ld_cs(const T* a) {
  T v;
  ld_cs(a, v);
  return v;
}
__device__ __forceinline__ void st_cs(float* a, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cs(double* a, double v) {
  asm volatile("st.global.cs.f64 [%0], %1;" ::"l"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cs(float2* a, float2 v) {
  asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(v.x), "f"(v.y) : "memory");
}

}  // namespace fj

// ------------------------------------------------------------------- host

namespace fj {
// One problem of a packed solve launch (several small problems of the same
// column count K in one cooperative launch): K columns of opinions on a
// graph, all device pointers.
struct PackItem {
  const fj_graph* g;
  const double* s;  // column 0 of the K columns; column c at s + c * ld
  int64_t ld;
  double* z;        // same layout as s, or null
  double* quant;    // [K][5]
  double* resid;    // [K]
  int* status;      // [3]: error bits, iterations, refinements
  char* ws;         // workspace of fj_solve_workspace_bytes(g, K, ...)
  size_t ws_bytes;
  int blocks;       // blocks of the problem's share of the launch
  fj_opts opts;     // the problem's tolerances and caps (the launch's
                    // precision is the same for all its problems)
};
// Stream-ordered allocation from the library's memory pool of the current
// device.  The pool keeps freed memory for reuse (its release threshold is
// unlimited), so repeated uploads and solves do not map and unmap pages.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t st);
// Returns the pool's unused memory to the system (fj_destroy).
void pool_trim(int device);
template <typename T>
inline cudaError_t malloc_async(T** p, size_t bytes, cudaStream_t st) {
  return pool_malloc_async(reinterpret_cast<void**>(p), bytes, st);
}
void set_error(const char* fmt, ...);
// Counts kernel launches made by the library (all contexts, this process).
void count_launches(int k);
fj_status cuda_fail(cudaError_t e, const char* what);
// Context internals shared by the C-ABI files (defined in fj_api.cpp).
fj_status ctx_device(fj_ctx* c, int* device, int* num_sms, cudaStream_t* st);
fj_status ctx_scratch(fj_ctx* c, int which, size_t bytes, char** out);
}  // namespace fj

#define FJ_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return fj::cuda_fail(e_, #call);     \
  } while (0)
