// fj_internal.cuh - shared device/host definitions of libfj (not installed).
//
// Data layout in device memory (one graph):
//   row_ptr  int32[n+1]      CSR row starts of the off-diagonal part of L
//   col      int32[nnz+pad]  neighbour ids, rows in input-edge order
//   val      float[nnz+pad]  edge weights w_ij (absent for unit weights)
//   dinv     float[n]        1 / (1 + d_i), the Jacobi preconditioner
//   tile_row int32[NT+1]     merge-path row coordinate of every tile start
// The diagonal 1 + d_i of I + L is never stored: (I + L) x is evaluated as
// x_i + sum_j w_ij (x_i - x_j), the edge form of L = B^T W B (Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fj.h"

namespace fj {

// Merge-path items (row ends + nonzeros) per warp tile.
constexpr int kTileItems = 256;
// Extra zeroed elements after col/val so that staging loads of the last tile
// never leave the allocation.
constexpr int kPad = 64;

// Error bits raised by device code.
enum : int {
  kErrBadId = 1,
  kErrBadWeight = 2,
  kErrTimeout = 4,
  kErrNumeric = 8,
  kErrNotConverged = 16,
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
  int64_t n_tiles;
  int weighted;
  int32_t* row_ptr;
  int32_t* col;
  float* val;
  float* dinv;
  int32_t* tile_row;
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

// Largest r in [lo, hi] with f(r) = row_ptr[r] + r <= d (merge-path split of
// diagonal d between the row-end list and the nonzero list).
__device__ __forceinline__ int64_t merge_path_row(const int32_t* row_ptr,
                                                  int64_t n, int64_t d) {
  int64_t lo = 0, hi = n;
  if (hi > d) hi = d;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)row_ptr[mid] + mid <= d)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

}  // namespace fj

// ------------------------------------------------------------------- host

namespace fj {
void set_error(const char* fmt, ...);
fj_status cuda_fail(cudaError_t e, const char* what);
}  // namespace fj

#define FJ_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return fj::cuda_fail(e_, #call);     \
  } while (0)
