// Shared helpers of the inrct CUDA library (error state, launch checks, small math).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cstdarg>

#include "../../include/inrct.h"

namespace inrct {

// Thread-local message of the last failing call (read by inrct_last_error()).
void set_error(const char* fmt, ...);
void clear_error();

// Kernel launches issued by this library (all threads).
void count_launch();

// Optional stage marks of grad_step (a CUDA event recorded at each mark while a
// profile is active; see inrct_profile_begin / inrct_profile_end).
enum ProfMark {
  kMarkStart = 0,    // grad_step entry
  kMarkEvalKernel,   // before the grid-evaluation MLP kernel
  kMarkEvalDone,     // after it
  kMarkProjDone,     // after projection + loss
  kMarkBackDone,     // after backprojection (and the ramp filter)
  kMarkVjpKernel,    // before the VJP MLP kernel
  kMarkVjpKernelDone,
  kMarkVjpDone,      // after the weight-gradient GEMM and reductions
  kMarkEnd,          // after Adam
  kNumMarks
};
void prof_mark(int mark, cudaStream_t st);

#define INRCT_REQUIRE(cond, ...)            \
  do {                                      \
    if (!(cond)) {                          \
      ::inrct::set_error(__VA_ARGS__);      \
      return INRCT_ERR_INVALID_ARG;         \
    }                                       \
  } while (0)

// Checks the launch just issued and counts it (inrct_launch_count()).
#define INRCT_CHECK_LAUNCH(what)                                                   \
  do {                                                                             \
    ::inrct::count_launch();                                                       \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      ::inrct::set_error("%s: %s", what, cudaGetErrorString(e_));                  \
      return INRCT_ERR_CUDA;                                                       \
    }                                                                              \
  } while (0)

#define INRCT_TRY(expr)           \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != INRCT_OK) return rc_; \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves aligned sub-buffers out of the caller's workspace, in order.
struct Carver {
  char* base;
  size_t cap;
  size_t off = 0;
  bool ok = true;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count, size_t align = 256) {
    off = align_up(off, align);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    if (off > cap) ok = false;
    return p;
  }
};

inline int64_t grid_points(const inrct_grid* g) {
  int64_t n = 1;
  for (int k = 0; k < g->d; k++) n *= g->N;
  return n;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Grid point i inside the field of view (inscribed disk / cylinder along z):
// (2 k_x + 1 - N)^2 + (2 k_y + 1 - N)^2 <= N^2, exact in 64-bit integers.
__host__ __device__ inline bool in_fov(int64_t i, int N) {
  const int64_t a = 2 * (i % N) + 1 - N, b = 2 * ((i / N) % N) + 1 - N;
  return a * a + b * b <= (int64_t)N * N;
}

}  // namespace inrct
