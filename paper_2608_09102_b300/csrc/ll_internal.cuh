// Internal declarations of the sm_103a solver library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ll_mg.h"

namespace llmg {

// ---------------------------------------------------------------------------
// error handling: every CUDA call is checked; failures unwind as a status
// ---------------------------------------------------------------------------
struct Status {
  int code;
};
// records the failed call (error name, source line) for ll_last_cuda_error
void note_cuda_error(cudaError_t e, const char* file, int line);
// the same for a failed consistency check of the library's own results
void note_internal_error(const char* what, const char* file, int line);
#define LL_CU(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      ::llmg::note_cuda_error(e_, __FILE__, __LINE__);                \
      throw ::llmg::Status{e_ == cudaErrorMemoryAllocation ? LL_ENOMEM : LL_ECUDA}; \
    }                                                                 \
  } while (0)
// called after every kernel launch: checks it and counts it
void count_launch();
#define LL_LAUNCHED()              \
  do {                             \
    LL_CU(cudaGetLastError());     \
    ::llmg::count_launch();        \
  } while (0)

constexpr int kBlock = 256;
constexpr int kRedBlocks = 1184;  // 8 x 148 SMs: fixed grid of reduction kernels
constexpr int kMaxRestart = 64;
constexpr int kMaxColours = 128;
constexpr int kMaxLevels = 32;
constexpr int kRowLanes = 4;  // lanes per block row in the coarse-level kernels

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Device allocation owned by the hierarchy (freed in the destructor).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    LL_CU(cudaMalloc((void**)&p, count * sizeof(T)));
    n = count;
  }
  void zero(cudaStream_t s) { LL_CU(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
  operator T*() const { return p; }
};

// ---------------------------------------------------------------------------
// integer mixing: the MurmurHash3 32-bit finaliser (a published function)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
// tie-break key of the undirected edge {lo, hi}
__host__ __device__ __forceinline__ uint32_t pair_key(uint32_t lo, uint32_t hi, uint32_t seed) {
  return mix32((lo * 2654435761u) ^ hi ^ seed);
}
// colouring priority of node v
__host__ __device__ __forceinline__ uint32_t node_key(uint32_t v, uint32_t seed) {
  return mix32((v * 2654435761u) ^ seed ^ 0x5bd1e995u);
}

// ---------------------------------------------------------------------------
// graphs and levels
// ---------------------------------------------------------------------------
// batched solves: the dense solve of one instance whose coarsest level is
// reached (its rows start at union row row0; N = 3 x cells), and one element
// range [e0, e1) of one instance's part of a union vector
struct CoarseTask {
  int row0, N;
  const double* ainv;
};
struct Chunk {
  int inst;
  long e0, e1;
};

struct DevGraph {  // CSR, no self loops, integer weights
  int n = 0;
  int nnz = 0;
  DBuf<int> rowptr, col, w;
};

// Red-black ("checkerboard") storage of grid fields: colour c = (x+y+z)&1,
// slot = c*Nh + (z*ny + y)*nxh + (x>>1), nxh = ceil(nx/2), Nh = nxh*ny*nz.
// Slots past the end of a row (odd nx) are padding and stay zero.
struct GridGeom {
  int nx, ny, nz, nxh;
  long nh;  // slots per colour
  long n;   // real cells
};

}  // namespace llmg
