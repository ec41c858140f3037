// The coarse tail of the V-cycle in one thread-block cluster.
//
// Below a few thousand cells a colour class holds too little work to fill the
// GPU, and one kernel launch per class is dominated by its start-up and by
// chains of dependent loads.  The levels from `first` down to the coarsest
// therefore run inside a single cluster of CTAs (one per SM) whose phases
// are separated by hardware cluster barriers: forward block-GS sweeps, the
// residual, the restriction, the coarsest solve, then the backward sweeps
// with the prolongation folded in -- the same arithmetic as the per-class
// kernels, in the same order.
//
// Every CTA of the cluster executes the same sequence of barriers: all loop
// bounds below depend only on the level descriptors, never on the thread,
// and no thread leaves the kernel early.
#pragma once

#include <cooperative_groups.h>

#include "ll_kernels.cuh"

namespace llmg {

constexpr int kTailThreads = 256;  // per CTA
constexpr int kTailMaxColours = 64;

template <typename T, typename TM>
struct TailLevel {
  int n = 0, ncol = 0;
  int cs[kTailMaxColours + 1] = {0};  // colour class starts
  const int* rowptr = nullptr;
  const int* diag = nullptr;
  const int* col = nullptr;
  const TM* val = nullptr;
  const T* dinv = nullptr;
  T* x = nullptr;
  T* b = nullptr;
  T* r = nullptr;
  const int* agg = nullptr;   // this level -> next level
  const int* mptr = nullptr;  // members of this level's cells in the finer level
  const int* mem = nullptr;
};

template <typename T, typename TM>
struct TailArgs {
  int first = 0, last = 0;  // tail levels [first, last]; last is the coarsest
  int nu_pre = 1, nu_post = 1;
  int N = 0;                       // unknowns of the coarsest level
  const double* ainv = nullptr;    // its inverse, column-major
  TailLevel<T, TM> L[kMaxLevels];
};

__device__ __forceinline__ void tail_sync() {
  __threadfence();  // make this phase's global writes visible cluster-wide
  cooperative_groups::this_cluster().sync();
}

// one colour class of level L with G lanes per row, spread over the cluster
template <typename T, typename TM, int G, int MODE>
__device__ __forceinline__ void tail_sweep(const TailLevel<T, TM>& L, int t, const T* e, long tid, long nthreads) {
  int r0 = L.cs[t], r1 = L.cs[t + 1];
  long work = (long)(r1 - r0) * G;
  for (long base = 0; base < work; base += nthreads) {  // uniform trip count
    long g = base + tid;
    int I = r0 + (int)(g / G);
    sweep_row<T, TM, G, MODE>(I, (int)(g % G), g < work, L.rowptr, L.diag, L.col, L.val, L.dinv, L.b, L.x, L.agg,
                              e);
  }
}

template <typename T, typename TM, int G>
__global__ void __launch_bounds__(kTailThreads) k_coarse_tail(const TailArgs<T, TM>* __restrict__ args) {
  const TailArgs<T, TM>& A = *args;
  long nthreads = (long)gridDim.x * blockDim.x;  // the grid is one cluster
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  // ---- down: pre-smoothing, residual, restriction
  for (int l = A.first; l < A.last; ++l) {
    const TailLevel<T, TM>& L = A.L[l];
    const TailLevel<T, TM>& N = A.L[l + 1];
    int K = L.ncol;
    if (A.nu_pre == 0) {
      for (long i = tid; i < 3L * L.n; i += nthreads) L.x[i] = (T)0;
      tail_sync();
    }
    for (int sweep = 0; sweep < A.nu_pre; ++sweep)
      for (int t = sweep == 0 ? 1 : 0; t < K; ++t) {  // colour 0 was written by the restriction
        if (sweep == 0) tail_sweep<T, TM, G, 0>(L, t, nullptr, tid, nthreads);
        else tail_sweep<T, TM, G, 1>(L, t, nullptr, tid, nthreads);
        tail_sync();
      }
    int skip_from = A.nu_pre >= 1 ? L.cs[K - 1] : L.n;
    long work = (long)skip_from * G;
    for (long base = 0; base < work; base += nthreads) {
      long g = base + tid;
      residual_row<T, TM, G>((int)(g / G), (int)(g % G), g < work, L.rowptr, L.col, L.val, L.b, L.x, L.r);
    }
    tail_sync();
    int init_end = (A.nu_pre >= 1 && l + 1 < A.last) ? N.cs[1] : 0;
    for (long I = tid; I < N.n; I += nthreads)
      restrict_row<T>((int)I, N.mptr, N.mem, skip_from, L.r, N.b, init_end, N.dinv, N.x);
    tail_sync();
  }
  // ---- coarsest: x = A^{-1} b
  {
    const TailLevel<T, TM>& C = A.L[A.last];
    for (long i = tid; i < A.N; i += nthreads) {
      double acc = 0.0;
      for (int j = 0; j < A.N; ++j) acc += A.ainv[(long)j * A.N + i] * (double)C.b[j];
      C.x[i] = (T)acc;
    }
    tail_sync();
  }
  // ---- up: backward sweeps with the prolongation folded into the first
  for (int l = A.last - 1; l >= A.first; --l) {
    const TailLevel<T, TM>& L = A.L[l];
    const TailLevel<T, TM>& N = A.L[l + 1];
    int K = L.ncol;
    if (A.nu_post == 0) {
      for (long I = tid; I < L.n; I += nthreads) {
        long a = 3L * L.agg[I];
        L.x[3 * I] += N.x[a];
        L.x[3 * I + 1] += N.x[a + 1];
        L.x[3 * I + 2] += N.x[a + 2];
      }
      tail_sync();
    }
    for (int sweep = 0; sweep < A.nu_post; ++sweep)
      for (int k = 0; k < K; ++k) {
        if (sweep == 0) tail_sweep<T, TM, G, 2>(L, K - 1 - k, N.x, tid, nthreads);
        else tail_sweep<T, TM, G, 1>(L, K - 1 - k, nullptr, tid, nthreads);
        tail_sync();
      }
  }
}

}  // namespace llmg
