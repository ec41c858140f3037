// The coarse tail of the V-cycle in one thread-block cluster.
//
// Below a few thousand cells a colour class holds too little work to fill the
// GPU, and one kernel launch per class is dominated by its start-up and by
// chains of dependent loads.  The levels from `first` down to the coarsest
// therefore run inside a single cluster of CTAs (one per SM) whose phases
// are separated by hardware cluster barriers: forward block-GS sweeps, the
// residual, the restriction, the coarsest solve, the prolongation, then the
// backward sweeps -- the same arithmetic as the per-class kernels, in the
// same order.
//
// Every CTA of the cluster executes the same sequence of barriers: all loop
// bounds below depend only on the level descriptors, never on the thread,
// and no thread leaves the kernel early.
#pragma once

#include <cooperative_groups.h>

#include "ll_kernels.cuh"

namespace llmg {

constexpr int kTailThreads = 256;  // per CTA
// blocks per lane loaded before the products, a fixed unroll here (the
// per-class kernels choose a warp-uniform one).  Float64: 2, since slots past
// a row's blocks still issue their multiply-adds under predication and the
// float64 pipe is slow (unroll 4: 0.59 ms of tail per GCR iteration at 128^3,
// unroll 2: 0.55 ms); float32 keeps 4 loads in flight per lane.
template <typename T> constexpr int kTailUnroll = 4;
template <> constexpr int kTailUnroll<double> = 2;

// levels below this many rows use 8 lanes per row: their classes leave most
// of the cluster's threads idle, and wider rows shorten each phase's chain
constexpr int kTailWideRows = 4096;
constexpr int kTailMaxColours = 64;

template <typename T, typename TM>
struct TailLevel {
  int n = 0, ncol = 0, nnzb = 0, nmem = 0;
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
  // batches (union hierarchies): the dense solves of the instances whose
  // coarsest level this is (their rows follow the colour classes); ucptr
  // holds the running sum of their sizes N (nuc + 1 entries)
  int nuc = 0;
  const CoarseTask* uc = nullptr;
  const int* ucptr = nullptr;
};

template <typename T, typename TM>
struct TailArgs {
  int first = 0, last = 0;  // tail levels [first, last]; last is the coarsest
  int solo_first = 0;       // levels [solo_first, last] run on the cluster's first CTA alone
  int nu_pre = 1, nu_post = 1;
  int N = 0;                       // unknowns of the coarsest level
  const double* ainv = nullptr;    // its inverse, column-major
  bool uni = false;                // a batch's union: dense solves per instance (TailLevel::uc)
  TailLevel<T, TM> L[kMaxLevels];
};

// The cluster barrier's arrive has release and its wait acquire semantics at
// cluster scope, for global memory as for shared: every thread of the
// cluster sees the writes of the phase before, so no separate fence is
// needed (a __threadfence() here measured 2.5 % slower tail phases).
__device__ __forceinline__ void tail_sync() { cooperative_groups::this_cluster().sync(); }

// barrier between the phases: the whole cluster, or one CTA
struct ClusterPhase {
  __device__ void operator()() const { tail_sync(); }
};
struct CtaPhase {
  __device__ void operator()() const { __syncthreads(); }
};

// one colour class of level L with G lanes per row, spread over the threads
template <typename T, typename TM, int G, int MODE>
__device__ __forceinline__ void tail_sweep(const TailLevel<T, TM>& L, int t, long tid, long nthreads) {
  int r0 = L.cs[t], r1 = L.cs[t + 1];
  long work = (long)(r1 - r0) * G;
  for (long base = 0; base < work; base += nthreads) {  // uniform trip count
    long g = base + tid;
    int I = r0 + (int)(g / G);
    sweep_row<T, TM, G, MODE, kTailUnroll<T>, -1>(I, (int)(g % G), g < work, L.rowptr, L.diag, L.col, L.val, L.dinv,
                                               L.b, L.x);
  }
}

// x = A_i^{-1} b for every instance i whose coarsest level L is (a batch's
// union), one unknown of one instance per thread; the same sums in the same
// order as kc_solve_batch.  Nothing in L's own phases reads these rows: their
// x is first read by the prolongation into the level above.
template <typename T, typename TM>
__device__ __forceinline__ void tail_union_coarse(const TailLevel<T, TM>& L, long tid, long nthreads) {
  if (L.nuc == 0) return;
  long total = L.ucptr[L.nuc];
  for (long w = tid; w < total; w += nthreads) {
    int lo = 0, hi = L.nuc - 1;  // the task holding unknown w
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (L.ucptr[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    CoarseTask t = L.uc[lo];
    int i = (int)(w - L.ucptr[lo]);
    const T* bb = L.b + 3L * t.row0;
    double acc = 0.0;
    for (int j = 0; j < t.N; ++j) acc += ro(t.ainv + (long)j * t.N + i) * (double)bb[j];
    L.x[3L * t.row0 + i] = (T)acc;
  }
}

// pre-smoothing, residual and restriction of level l
template <typename T, typename TM, int G, typename Sync>
__device__ __forceinline__ void tail_down(const TailArgs<T, TM>& A, int l, long tid, long nthreads, Sync sync) {
  const TailLevel<T, TM>& L = A.L[l];
  const TailLevel<T, TM>& N = A.L[l + 1];
  tail_union_coarse(L, tid, nthreads);
  int K = L.ncol;
  if (A.nu_pre == 0) {
    for (long i = tid; i < 3L * L.n; i += nthreads) L.x[i] = (T)0;
    sync();
  }
  for (int sweep = 0; sweep < A.nu_pre; ++sweep)
    for (int t = sweep == 0 ? 1 : 0; t < K; ++t) {  // colour 0 was written by the restriction
      if (sweep == 0) tail_sweep<T, TM, G, 0>(L, t, tid, nthreads);
      else tail_sweep<T, TM, G, 1>(L, t, tid, nthreads);
      sync();
    }
  int skip_from = A.nu_pre >= 1 ? L.cs[K - 1] : L.n;
  long work = (long)skip_from * G;
  for (long base = 0; base < work; base += nthreads) {
    long g = base + tid;
    if (A.nu_pre == 1)  // right after one forward sweep: the higher colours' part only
      residual_row<T, TM, G, true, kTailUnroll<T>, -1>((int)(g / G), (int)(g % G), g < work, L.rowptr, L.diag,
                                                    L.col, L.val, L.b, L.x, L.r);
    else
      residual_row<T, TM, G, false, kTailUnroll<T>, -1>((int)(g / G), (int)(g % G), g < work, L.rowptr, L.diag,
                                                     L.col, L.val, L.b, L.x, L.r);
  }
  sync();
  int init_end = (A.nu_pre >= 1 && l + 1 < A.last) ? N.cs[1] : 0;
  for (long I = tid; I < N.n; I += nthreads)
    restrict_row<T>((int)I, N.mptr, N.mem, skip_from, L.r, N.b, init_end, N.dinv, N.x);
  sync();
}

// coarsest: x = A^{-1} b (a union: every instance's own dense solve)
template <typename T, typename TM, typename Sync>
__device__ __forceinline__ void tail_coarsest(const TailArgs<T, TM>& A, long tid, long nthreads, Sync sync) {
  const TailLevel<T, TM>& C = A.L[A.last];
  if (A.uni) {
    tail_union_coarse(C, tid, nthreads);
    sync();
    return;
  }
  for (long i = tid; i < A.N; i += nthreads) {
    double acc = 0.0;
    for (int j = 0; j < A.N; ++j) acc += ro(A.ainv + (long)j * A.N + i) * (double)C.b[j];
    C.x[i] = (T)acc;
  }
  sync();
}

// the prolongation x += P e (one phase: folded into the first backward sweep
// it measured 0.8 % slower per step), then the backward sweeps of level l
template <typename T, typename TM, int G, typename Sync>
__device__ __forceinline__ void tail_up(const TailArgs<T, TM>& A, int l, long tid, long nthreads, Sync sync) {
  const TailLevel<T, TM>& L = A.L[l];
  const TailLevel<T, TM>& N = A.L[l + 1];
  int K = L.ncol;
  for (long I = tid; I < L.n; I += nthreads) {
    int a = L.agg[I];
    if (a < 0) continue;  // a batch's padding rows
    L.x[3 * I] += N.x[3L * a];
    L.x[3 * I + 1] += N.x[3L * a + 1];
    L.x[3 * I + 2] += N.x[3L * a + 2];
  }
  sync();
  for (int sweep = 0; sweep < A.nu_post; ++sweep)
    for (int k = 0; k < K; ++k) {
      tail_sweep<T, TM, G, 1>(L, K - 1 - k, tid, nthreads);
      sync();
    }
}

// Ask L2 for the bytes [p, p + bytes) (128-byte lines, spread over the
// threads); nothing waits for them.
__device__ __forceinline__ void l2_prefetch(const void* p, long bytes, long tid, long nthreads) {
  const char* c = (const char*)p;
  for (long o = tid * 128; o < bytes; o += nthreads * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// The operators and transfers of the tail levels are read once per V-cycle
// and the fine levels' traffic in between evicts them from L2, so each
// phase would wait for DRAM on its first loads.  One prefetch of all of
// them at the start overlaps those misses.
template <typename T, typename TM>
__device__ void tail_prefetch(const TailArgs<T, TM>& A, long tid, long nthreads) {
  for (int l = A.first; l <= A.last; ++l) {
    const TailLevel<T, TM>& L = A.L[l];
    l2_prefetch(L.rowptr, (L.n + 1) * 4L, tid, nthreads);
    l2_prefetch(L.diag, L.n * 4L, tid, nthreads);
    l2_prefetch(L.col, L.nnzb * 4L, tid, nthreads);
    l2_prefetch(L.val, L.nnzb * 9L * (long)sizeof(TM), tid, nthreads);
    l2_prefetch(L.dinv, L.n * 9L * (long)sizeof(T), tid, nthreads);
    if (l < A.last) l2_prefetch(L.agg, L.n * 4L, tid, nthreads);
    if (l > A.first) {
      l2_prefetch(L.mptr, (L.n + 1) * 4L, tid, nthreads);
      l2_prefetch(L.mem, L.nmem * 4L, tid, nthreads);
    }
  }
  l2_prefetch(A.ainv, (long)A.N * A.N * 8, tid, nthreads);  // a union's inverses are read straight from memory
}

// The levels from `first` run on the whole cluster, phases separated by
// cluster barriers.  The smallest levels (from `solo_first`) hold only a few
// hundred rows: there a phase is latency, and the first CTA runs them alone
// with CTA barriers, which cost far less than cluster-wide ones, while the
// other CTAs wait at the next cluster barrier.
// One CTA per SM by construction (one cluster of CTAs on distinct SMs), so the
// compiler may use the whole register file (avoids spills in float32).
template <typename T, typename TM, int G>
__global__ void __launch_bounds__(kTailThreads, 1) k_coarse_tail(const TailArgs<T, TM>* __restrict__ args) {
  const TailArgs<T, TM>& A = *args;
  long nthreads = (long)gridDim.x * blockDim.x;  // the grid is one cluster
  long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  tail_prefetch(A, tid, nthreads);
  for (int l = A.first; l < A.solo_first && l < A.last; ++l) {
    if (A.L[l].n < kTailWideRows) tail_down<T, TM, 8>(A, l, tid, nthreads, ClusterPhase());
    else tail_down<T, TM, G>(A, l, tid, nthreads, ClusterPhase());
  }
  if (A.solo_first >= A.last) {
    tail_coarsest<T, TM>(A, tid, nthreads, ClusterPhase());
  } else {
    if (blockIdx.x == 0) {  // uniform per CTA; no cluster barrier inside
      long t = threadIdx.x, nt = blockDim.x;
      for (int l = A.solo_first; l < A.last; ++l) tail_down<T, TM, G>(A, l, t, nt, CtaPhase());
      tail_coarsest<T, TM>(A, t, nt, CtaPhase());
      for (int l = A.last - 1; l >= A.solo_first; --l) tail_up<T, TM, G>(A, l, t, nt, CtaPhase());
    }
    tail_sync();  // the first CTA's results, visible to the cluster
  }
  for (int l = (A.solo_first < A.last ? A.solo_first : A.last) - 1; l >= A.first; --l) {
    if (A.L[l].n < kTailWideRows) tail_up<T, TM, 8>(A, l, tid, nthreads, ClusterPhase());
    else tail_up<T, TM, G>(A, l, tid, nthreads, ClusterPhase());
  }
}

}  // namespace llmg
