// Device kernels of the numeric setup, the V-cycle and the GCR iteration.
// Included by ll_solver.cu only.
#pragma once
#include <type_traits>

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

#include "ll_internal.cuh"

namespace llmg {

// ---------------------------------------------------------------------------
// red-black slot geometry of level 0
// ---------------------------------------------------------------------------
struct SlotPos {
  int x, y, z;
  long row;
  bool real;
};
__device__ __forceinline__ SlotPos slot_pos(const GridGeom& g, int c, long r) {
  SlotPos p;
  int i = (int)(r % g.nxh);
  p.row = r / g.nxh;
  p.y = (int)(p.row % g.ny);
  p.z = (int)(p.row / g.ny);
  p.x = 2 * i + ((c + p.y + p.z) & 1);
  p.real = p.x < g.nx;
  return p;
}

// visit(slot) for each face neighbour (all of the other colour), in the order
// of slot_neighbours; returns the count.  No index array: an array indexed
// in a loop lives in local memory, and each neighbour's load would then wait
// for the one before it.
template <typename V>
__device__ __forceinline__ int for_neighbours(const GridGeom& g, int c, const SlotPos& p, V&& visit) {
  long base = (long)(1 - c) * g.nh;
  long row = p.row * g.nxh;
  int d = 0;
  if (p.z > 0) visit(base + row - (long)g.ny * g.nxh + (p.x >> 1)), ++d;
  if (p.y > 0) visit(base + row - g.nxh + (p.x >> 1)), ++d;
  if (p.x > 0) visit(base + row + ((p.x - 1) >> 1)), ++d;
  if (p.x < g.nx - 1) visit(base + row + ((p.x + 1) >> 1)), ++d;
  if (p.y < g.ny - 1) visit(base + row + g.nxh + (p.x >> 1)), ++d;
  if (p.z < g.nz - 1) visit(base + row + (long)g.ny * g.nxh + (p.x >> 1)), ++d;
  return d;
}

// slots of the face neighbours (all of the other colour); returns the count
__device__ __forceinline__ int slot_neighbours(const GridGeom& g, int c, const SlotPos& p, long* s) {
  long base = (long)(1 - c) * g.nh;
  long row = p.row * g.nxh;
  int d = 0;
  if (p.z > 0) s[d++] = base + row - (long)g.ny * g.nxh + (p.x >> 1);
  if (p.y > 0) s[d++] = base + row - g.nxh + (p.x >> 1);
  if (p.x > 0) s[d++] = base + row + ((p.x - 1) >> 1);
  if (p.x < g.nx - 1) s[d++] = base + row + ((p.x + 1) >> 1);
  if (p.y < g.ny - 1) s[d++] = base + row + g.nxh + (p.x >> 1);
  if (p.z < g.nz - 1) s[d++] = base + row + (long)g.ny * g.nxh + (p.x >> 1);
  return d;
}

// ---------------------------------------------------------------------------
// 3x3 helpers (row-major blocks)
// ---------------------------------------------------------------------------
// inverse by the adjugate; returns false for a zero or non-finite determinant
__host__ __device__ __forceinline__ bool inv3(const double* a, double* o) {
  double c00 = a[4] * a[8] - a[5] * a[7];
  double c01 = a[5] * a[6] - a[3] * a[8];
  double c02 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(det != 0.0) || !isfinite(det)) return false;
  double id = 1.0 / det;
  o[0] = c00 * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[3] = c01 * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[6] = c02 * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}

// the same inverse in float32 (the mixed path's Galerkin levels)
__device__ __forceinline__ bool inv3(const float* a, float* o) {
  float c00 = a[4] * a[8] - a[5] * a[7];
  float c01 = a[5] * a[6] - a[3] * a[8];
  float c02 = a[3] * a[7] - a[4] * a[6];
  float det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(det != 0.0f) || !isfinite(det)) return false;
  float id = 1.0f / det;
  o[0] = c00 * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[3] = c01 * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[6] = c02 * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

// float32 inverse of a 3x3 matrix (row-major) by cofactors
__device__ __forceinline__ void inv3f(const float* a, float* o) {
  float c00 = a[4] * a[8] - a[5] * a[7];
  float c01 = a[5] * a[6] - a[3] * a[8];
  float c02 = a[3] * a[7] - a[4] * a[6];
  float id = 1.0f / (a[0] * c00 + a[1] * c01 + a[2] * c02);
  o[0] = c00 * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[3] = c01 * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[6] = c02 * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

// Level-0 coefficients of the float32 V-cycle formed in the kernels from m~
// (12 bytes per slot) instead of read as C(m~)/h^2 and D^-1 (72 bytes): the
// float32 level-0 kernels are bound by memory, not by float32 arithmetic.
// m32 holds m~ per slot, SoA [3][2 Nh]; the numeric setup writes it (and
// checks in float64 that every D is invertible).
struct OnFly {
  const float* m32;
  float alpha, ih2, inv_dt;
};
// C(m~)/h^2 of slot sl, C(m) = [m]x + alpha (m m^T - |m|^2 I), row-major
__device__ __forceinline__ void onfly_c(const OnFly& q, long sl, long n2, float* C) {
  float m1 = ld(q.m32 + sl), m2 = ld(q.m32 + n2 + sl), m3 = ld(q.m32 + 2 * n2 + sl);
  float s = m1 * m1 + m2 * m2 + m3 * m3, a = q.alpha;
  C[0] = a * (m1 * m1 - s);
  C[1] = -m3 + a * m1 * m2;
  C[2] = m2 + a * m1 * m3;
  C[3] = m3 + a * m2 * m1;
  C[4] = a * (m2 * m2 - s);
  C[5] = -m1 + a * m2 * m3;
  C[6] = -m2 + a * m3 * m1;
  C[7] = m1 + a * m3 * m2;
  C[8] = a * (m3 * m3 - s);
#pragma unroll
  for (int e = 0; e < 9; ++e) C[e] *= q.ih2;
}
// D^-1 = (I/dt - deg C(m~)/h^2)^-1 from C as onfly_c gives it
__device__ __forceinline__ void onfly_dinv(const OnFly& q, const float* C, int deg, float* Di) {
  float D[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) D[e] = -(float)deg * C[e];
  D[0] += q.inv_dt;
  D[4] += q.inv_dt;
  D[8] += q.inv_dt;
  inv3f(D, Di);
}

// ---------------------------------------------------------------------------
// numeric setup, level 0: per slot C(m~)/h^2 and the inverse of the diagonal
// block I/dt - deg C(m~)/h^2.  C(m) = [m]_x + alpha (m m^T - |m|^2 I)  (the
// component form of the damped scheme, Sec. 2.1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k0_coef(GridGeom g, const double* __restrict__ m, double alpha, double dt, double ih2,
                        double* __restrict__ chat64, T* __restrict__ chat, T* __restrict__ dinv,
                        int* __restrict__ bad, float* __restrict__ m32 = nullptr,
                        float* __restrict__ chat_lo = nullptr) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Di[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (p.real) {
    long k = p.x + (long)g.nx * (p.y + (long)g.ny * p.z);
    double m1 = m[k], m2 = m[g.n + k], m3 = m[2 * g.n + k];
    double s = m1 * m1 + m2 * m2 + m3 * m3;
    C[0] = alpha * (m1 * m1 - s);
    C[1] = -m3 + alpha * m1 * m2;
    C[2] = m2 + alpha * m1 * m3;
    C[3] = m3 + alpha * m2 * m1;
    C[4] = alpha * (m2 * m2 - s);
    C[5] = -m1 + alpha * m2 * m3;
    C[6] = -m2 + alpha * m3 * m1;
    C[7] = m1 + alpha * m3 * m2;
    C[8] = alpha * (m3 * m3 - s);
    int deg = (p.x > 0) + (p.x < g.nx - 1) + (p.y > 0) + (p.y < g.ny - 1) + (p.z > 0) + (p.z < g.nz - 1);
    double D[9];
    for (int e = 0; e < 9; ++e) {
      C[e] *= ih2;
      D[e] = -deg * C[e];
    }
    D[0] += 1.0 / dt;
    D[4] += 1.0 / dt;
    D[8] += 1.0 / dt;
    if (!inv3(D, Di)) atomicExch(bad, 1);
  }
  for (int e = 0; e < 9; ++e) {
    if (chat64) chat64[e * n2 + sl] = C[e];
    if (chat) chat[e * n2 + sl] = (T)C[e];
    if (dinv) dinv[e * n2 + sl] = (T)Di[e];
    // C = chat + chat_lo to about 2^-48 (chat = C rounded to float32)
    if (chat_lo) chat_lo[e * n2 + sl] = (float)(C[e] - (double)(float)C[e]);
  }
  if (m32) {  // m~ per slot for the float32 kernels that form C and D^-1 themselves
    long k = p.real ? p.x + (long)g.nx * (p.y + (long)g.ny * p.z) : 0;
    for (int q = 0; q < 3; ++q) m32[q * n2 + sl] = p.real ? (float)m[q * g.n + k] : 0.0f;
  }
}

// ---------------------------------------------------------------------------
// numeric Galerkin products (Eq. galerkin), accumulated in T: float64 for the
// float64 path, float32 for the mixed path's float32 preconditioner (its
// coarse operators are stored in float32 or bfloat16 anyway; float64 sums
// there cost the float64 pipe, which bounds these kernels)
// ---------------------------------------------------------------------------
// row of every block of a BSR level
__global__ void k_block_rows(int n, const int* __restrict__ rowptr, int* __restrict__ prow) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int p = rowptr[I]; p < rowptr[I + 1]; ++p) prow[p] = I;
}

// One thread per coarse block: neighbouring threads write neighbouring
// blocks (coalesced stores), or, with perm, the blocks in the order perm (by
// decreasing slot-list length, ties by index: the lanes of a warp sum lists
// of about the same length).  Each block sums its slot list in a fixed order.
// The diagonal blocks' inverses are a separate pass (k_block_dinv): inside
// this kernel only about one lane in 13 holds a diagonal block, and the warp
// would issue the inverse's float64 instructions for all 32 lanes.
// level 1: A_1(I,J) = delta_IJ |G_I|/dt I + sum_{k in G_I} w_kJ Chat_k
template <typename T>
__global__ void k_galerkin_l1_blk(int nnzb, const int* __restrict__ perm, const int* __restrict__ prow,
                                  const int* __restrict__ col, const int* __restrict__ sptr,
                                  const int* __restrict__ sidx, const int* __restrict__ sw,
                                  const int* __restrict__ mptr, long n2, const T* __restrict__ chat, T inv_dt,
                                  T* __restrict__ val) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  int p = perm ? perm[t] : t;
  int I = prow[p];
  T a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int q = sptr[p]; q < sptr[p + 1]; ++q) {
    long k = sidx[q];
    T w = (T)sw[q];
    for (int e = 0; e < 9; ++e) a[e] += w * chat[e * n2 + k];
  }
  if (col[p] == I) {
    T sz = (T)(mptr[I + 1] - mptr[I]) * inv_dt;
    a[0] += sz;
    a[4] += sz;
    a[8] += sz;
  }
  for (int e = 0; e < 9; ++e) val[9 * (long)p + e] = a[e];
}

// levels >= 2: sum of the fine blocks of each coarse slot
template <typename T>
__global__ void k_galerkin_bsr_blk(int nnzb, const int* __restrict__ perm, const int* __restrict__ sptr,
                                   const int* __restrict__ sidx, const T* __restrict__ fval, T* __restrict__ val) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  int p = perm ? perm[t] : t;
  T a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int q = sptr[p]; q < sptr[p + 1]; ++q) {
    const T* f = fval + 9 * (long)sidx[q];
    for (int e = 0; e < 9; ++e) a[e] += f[e];
  }
  for (int e = 0; e < 9; ++e) val[9 * (long)p + e] = a[e];
}

// inverse of every diagonal block of a Galerkin level, one thread per row;
// a singular block sets *bad
template <typename T>
__global__ void k_block_dinv(int n, const int* __restrict__ diag, const T* __restrict__ val, T* __restrict__ dinv,
                             int* __restrict__ bad) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const T* d = val + 9 * (long)diag[I];
  T a[9], o[9];
  for (int e = 0; e < 9; ++e) a[e] = d[e];
  if (!inv3(a, o)) atomicExch(bad, 1);
  for (int e = 0; e < 9; ++e) dinv[9 * (long)I + e] = o[e];
}

// float32 -> bfloat16 (round to nearest even)
__global__ void k_cast_bf16(long n, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// ---------------------------------------------------------------------------
// coarsest level: dense LU with partial pivoting (one CTA), unknown 3I + c
// ---------------------------------------------------------------------------
template <typename TV>
__global__ void k_dense_from_bsr(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const TV* __restrict__ val, double* __restrict__ a) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int N = 3 * n;
  for (int r = 0; r < 3; ++r)
    for (int j = 0; j < N; ++j) a[(long)(3 * I + r) * N + j] = 0.0;
  for (int p = rowptr[I]; p < rowptr[I + 1]; ++p) {
    int J = col[p];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) a[(long)(3 * I + r) * N + 3 * J + c] = (double)val[9 * (long)p + 3 * r + c];
  }
}

// In place: a = L\U (unit L), perm[i] = original row now in position i.
__global__ void k_lu_factor(int N, double* __restrict__ a, int* __restrict__ perm, int* __restrict__ status) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  __shared__ int piv;
  int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < N; i += nt) perm[i] = i;
  if (t == 0) *status = 0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    // pivot search: largest |a_ik|, ties to the lowest row
    double bv = -1.0;
    int bi = N;
    for (int i = k + t; i < N; i += nt) {
      double v = fabs(a[(long)i * N + k]);
      if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
      }
    }
    sval[t] = bv;
    sidx[t] = bi;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (t < o) {
        double v2 = sval[t + o];
        int i2 = sidx[t + o];
        if (v2 > sval[t] || (v2 == sval[t] && i2 < sidx[t])) {
          sval[t] = v2;
          sidx[t] = i2;
        }
      }
      __syncthreads();
    }
    if (t == 0) {
      piv = sidx[0];
      if (!(sval[0] > 0.0)) *status = 1;
    }
    __syncthreads();
    int p = piv;
    if (p != k && p < N) {
      for (int j = t; j < N; j += nt) {
        double x = a[(long)k * N + j];
        a[(long)k * N + j] = a[(long)p * N + j];
        a[(long)p * N + j] = x;
      }
      if (t == 0) {
        int x = perm[k];
        perm[k] = perm[p];
        perm[p] = x;
      }
    }
    __syncthreads();
    double akk = a[(long)k * N + k];
    for (int i = k + 1 + t; i < N; i += nt) a[(long)i * N + k] /= akk;
    __syncthreads();
    int m = N - k - 1;
    for (long e = t; e < (long)m * m; e += nt) {
      int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      a[(long)i * N + j] -= a[(long)i * N + k] * a[(long)k * N + j];
    }
    __syncthreads();
  }
}

// Coarsest inverse for up to kGjMax unknowns: in-place Gauss-Jordan
// elimination with partial pivoting on one thread-block cluster of P CTAs.
// Column j of the matrix lives in the shared memory of CTA j % P at local
// column j / P, one warp per local column, lanes over rows.  The warp holding
// column k finds the pivot row p (largest |a_ik| over i >= k, ties to the
// lowest row, as in k_lu_factor), publishes p, column k with rows k and p
// exchanged and the pivot's reciprocal in its CTA's shared memory, and sets
// its own column to e_p.  After a cluster barrier every warp reads them
// through distributed shared memory and applies step k to its column: rows k
// and p exchanged, row k times the reciprocal, f_i times row k subtracted from
// every other row i.  The warp holding column k + 1 publishes step k + 1 right
// after its own update of step k, while the other warps are still updating,
// so each step costs one barrier.  Column k then holds a column of the inverse
// with its rows in pivot order; undoing the row exchanges in reverse order on
// the columns puts the inverse in order.  N^3 multiply-adds spread over P SMs.
// The published column is double-buffered: step k + 2 is published after the
// barrier that ends step k's reads.  a: row-major N x N; ainv: column-major;
// *status = 1 on a zero or non-finite pivot.
constexpr int kGjMax = 256;               // at most 32 local columns (warps) per CTA
constexpr int kGjRows = kGjMax / 32;      // rows per lane

// pivot search and publication of step k by the warp holding column k
__device__ __forceinline__ void gj_publish(int N, int k, double* colv, double* pub, int* pubp, int lane,
                                           int* status) {
  const int buf = k & 1;
  double bv = -1.0;
  int bi = N;
  for (int i = k + lane; i < N; i += 32) {  // rows ascending per lane: the first maximum
    double v = fabs(colv[i]);
    if (v > bv) {
      bv = v;
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
    int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 > bv || (v2 == bv && i2 < bi)) {
      bv = v2;
      bi = i2;
    }
  }
  int p = bi;
  if (!(bv > 0.0) || !isfinite(bv)) {
    if (lane == 0) atomicExch(status, 1);
    p = k;
  }
  double* f = pub + buf * (N + 1);
  for (int i = lane; i < N; i += 32) f[i] = colv[i == k ? p : (i == p ? k : i)];
  if (lane == 0) {
    f[N] = 1.0 / colv[p];
    pubp[buf] = p;
  }
  __syncwarp();
  for (int i = lane; i < N; i += 32) colv[i] = i == p ? 1.0 : 0.0;
  __syncwarp();
}

__global__ void __launch_bounds__(1024, 1) k_gj_inverse(int N, const double* __restrict__ a,
                                                        double* __restrict__ ainv, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks(), r = (int)cl.block_rank();
  const int W = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ double gj_sm[];
  double* colv = gj_sm + (size_t)w * N;  // this warp's column
  double* pub = gj_sm + (size_t)W * N;   // 2 x (N + 1): column k, then 1 / pivot
  __shared__ int pubp[2];
  __shared__ int pivs[kGjMax];
  __shared__ int dest[kGjMax];
  __shared__ int q[kGjMax];
  const int j = w * P + r;
  const bool have = j < N;
  if (have)
    for (int i = lane; i < N; i += 32) colv[i] = a[(long)i * N + j];
  if (r == 0 && threadIdx.x == 0) *status = 0;
  cl.sync();  // status cleared before any pivot can set it
  if (j == 0) gj_publish(N, 0, colv, pub, pubp, lane, status);
  cl.sync();
  for (int k = 0; k < N; ++k) {
    const int buf = k & 1, o = k % P;
    const double* f = cl.map_shared_rank(pub + buf * (N + 1), o);
    const int p = *cl.map_shared_rank(&pubp[buf], o);
    if (threadIdx.x == 0) pivs[k] = p;
    if (have) {
      // every remote load issued before the first use; row blocks past N
      // skipped whole (a masked float64 instruction costs as much as a full one)
      double fr[kGjRows];
#pragma unroll
      for (int t = 0; t < kGjRows; ++t) {
        if (32 * t >= N) break;
        fr[t] = lane + 32 * t < N ? f[lane + 32 * t] : 0.0;
      }
      double ip = f[N];
      if (lane == 0 && p != k) {
        double t = colv[k];
        colv[k] = colv[p];
        colv[p] = t;
      }
      __syncwarp();
      double rk = colv[k] * ip;
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kGjRows; ++t) {
        if (32 * t >= N) break;
        int i = lane + 32 * t;
        if (i < N) colv[i] = i == k ? rk : colv[i] - fr[t] * rk;
      }
      __syncwarp();
      if (j == k + 1) gj_publish(N, k + 1, colv, pub, pubp, lane, status);
    }
    cl.sync();
  }
  cl.sync();  // no CTA leaves while another may still read its published column
  if (threadIdx.x == 0) {
    // q[jj]: the column that ends as column jj of the inverse (the row
    // exchanges undone on the columns in reverse order); dest: its inverse map
    for (int jj = 0; jj < N; ++jj) q[jj] = jj;
    for (int k = N - 1; k >= 0; --k) {
      int t = q[k];
      q[k] = q[pivs[k]];
      q[pivs[k]] = t;
    }
    for (int jj = 0; jj < N; ++jj) dest[q[jj]] = jj;
  }
  __syncthreads();
  if (have)
    for (int i = lane; i < N; i += 32) ainv[(long)dest[j] * N + i] = colv[i];
}

// Columns of the inverse from the LU factors: column j solves L U x = P e_j
// (one thread per column, the column itself as workspace), stored
// column-major: ainv[j*N + i] = (A^{-1})_ij.
__global__ void k_lu_inverse(int N, const double* __restrict__ a, const int* __restrict__ perm,
                             double* __restrict__ ainv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    double* y = ainv + (long)j * N;
    for (int i = 0; i < N; ++i) {  // forward, unit lower; (P e_j)_i = [perm_i == j]
      double v = perm[i] == j ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= a[(long)i * N + k] * y[k];
      y[i] = v;
    }
    for (int i = N - 1; i >= 0; --i) {  // backward
      double v = y[i];
      for (int k = i + 1; k < N; ++k) v -= a[(long)i * N + k] * y[k];
      y[i] = v / a[(long)i * N + i];
    }
  }
}

// x = A^{-1} b with the column-major inverse; b staged in shared memory
template <typename T>
__global__ void kc_solve(int N, const double* __restrict__ ainv, const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ double sb[];
  for (int j = threadIdx.x; j < N; j += blockDim.x) sb[j] = (double)b[j];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int j = 0; j < N; ++j) acc += ainv[(long)j * N + i] * sb[j];
  x[i] = (T)acc;
}

// ---------------------------------------------------------------------------
// level-0 V-cycle kernels (red-black slots, matrix free)
// ---------------------------------------------------------------------------
// Block Gauss-Seidel update of the cells of colour c:
//   x_k = Dinv_k (b_k - Chat_k S_k),  S_k = sum of the neighbours' x.
// mode 0: neighbours are zero (first half-sweep from x = 0);
// mode 1: plain update.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k0_smooth(GridGeom g, int c, const double* __restrict__ b, T* __restrict__ x,
                                                 const T* __restrict__ chat, const T* __restrict__ dinv) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= g.nh) return;
  long n2 = 2 * g.nh;
  long sl = (long)c * g.nh + r;
  SlotPos p = slot_pos(g, c, r);
  if (!p.real) return;
  T v0 = (T)b[sl], v1 = (T)b[n2 + sl], v2 = (T)b[2 * n2 + sl];
  if (MODE != 0) {
    T s0 = 0, s1 = 0, s2 = 0;
    for_neighbours(g, c, p, [&](long l) {
      s0 += x[l];
      s1 += x[n2 + l];
      s2 += x[2 * n2 + l];
    });
    const T* C = chat + sl;
    T c0 = ld(C), c1 = ld(C + n2), c2 = ld(C + 2 * n2), c3 = ld(C + 3 * n2), c4 = ld(C + 4 * n2),
      c5 = ld(C + 5 * n2), c6 = ld(C + 6 * n2), c7 = ld(C + 7 * n2), c8 = ld(C + 8 * n2);
    v0 = fma(-c0, s0, v0);
    v0 = fma(-c1, s1, v0);
    v0 = fma(-c2, s2, v0);
    v1 = fma(-c3, s0, v1);
    v1 = fma(-c4, s1, v1);
    v1 = fma(-c5, s2, v1);
    v2 = fma(-c6, s0, v2);
    v2 = fma(-c7, s1, v2);
    v2 = fma(-c8, s2, v2);
  }
  const T* D = dinv + sl;
  T d0 = ld(D), d1 = ld(D + n2), d2 = ld(D + 2 * n2), d3 = ld(D + 3 * n2), d4 = ld(D + 4 * n2),
    d5 = ld(D + 5 * n2), d6 = ld(D + 6 * n2), d7 = ld(D + 7 * n2), d8 = ld(D + 8 * n2);
  x[sl] = d0 * v0 + d1 * v1 + d2 * v2;
  x[n2 + sl] = d3 * v0 + d4 * v1 + d5 * v2;
  x[2 * n2 + sl] = d6 * v0 + d7 * v1 + d8 * v2;
}

// operator at one slot: y = x/dt + Chat (S - deg x), S = sum of neighbours
template <typename T, typename TX>
__device__ __forceinline__ void slot_apply(const GridGeom& g, int c, long sl, const SlotPos& p, const TX* x,
                                           const T* chat, T inv_dt, T* y) {
  long n2 = 2 * g.nh;
  T x0 = (T)x[sl], x1 = (T)x[n2 + sl], x2 = (T)x[2 * n2 + sl];
  T s0 = 0, s1 = 0, s2 = 0;
  int d = for_neighbours(g, c, p, [&](long l) {
    s0 += (T)x[l];
    s1 += (T)x[n2 + l];
    s2 += (T)x[2 * n2 + l];
  });
  T fd = (T)d;
  s0 -= fd * x0;
  s1 -= fd * x1;
  s2 -= fd * x2;
  const T* C = chat + sl;
  y[0] = x0 * inv_dt + ld(C) * s0 + ld(C + n2) * s1 + ld(C + 2 * n2) * s2;
  y[1] = x1 * inv_dt + ld(C + 3 * n2) * s0 + ld(C + 4 * n2) * s1 + ld(C + 5 * n2) * s2;
  y[2] = x2 * inv_dt + ld(C + 6 * n2) * s0 + ld(C + 7 * n2) * s1 + ld(C + 8 * n2) * s2;
}

// residual of one slot: r = b - x/dt - Chat (S - deg x), negated FMAs
template <typename T, typename TX>
__device__ __forceinline__ void slot_residual(const GridGeom& g, int c, long sl, const SlotPos& p, const double* b,
                                              const TX* x, const T* chat, T inv_dt, T* r) {
  long n2 = 2 * g.nh;
  T x0 = (T)x[sl], x1 = (T)x[n2 + sl], x2 = (T)x[2 * n2 + sl];
  T s0 = 0, s1 = 0, s2 = 0;
  int d = for_neighbours(g, c, p, [&](long l) {
    s0 += (T)x[l];
    s1 += (T)x[n2 + l];
    s2 += (T)x[2 * n2 + l];
  });
  T fd = (T)d;
  s0 = fma(-fd, x0, s0);
  s1 = fma(-fd, x1, s1);
  s2 = fma(-fd, x2, s2);
  const T* C = chat + sl;
  T r0 = fma(-inv_dt, x0, (T)b[sl]), r1 = fma(-inv_dt, x1, (T)b[n2 + sl]), r2 = fma(-inv_dt, x2, (T)b[2 * n2 + sl]);
  r0 = fma(-ld(C), s0, r0);
  r0 = fma(-ld(C + n2), s1, r0);
  r0 = fma(-ld(C + 2 * n2), s2, r0);
  r1 = fma(-ld(C + 3 * n2), s0, r1);
  r1 = fma(-ld(C + 4 * n2), s1, r1);
  r1 = fma(-ld(C + 5 * n2), s2, r1);
  r2 = fma(-ld(C + 6 * n2), s0, r2);
  r2 = fma(-ld(C + 7 * n2), s1, r2);
  r2 = fma(-ld(C + 8 * n2), s2, r2);
  r[0] = r0;
  r[1] = r1;
  r[2] = r2;
}

// Residual and restriction (P^T) in one pass: bc_I = sum over the members k
// of aggregate I of (b - A x)_k.  After a forward half-sweep of colour 1 the
// colour-1 residuals vanish, so only the colour-0 members are listed.
// Residual of a colour-0 cell right after one forward red-black sweep from
// x = 0: the cell was solved with its neighbours (all colour 1) still zero,
// so b_k - D_k x_k = 0 and only the neighbours' later update remains:
//   r_k = - C^_k sum_{j ~ k} x_j   (exact up to rounding).
template <typename T>
__device__ __forceinline__ void slot_residual_after_sweep(const GridGeom& g, long sl, const SlotPos& p,
                                                          const T* x, const T* chat, T* r) {
  long n2 = 2 * g.nh;
  T s0 = 0, s1 = 0, s2 = 0;
  for_neighbours(g, 0, p, [&](long l) {
    s0 += x[l];
    s1 += x[n2 + l];
    s2 += x[2 * n2 + l];
  });
  const T* C = chat + sl;
  r[0] = -(ld(C) * s0 + ld(C + n2) * s1 + ld(C + 2 * n2) * s2);
  r[1] = -(ld(C + 3 * n2) * s0 + ld(C + 4 * n2) * s1 + ld(C + 5 * n2) * s2);
  r[2] = -(ld(C + 6 * n2) * s0 + ld(C + 7 * n2) * s1 + ld(C + 8 * n2) * s2);
}

// k0_smooth for the float32 V-cycle with the coefficients formed from m~
// (OnFly); the same operations in the same order once C and D^-1 are formed
template <int MODE>
__global__ void __launch_bounds__(256) k0_smooth_onfly(GridGeom g, int c, const double* __restrict__ b,
                                                       float* __restrict__ x, OnFly q) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= g.nh) return;
  long n2 = 2 * g.nh;
  long sl = (long)c * g.nh + r;
  SlotPos p = slot_pos(g, c, r);
  if (!p.real) return;
  float v0 = (float)b[sl], v1 = (float)b[n2 + sl], v2 = (float)b[2 * n2 + sl];
  float C[9];
  onfly_c(q, sl, n2, C);
  int deg = (p.x > 0) + (p.x < g.nx - 1) + (p.y > 0) + (p.y < g.ny - 1) + (p.z > 0) + (p.z < g.nz - 1);
  if (MODE != 0) {
    float s0 = 0, s1 = 0, s2 = 0;
    for_neighbours(g, c, p, [&](long l) {
      s0 += x[l];
      s1 += x[n2 + l];
      s2 += x[2 * n2 + l];
    });
    v0 = fmaf(-C[0], s0, v0);
    v0 = fmaf(-C[1], s1, v0);
    v0 = fmaf(-C[2], s2, v0);
    v1 = fmaf(-C[3], s0, v1);
    v1 = fmaf(-C[4], s1, v1);
    v1 = fmaf(-C[5], s2, v1);
    v2 = fmaf(-C[6], s0, v2);
    v2 = fmaf(-C[7], s1, v2);
    v2 = fmaf(-C[8], s2, v2);
  }
  float D[9];
  onfly_dinv(q, C, deg, D);
  x[sl] = D[0] * v0 + D[1] * v1 + D[2] * v2;
  x[n2 + sl] = D[3] * v0 + D[4] * v1 + D[5] * v2;
  x[2 * n2 + sl] = D[6] * v0 + D[7] * v1 + D[8] * v2;
}

// The float32 V-cycle's colour-0 residual right after one forward sweep
// (slot_residual_after_sweep, C formed from m~) and its restriction in one
// kernel, thread t taking aggregate order[t]; for I < init_end also the
// first colour of the next level's forward sweep
__global__ void k0_restrict_onfly(GridGeom g, const float* __restrict__ x, OnFly q, int nc,
                                  const int* __restrict__ mptr, const int* __restrict__ mem, float* __restrict__ bc,
                                  int init_end, const float* __restrict__ dinvc, float* __restrict__ xc,
                                  const int* __restrict__ order) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  int I = order[t];
  long n2 = 2 * g.nh;
  float a0 = 0, a1 = 0, a2 = 0;
  for (int qm = mptr[I]; qm < mptr[I + 1]; ++qm) {
    long sl = mem[qm];
    SlotPos p = slot_pos(g, 0, sl % g.nh);
    float s0 = 0, s1 = 0, s2 = 0;
    for_neighbours(g, 0, p, [&](long l) {
      s0 += x[l];
      s1 += x[n2 + l];
      s2 += x[2 * n2 + l];
    });
    float C[9];
    onfly_c(q, sl, n2, C);
    a0 += -(C[0] * s0 + C[1] * s1 + C[2] * s2);
    a1 += -(C[3] * s0 + C[4] * s1 + C[5] * s2);
    a2 += -(C[6] * s0 + C[7] * s1 + C[8] * s2);
  }
  bc[3L * I] = a0;
  bc[3L * I + 1] = a1;
  bc[3L * I + 2] = a2;
  if (I < init_end) {  // first colour of the next level's forward sweep
    const float* D = dinvc + 9L * I;
    xc[3L * I] = D[0] * a0 + D[1] * a1 + D[2] * a2;
    xc[3L * I + 1] = D[3] * a0 + D[4] * a1 + D[5] * a2;
    xc[3L * I + 2] = D[6] * a0 + D[7] * a1 + D[8] * a2;
  }
}

// Residual and restriction in one kernel (after nu_pre >= 2 sweeps):
// bc_I = sum over the members k of aggregate I of b_k - (A x)_k
template <typename T>
__global__ void k0_restrict(GridGeom g, const double* __restrict__ b, const T* __restrict__ x,
                            const T* __restrict__ chat, T inv_dt, int nc, const int* __restrict__ mptr,
                            const int* __restrict__ mem, T* __restrict__ bc, int init_end,
                            const T* __restrict__ dinvc, T* __restrict__ xc, const int* __restrict__ order) {
  // thread t takes aggregate order[t]: neighbouring threads take neighbouring
  // aggregates of the grid, so their member cells share cache lines
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  int I = order[t];
  T a0 = 0, a1 = 0, a2 = 0;
  for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
    long sl = mem[q];
    int c = (int)(sl / g.nh);
    SlotPos p = slot_pos(g, c, sl % g.nh);
    T r[3];
    slot_residual<T, T>(g, c, sl, p, b, x, chat, inv_dt, r);
    a0 += r[0];
    a1 += r[1];
    a2 += r[2];
  }
  bc[3L * I] = a0;
  bc[3L * I + 1] = a1;
  bc[3L * I + 2] = a2;
  if (I < init_end) {  // first colour of the next level's forward sweep
    const T* D = dinvc + 9L * I;
    xc[3L * I] = D[0] * a0 + D[1] * a1 + D[2] * a2;
    xc[3L * I + 1] = D[3] * a0 + D[4] * a1 + D[5] * a2;
    xc[3L * I + 2] = D[6] * a0 + D[7] * a1 + D[8] * a2;
  }
}

// The residual of the colour-0 cells right after one forward sweep
// (slot_residual_after_sweep), one thread per colour-0 slot, into the
// colour-0 part r0 of a red-black vector (3 x nh, component-major): every
// load is by slot, so the entry-major coefficients are read coalesced.
template <typename T>
__global__ void k0_residual_c0(GridGeom g, const T* __restrict__ x, const T* __restrict__ chat,
                               T* __restrict__ r0) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= g.nh) return;
  SlotPos p = slot_pos(g, 0, sl);
  T r[3] = {0, 0, 0};
  if (p.real) slot_residual_after_sweep<T>(g, sl, p, x, chat, r);
  r0[sl] = r[0];
  r0[g.nh + sl] = r[1];
  r0[2 * g.nh + sl] = r[2];
}

// restriction of that residual: bc_I = sum over the colour-0 members of
// aggregate I (mptr0 / mem0); for I < init_end, xc_I = Dinvc_I bc_I (the
// first colour of the next level's forward sweep).  Thread t takes aggregate
// order[t], as k0_restrict.
template <typename T>
__global__ void k0_restrict_c0(GridGeom g, const T* __restrict__ r0, int nc, const int* __restrict__ mptr,
                               const int* __restrict__ mem, T* __restrict__ bc, int init_end,
                               const T* __restrict__ dinvc, T* __restrict__ xc, const int* __restrict__ order) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  int I = order[t];
  T a0 = 0, a1 = 0, a2 = 0;
  for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
    long sl = mem[q];
    a0 += r0[sl];
    a1 += r0[g.nh + sl];
    a2 += r0[2 * g.nh + sl];
  }
  bc[3L * I] = a0;
  bc[3L * I + 1] = a1;
  bc[3L * I + 2] = a2;
  if (I < init_end) {
    const T* D = dinvc + 9L * I;
    xc[3L * I] = D[0] * a0 + D[1] * a1 + D[2] * a2;
    xc[3L * I + 1] = D[3] * a0 + D[4] * a1 + D[5] * a2;
    xc[3L * I + 2] = D[6] * a0 + D[7] * a1 + D[8] * a2;
  }
}

// restriction of b itself (no pre-smoothing: x = 0)
template <typename T>
__global__ void k0_restrict_b(GridGeom g, const double* __restrict__ b, int nc, const int* __restrict__ mptr,
                              const int* __restrict__ mem, T* __restrict__ bc) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  long n2 = 2 * g.nh;
  T a0 = 0, a1 = 0, a2 = 0;
  for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
    long sl = mem[q];
    a0 += (T)b[sl];
    a1 += (T)b[n2 + sl];
    a2 += (T)b[2 * n2 + sl];
  }
  bc[3L * I] = a0;
  bc[3L * I + 1] = a1;
  bc[3L * I + 2] = a2;
}

// x_k += e[agg(k)] on the real slots [first, first + count)
template <typename T>
__global__ void k0_prolong(GridGeom g, const int* __restrict__ agg, const T* __restrict__ e, T* __restrict__ x,
                           long first, long count) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (i >= count) return;
  long sl = first + i;
  int a = agg[sl];
  if (a < 0) return;
  x[sl] += e[3L * a];
  x[n2 + sl] += e[3L * a + 1];
  x[2 * n2 + sl] += e[3L * a + 2];
}

template <typename T>
__global__ void k_zero(long n, T* __restrict__ p) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = (T)0;
}

// ---------------------------------------------------------------------------
// coarse levels: 3x3 BSR, cell-major vectors; a group of G lanes per row
// ---------------------------------------------------------------------------
// Sums of a, b, c over the G lanes of each group, left in every lane of the
// group; every lane of the warp must call it.  Float64, G = 4 or 8: the
// first round leaves the partial sums of a and b in the lower half of the
// group and those of c in the upper half, the later rounds halve the values
// per lane again, and three shuffles gather the results.  That takes 4
// float64 adds per lane instead of the butterfly's 3 log2(G), on a pipe that
// retires 2 float64 operations per clock per SM here; the lanes are paired
// as in the butterfly, so the sums are the same bit for bit.
template <int G, typename T>
__device__ __forceinline__ void group_sum3(T& a, T& b, T& c) {
  constexpr unsigned kFull = 0xffffffffu;
  if constexpr (std::is_same<T, double>::value && (G == 4 || G == 8)) {
    int lane = threadIdx.x & 31, base = lane & ~(G - 1);
    bool hi = lane & (G / 2);
    double k0 = hi ? c : a, k1 = hi ? 0.0 : b;  // kept
    double s0 = hi ? a : c, s1 = hi ? b : 0.0;  // sent to the partner half
    k0 += __shfl_xor_sync(kFull, s0, G / 2);
    k1 += __shfl_xor_sync(kFull, s1, G / 2);
    if constexpr (G == 8) {
      bool m = lane & 2;  // a (lanes 0, 1), b (2, 3), c (4, 5), zero (6, 7)
      double kk = m ? k1 : k0, ss = m ? k0 : k1;
      kk += __shfl_xor_sync(kFull, ss, 2);
      kk += __shfl_xor_sync(kFull, kk, 1);
      a = __shfl_sync(kFull, kk, base);
      b = __shfl_sync(kFull, kk, base + 2);
      c = __shfl_sync(kFull, kk, base + 4);
    } else {  // a and b in lanes 0, 1; c in lanes 2, 3
      k0 += __shfl_xor_sync(kFull, k0, 1);
      k1 += __shfl_xor_sync(kFull, k1, 1);
      a = __shfl_sync(kFull, k0, base);
      b = __shfl_sync(kFull, k1, base);
      c = __shfl_sync(kFull, k0, base + 2);
    }
  } else {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      c += __shfl_xor_sync(kFull, c, o);
    }
  }
}

// widen a stored matrix value to the arithmetic type
template <typename T, typename TM>
__device__ __forceinline__ T widen(TM v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

// Loads of the operator, its structure and the transfers, which no kernel
// of a solve writes, go through the read-only data path: its cache lines
// survive the cluster barriers of the coarse tail (whose acquire side
// invalidates the coherent L1 lines), so a phase reads them from L1.
template <typename V>
__device__ __forceinline__ V ro(const V* p) {
  return __ldg(p);
}

// a -= A_IJ v  for one 3x3 block stored as TM (negated fused multiply-adds)
template <typename T, typename TM>
__device__ __forceinline__ void block_msub(const TM* __restrict__ A, T v0, T v1, T v2, T& a0, T& a1, T& a2) {
  a0 = fma(-widen<T, TM>(ro(A + 0)), v0, a0);
  a0 = fma(-widen<T, TM>(ro(A + 1)), v1, a0);
  a0 = fma(-widen<T, TM>(ro(A + 2)), v2, a0);
  a1 = fma(-widen<T, TM>(ro(A + 3)), v0, a1);
  a1 = fma(-widen<T, TM>(ro(A + 4)), v1, a1);
  a1 = fma(-widen<T, TM>(ro(A + 5)), v2, a1);
  a2 = fma(-widen<T, TM>(ro(A + 6)), v0, a2);
  a2 = fma(-widen<T, TM>(ro(A + 7)), v1, a2);
  a2 = fma(-widen<T, TM>(ro(A + 8)), v2, a2);
}

// a -= sum over the blocks p = p0, p0 + G, ... < p1 of A_p v_{col p}, with the
// column indices of U blocks loaded first, then their x values, then the
// products: two dependent memory round trips per U blocks instead of per
// block.
template <typename T, typename TM, int G, int U>
__device__ __forceinline__ void row_msub(int p0, int p1, const int* __restrict__ col, const TM* __restrict__ val,
                                         const T* __restrict__ x, T& a0, T& a1, T& a2) {
  for (int base = p0; base < p1; base += G * U) {
    int J[U];
#pragma unroll
    for (int u = 0; u < U; ++u) J[u] = base + u * G < p1 ? ro(col + base + u * G) : -1;
    T v[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (J[u] >= 0) {
        v[u][0] = x[3L * J[u]];
        v[u][1] = x[3L * J[u] + 1];
        v[u][2] = x[3L * J[u] + 2];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (J[u] >= 0) block_msub<T, TM>(val + 9L * (base + u * G), v[u][0], v[u][1], v[u][2], a0, a1, a2);
  }
}

// a -= sum over the off-diagonal blocks of row [p0, p1) with diagonal pd, in
// one lane-strided loop over the row's off-diagonal slots q (prefix then
// suffix, the diagonal skipped): a row visits ceil((p1 - p0 - 1) / G) slots
// instead of separate prefix and suffix loops.
template <typename T, typename TM, int G, int U>
__device__ __forceinline__ void row_msub_off(int p0, int pd, int p1, int lane, const int* __restrict__ col,
                                             const TM* __restrict__ val, const T* __restrict__ x, T& a0, T& a1,
                                             T& a2) {
  int npre = pd - p0, noff = p1 - p0 - 1;
  for (int base = lane; base < noff; base += G * U) {
    int J[U], P[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int q = base + u * G;
      P[u] = p0 + q + (q >= npre ? 1 : 0);
      J[u] = q < noff ? ro(col + P[u]) : -1;
    }
    T v[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (J[u] >= 0) {
        v[u][0] = x[3L * J[u]];
        v[u][1] = x[3L * J[u] + 1];
        v[u][2] = x[3L * J[u] + 2];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (J[u] >= 0) block_msub<T, TM>(val + 9L * P[u], v[u][0], v[u][1], v[u][2], a0, a1, a2);
  }
}

// Slots of one lane in a row's lane-strided range of n block slots.
template <int G>
__device__ __forceinline__ int lane_slots(int n, int lane) {
  return n > lane ? (n - lane + G - 1) / G : 0;
}
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// The unroll a warp uses in row_msub / row_msub_off: the largest slot count of
// its lanes, capped at U (0: no lane has a block).  With a fixed unroll, slots
// that no lane of the warp has still issue their multiply-adds under
// predication, and masked-off float64 instructions cost float64 pipe time as
// if they ran; that pipe (2 multiply-adds per clock per SM here) sets the pace
// of the float64 sweeps.  Every lane of the warp must call this.
template <int U>
__device__ __forceinline__ int warp_unroll(int n) {
  int m = __reduce_max_sync(0xffffffffu, n);
  return m < U ? m : U;
}

// f(std::integral_constant<int, UU>) with UU the smallest compiled unroll
// >= u: the unrolls 1, 2 and 3 are compiled where bit 0, 1 and 2 of USET are
// set, and U always.  u <= 0: nothing.
template <int U, int USET, typename F>
__device__ __forceinline__ void with_unroll(int u, F&& f) {
  if (u <= 0) return;
  if (USET > 0 && (USET & 1) && u == 1) f(std::integral_constant<int, cmin(U, 1)>{});
  else if (USET > 0 && (USET & 2) && u <= 2) f(std::integral_constant<int, cmin(U, 2)>{});
  else if (USET > 0 && (USET & 4) && u <= 3) f(std::integral_constant<int, cmin(U, 3)>{});
  else f(std::integral_constant<int, U>{});
}

// Block Gauss-Seidel update of one row of a colour class, G lanes per row.
// Coarse levels are renumbered so that each colour class is the contiguous
// row range [r0, r1), colours ascending, and every row's blocks are sorted by
// column: the columns of lower colours form the prefix [rowptr_I, diag_I),
// those of higher colours the suffix (diag_I, rowptr_{I+1}) (rows of one
// colour are not coupled).  Hence
//   MODE 0, forward sweep from x = 0: only the prefix (already updated) counts;
//   MODE 1, plain sweep: prefix and suffix, all current (the coarse
//           correction is added to x by a separate prolongation pass first).
// x_I = Dinv_I (b_I - sum_{J != I} A_IJ x_J); the lanes of a group share the
// three output components.  Every lane of the warp must call this (shuffles).
// sweep_row with the row's block range already loaded: p0 = rowptr_I,
// pd = diag_I, p1 = rowptr_{I+1}
template <typename T, typename TM, int G, int MODE, int U = 4, int USET = 7>
__device__ __forceinline__ void sweep_row_at(int I, int lane, bool active, int p0, int pd, int p1,
                                             const int* __restrict__ col, const TM* __restrict__ val,
                                             const T* __restrict__ dinv, const T* __restrict__ b,
                                             T* __restrict__ x) {
  static_assert(G >= 3, "one lane per output component");
  static_assert(MODE == 0 || MODE == 1, "sweep mode");
  T a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0, d0 = 0, d1 = 0, d2 = 0;
  // USET < 0: the fixed unroll U (the coarse tail, where the warp-uniform
  // unroll measured slower: more copies of the loop in a kernel that already
  // uses the full register budget)
  int n = !active ? 0 : MODE == 0 ? lane_slots<G>(pd - p0, lane) : lane_slots<G>(p1 - p0 - 1, lane);
  int u = USET < 0 ? (active ? U : 0) : warp_unroll<U>(n);
  if (active)
    with_unroll<U, USET>(u, [&](auto uc) {
      constexpr int UU = decltype(uc)::value;
      if (MODE == 0) row_msub<T, TM, G, UU>(p0 + lane, pd, col, val, x, a0, a1, a2);  // prefix
      else row_msub_off<T, TM, G, UU>(p0, pd, p1, lane, col, val, x, a0, a1, a2);
    });
  if (active && lane < 3) {  // issued before the group sum, whose latency hides theirs
    b0 = b[3L * I]; b1 = b[3L * I + 1]; b2 = b[3L * I + 2];
    const T* D = dinv + 9L * I + 3 * lane;
    d0 = ro(D); d1 = ro(D + 1); d2 = ro(D + 2);
  }
  group_sum3<G>(a0, a1, a2);  // every lane of the group now holds -sum A v
  if (active && lane < 3) x[3L * I + lane] = d0 * (b0 + a0) + d1 * (b1 + a1) + d2 * (b2 + a2);
}

template <typename T, typename TM, int G, int MODE, int U = 4, int USET = 7>
__device__ __forceinline__ void sweep_row(int I, int lane, bool active, const int* __restrict__ rowptr,
                                          const int* __restrict__ diag, const int* __restrict__ col,
                                          const TM* __restrict__ val, const T* __restrict__ dinv,
                                          const T* __restrict__ b, T* __restrict__ x) {
  int p0 = 0, pd = 0, p1 = 0;
  if (active) {
    p0 = ro(rowptr + I);
    pd = ro(diag + I);
    p1 = MODE == 0 ? 0 : ro(rowptr + I + 1);
  }
  sweep_row_at<T, TM, G, MODE, U, USET>(I, lane, active, p0, pd, p1, col, val, dinv, b, x);
}


// PDL: launched as a programmatic dependent of the kernel before it (the
// float32 sweeps, which are latency-bound): the row's block range is loaded
// and its read-only operator data prefetched into L1 while that kernel may
// still be finishing; griddepcontrol.wait then waits for its writes (x, b)
// before the row reads them.  Nothing launched in the same graph or stream
// writes the operator, whose values come from the numeric setup, which the
// host waits for.
template <typename T, typename TM, int G, int MODE, bool PDL = false>
__global__ void __launch_bounds__(256) kb_sweep(int r0, int r1, const int* __restrict__ rowptr,
                                                const int* __restrict__ diag, const int* __restrict__ col,
                                                const TM* __restrict__ val, const T* __restrict__ dinv,
                                                const T* __restrict__ b, T* __restrict__ x) {
  long gt = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int I = r0 + (int)(gt / G);
  bool active = I < r1;
  int p0 = 0, pd = 0, p1 = 0;
  if (active) {
    p0 = ro(rowptr + I);
    pd = ro(diag + I);
    p1 = MODE == 0 ? 0 : ro(rowptr + I + 1);
  }
  if (PDL) {
    if (active) {
      int lane = threadIdx.x % G, pe = MODE == 0 ? pd : p1;
      for (int q = p0 + lane; q < pe; q += G) {
        const char* v = (const char*)(val + 9L * q);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(col + q));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(v));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(v + 9 * sizeof(TM) - 1));
      }
      if (lane < 3) asm volatile("prefetch.global.L1 [%0];" ::"l"(dinv + 9L * I + 3 * lane));
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  sweep_row_at<T, TM, G, MODE>(I, threadIdx.x % G, active, p0, pd, p1, col, val, dinv, b, x);
}

// ---- SELL-32 form of a float64 coarse level (large colour classes) -------
// Chunk c holds the rows [32c, 32c + 32) of the level; slot group g = soff[c]
// + s holds the s-th off-diagonal block of each of the chunk's rows (prefix,
// i.e. lower colours, first, then the suffix, each by ascending column):
// column at scol[32 g + lane], entry k of the block at sval[(9 g + k) 32 +
// lane], so a warp reads each entry of 32 rows' blocks as 256 contiguous
// bytes.  A chunk has as many slot groups as its longest row has
// off-diagonal blocks; shorter rows' slots hold column -1.
constexpr int kSell = 32;

// slot groups of each chunk: its longest row's off-diagonal block count
__global__ void k_sell_width(int n, const int* __restrict__ rowptr, int* __restrict__ width) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c * kSell >= n) return;
  int w = 0;
  for (int I = c * kSell; I < min(n, (c + 1) * kSell); ++I) w = max(w, rowptr[I + 1] - rowptr[I] - 1);
  width[c] = w;
}

// chunk of each slot group
__global__ void k_sell_groups(int nch, const int* __restrict__ soff, int* __restrict__ sgc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  for (int g = soff[c]; g < soff[c + 1]; ++g) sgc[g] = c;
}

// BSR block position of slot (g, lane), or -1 for a padding slot
__device__ __forceinline__ long sell_block(long g, int lane, int n, const int* __restrict__ sgc,
                                           const int* __restrict__ soff, const int* __restrict__ rowptr,
                                           const int* __restrict__ diag) {
  int c = sgc[g];
  int I = c * kSell + lane, s = (int)(g - soff[c]);
  if (I >= n) return -1;
  int p0 = rowptr[I], pd = diag[I];
  if (s >= rowptr[I + 1] - p0 - 1) return -1;
  return p0 + s + (s >= pd - p0 ? 1 : 0);
}

// columns of the slots (symbolic setup), one thread per slot
__global__ void k_sell_cols(long groups, int n, const int* __restrict__ sgc, const int* __restrict__ soff,
                            const int* __restrict__ rowptr, const int* __restrict__ diag, const int* __restrict__ col,
                            int* __restrict__ scol) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= groups * kSell) return;
  long p = sell_block(t / kSell, (int)(t % kSell), n, sgc, soff, rowptr, diag);
  scol[t] = p < 0 ? -1 : col[p];
}

// block values of the slots (numeric setup, after the Galerkin product),
// one thread per slot: reads its block's 72 bytes, writes 9 coalesced rows
__global__ void k_sell_values(long groups, int n, const int* __restrict__ sgc, const int* __restrict__ soff,
                              const int* __restrict__ rowptr, const int* __restrict__ diag,
                              const double* __restrict__ val, double* __restrict__ sval) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= groups * kSell) return;
  long g = t / kSell;
  int lane = (int)(t % kSell);
  long p = sell_block(g, lane, n, sgc, soff, rowptr, diag);
  double* dst = sval + 9 * g * kSell + lane;
#pragma unroll
  for (int k = 0; k < 9; ++k) dst[k * kSell] = p < 0 ? 0.0 : val[9 * p + k];
}

// Block Gauss-Seidel update of the rows [r0, r1) of one colour class of a
// SELL-32 float64 level, modes 0 (forward sweep from zero: prefix only) and 1
// (plain sweep) of sweep_row_at, with G = 1, 2 or 4 lanes per row.  The
// float64 pipe (2 multiply-adds per clock per SM here) bounds the large
// classes, and masked-off float64 instructions cost it as much as live ones:
// with one lane per row there is no group sum and no idle slot, since rows
// within a class are ordered by their exact prefix and off-diagonal counts
// and the 32 rows of a chunk visit nearly the same number of slots.  Two
// lanes per row shorten each row's chain of loads for the longer full rows.
// U slots per lane are loaded before their multiply-adds, and the next
// slots' columns are in flight during them.
template <int MODE, int G, int U>
__global__ void __launch_bounds__(128) ks_sweep(int r0, int r1, const int* __restrict__ rowptr,
                                                const int* __restrict__ diag, const int* __restrict__ soff,
                                                const int* __restrict__ scol, const double* __restrict__ sval,
                                                const double* __restrict__ dinv, const double* __restrict__ b,
                                                double* __restrict__ x) {
  static_assert(G == 1 || G == 2 || G == 4, "lanes per row");
  static_assert(MODE == 0 || MODE == 1, "the prolongation is a separate pass on these levels");
  // warp w covers rows [(w % G) 32/G, +32/G) of chunk w / G, counted from the
  // class's first chunk; lane L takes row L / G of those and the slots h,
  // h + G, h + 2G, ... with h = L % G
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int w = (int)(t / 32), L = (int)(t % 32), h = L % G;
  int crow = (w % G) * (32 / G) + L / G;
  int I = (r0 & ~(kSell - 1)) + (w / G) * kSell + crow;
  bool active = I >= r0 && I < r1;
  if (G == 1 && !active) return;  // no shuffles below when G == 1
  int n = 0;
  long g0 = 0;
  if (active) {
    int p0 = ro(rowptr + I);
    n = MODE == 0 ? ro(diag + I) - p0 : ro(rowptr + I + 1) - p0 - 1;
    g0 = ro(soff + I / kSell);
  }
  const int* cp = scol + g0 * kSell + crow;
  const double* vp = sval + 9 * g0 * kSell + crow;
  double a0 = 0, a1 = 0, a2 = 0;
  // columns of the lane's slots j, ..., j + U - 1 (-1 past the row's end)
  auto cols = [&](int j, int (&J)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int q = G * (j + u) + h;
      J[u] = q < n ? ro(cp + (long)q * kSell) : -1;
    }
  };
  int Jn[U];
  cols(0, Jn);
  for (int j = 0; G * j + h < n; j += U) {
    int J[U];
    double v[U][3], A[U][9];
#pragma unroll
    for (int u = 0; u < U; ++u) J[u] = Jn[u];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (J[u] >= 0) {
        v[u][0] = x[3L * J[u]];
        v[u][1] = x[3L * J[u] + 1];
        v[u][2] = x[3L * J[u] + 2];
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (J[u] >= 0) {
        long q = G * (j + u) + h;
#pragma unroll
        for (int k = 0; k < 9; ++k) A[u][k] = ro(vp + (9 * q + k) * kSell);
      }
    cols(j + U, Jn);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (J[u] >= 0) {
        a0 = fma(-A[u][0], v[u][0], a0);
        a0 = fma(-A[u][1], v[u][1], a0);
        a0 = fma(-A[u][2], v[u][2], a0);
        a1 = fma(-A[u][3], v[u][0], a1);
        a1 = fma(-A[u][4], v[u][1], a1);
        a1 = fma(-A[u][5], v[u][2], a1);
        a2 = fma(-A[u][6], v[u][0], a2);
        a2 = fma(-A[u][7], v[u][1], a2);
        a2 = fma(-A[u][8], v[u][2], a2);
      }
  }
#pragma unroll
  for (int m = G / 2; m >= 1; m /= 2) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, m);
    a1 += __shfl_xor_sync(0xffffffffu, a1, m);
    a2 += __shfl_xor_sync(0xffffffffu, a2, m);
  }
  if (!active || h != 0) return;
  double t0 = b[3L * I] + a0, t1 = b[3L * I + 1] + a1, t2 = b[3L * I + 2] + a2;
  const double* D = dinv + 9L * I;
  x[3L * I] = ro(D) * t0 + ro(D + 1) * t1 + ro(D + 2) * t2;
  x[3L * I + 1] = ro(D + 3) * t0 + ro(D + 4) * t1 + ro(D + 5) * t2;
  x[3L * I + 2] = ro(D + 6) * t0 + ro(D + 7) * t1 + ro(D + 8) * t2;
}

// residual_row with the row's block range [p0, p1) already loaded
template <typename T, typename TM, int G, bool SUFFIX, int U = 4, int USET = 7>
__device__ __forceinline__ void residual_row_at(int I, int lane, bool active, int p0, int p1,
                                                const int* __restrict__ col, const TM* __restrict__ val,
                                                const T* __restrict__ b, const T* __restrict__ x,
                                                T* __restrict__ r) {
  static_assert(G >= 3, "one lane per output component");
  T a0 = 0, a1 = 0, a2 = 0, bc = 0;
  int u = USET < 0 ? (active ? U : 0) : warp_unroll<U>(active ? lane_slots<G>(p1 - p0, lane) : 0);
  if (active) {
    if (!SUFFIX && lane < 3) bc = b[3L * I + lane];
    with_unroll<U, USET>(u, [&](auto uc) {
      row_msub<T, TM, G, decltype(uc)::value>(p0 + lane, p1, col, val, x, a0, a1, a2);
    });
  }
  group_sum3<G>(a0, a1, a2);
  if (active && lane < 3) r[3L * I + lane] = bc + (lane == 0 ? a0 : lane == 1 ? a1 : a2);
}

// r_I = b_I - (A x)_I, G lanes per row (all lanes of the warp call it).
// SUFFIX: right after one forward block-GS sweep from x = 0, row I was
// updated as x_I = D_I^-1 (b_I - sum_{J < I} A_IJ x_J) with every lower
// colour already final, so b_I - sum_{J <= I} A_IJ x_J = 0 and the residual
// is only the part of the columns updated later:
//   r_I = - sum_{J in higher colours} A_IJ x_J   (exact up to rounding),
// half of the off-diagonal blocks and no b.
template <typename T, typename TM, int G, bool SUFFIX = false, int U = 4, int USET = 7>
__device__ __forceinline__ void residual_row(int I, int lane, bool active, const int* __restrict__ rowptr,
                                             const int* __restrict__ diag, const int* __restrict__ col,
                                             const TM* __restrict__ val, const T* __restrict__ b,
                                             const T* __restrict__ x, T* __restrict__ r) {
  int p0 = 0, p1 = 0;
  if (active) {
    p0 = SUFFIX ? ro(diag + I) + 1 : ro(rowptr + I);
    p1 = ro(rowptr + I + 1);
  }
  residual_row_at<T, TM, G, SUFFIX, U, USET>(I, lane, active, p0, p1, col, val, b, x, r);
}

template <typename T, typename TM, int G, bool SUFFIX>
__global__ void __launch_bounds__(256) kb_residual(int rend, const int* __restrict__ rowptr,
                                                   const int* __restrict__ diag, const int* __restrict__ col,
                                                   const TM* __restrict__ val, const T* __restrict__ b,
                                                   const T* __restrict__ x, T* __restrict__ r) {
  long gt = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int I = (int)(gt / G);
  bool active = I < rend;
  int p0 = 0, p1 = 0;
  if (active) {
    p0 = SUFFIX ? ro(diag + I) + 1 : ro(rowptr + I);
    p1 = ro(rowptr + I + 1);
  }
  residual_row_at<T, TM, G, SUFFIX>(I, threadIdx.x % G, active, p0, p1, col, val, b, x, r);
}

// Restriction plus the first colour of the next level's forward sweep:
// bc_I = sum of r over the members of aggregate I, skipping members
// >= skip_from (the last colour of a forward sweep, whose residual vanishes);
// for I < init_end, xc_I = Dinvc_I bc_I.
template <typename T>
__device__ __forceinline__ void restrict_row(int I, const int* __restrict__ mptr, const int* __restrict__ mem,
                                             int skip_from, const T* __restrict__ r, T* __restrict__ bc, int init_end,
                                             const T* __restrict__ dinvc, T* __restrict__ xc) {
  T a0 = 0, a1 = 0, a2 = 0;
  int q1 = ro(mptr + I + 1);
  for (int q = ro(mptr + I); q < q1; ++q) {
    long k = ro(mem + q);
    if (k >= skip_from) continue;
    a0 += r[3 * k];
    a1 += r[3 * k + 1];
    a2 += r[3 * k + 2];
  }
  bc[3L * I] = a0;
  bc[3L * I + 1] = a1;
  bc[3L * I + 2] = a2;
  if (I < init_end) {
    const T* D = dinvc + 9L * I;
    xc[3L * I] = ro(D) * a0 + ro(D + 1) * a1 + ro(D + 2) * a2;
    xc[3L * I + 1] = ro(D + 3) * a0 + ro(D + 4) * a1 + ro(D + 5) * a2;
    xc[3L * I + 2] = ro(D + 6) * a0 + ro(D + 7) * a1 + ro(D + 8) * a2;
  }
}

template <typename T>
__global__ void kb_restrict(int nc, const int* __restrict__ mptr, const int* __restrict__ mem, int skip_from,
                            const T* __restrict__ r, T* __restrict__ bc, int init_end, const T* __restrict__ dinvc,
                            T* __restrict__ xc) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < nc) restrict_row<T>(I, mptr, mem, skip_from, r, bc, init_end, dinvc, xc);
}

// cell-major permutation of a coarse vector: out[r] = in[perm[r]] (3 comps)
template <typename T>
__global__ void kb_gather3(int n, const int* __restrict__ perm, const T* __restrict__ in, T* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  long o = 3L * perm[r];
  out[3L * r] = in[o];
  out[3L * r + 1] = in[o + 1];
  out[3L * r + 2] = in[o + 2];
}
template <typename T>
__global__ void kb_scatter3(int n, const int* __restrict__ perm, const T* __restrict__ in, T* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  long o = 3L * perm[r];
  out[o] = in[3L * r];
  out[o + 1] = in[3L * r + 1];
  out[o + 2] = in[3L * r + 2];
}

template <typename T>
__global__ void kb_prolong(int n, const int* __restrict__ agg, const T* __restrict__ e, T* __restrict__ x) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n || agg[I] < 0) return;  // -1: no aggregate (padding rows of a batch)
  long a = 3L * agg[I];
  x[3L * I] += e[a];
  x[3L * I + 1] += e[a + 1];
  x[3L * I + 2] += e[a + 2];
}

// ---------------------------------------------------------------------------
// float64 outer operator and GCR vector kernels (red-black layout)
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_store(double* v, double* partial, int nvals) {
  __shared__ double sh[NV][kBlock / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double a = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  if (threadIdx.x < nvals && threadIdx.x < NV) {
    double a = 0;
    for (int w = 0; w < kBlock / 32; ++w) a += sh[threadIdx.x][w];
    partial[(long)threadIdx.x * kRedBlocks + blockIdx.x] = a;
  }
}

// out[q] = sum of partial[q][0..kRedBlocks), fixed order
__global__ void k_finish(const double* __restrict__ partial, double* __restrict__ out,
                         const double* __restrict__ gate = nullptr) {
  if (gate && *gate == 0.0) return;
  __shared__ double sh[kBlock];
  int q = blockIdx.x;
  double a = 0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kBlock) a += partial[(long)q * kRedBlocks + i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[q] = sh[0];
}

// ---------------------------------------------------------------------------
// K-cycle: two inner GCR steps on a coarse level (scalars on the device)
// ---------------------------------------------------------------------------
// y = A x, G lanes per row
template <typename T, typename TM, int G>
__global__ void __launch_bounds__(256) kb_spmv(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                               const TM* __restrict__ val, const T* __restrict__ x,
                                               T* __restrict__ y) {
  long gt = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int I = (int)(gt / G);
  int lane = threadIdx.x % G;
  bool active = I < n;
  T a0 = 0, a1 = 0, a2 = 0;
  int p0 = active ? rowptr[I] : 0, p1 = active ? rowptr[I + 1] : 0;
  int u = warp_unroll<4>(active ? lane_slots<G>(p1 - p0, lane) : 0);
  if (active)
    with_unroll<4, 7>(u, [&](auto uc) {
      row_msub<T, TM, G, decltype(uc)::value>(p0 + lane, p1, col, val, x, a0, a1, a2);
    });
  group_sum3<G>(a0, a1, a2);
  if (active)
    for (int c = lane; c < 3; c += G) y[3L * I + c] = -(c == 0 ? a0 : c == 1 ? a1 : a2);
}

// partial dots u_q . v_q (q < NQ) of coarse vectors, accumulated in float64
template <typename T, int NQ>
__global__ void __launch_bounds__(256) kd_dots(long n, const T* __restrict__ u0, const T* __restrict__ v0,
                                               const T* __restrict__ u1, const T* __restrict__ v1,
                                               double* __restrict__ partial) {
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    acc[0] += (double)u0[i] * (double)v0[i];
    if (NQ > 1) acc[NQ - 1] += (double)u1[i] * (double)v1[i];
  }
  block_reduce_store<NQ>(acc, partial, NQ);
}

// y = u - (ks[num] / ks[den]) v   (ks: the level's device scalars); a zero
// denominator means v = 0 and the coefficient is taken as 0
template <typename T>
__global__ void kk_axpy(long n, const T* u, const T* __restrict__ v, const double* __restrict__ ks,
                        int num, int den, T* y) {  // y may alias u
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double d = ks[den];
  if (i < n) y[i] = u[i] - (T)(d > 0 ? ks[num] / d : 0.0) * v[i];
}

// x = y1 z1 + y2 x with y2 = d2r/d22, y1 = (d1r - d12 y2)/d11:
// the minimiser of |r - A e| over span{z1, z2} (back substitution of the
// 2x2 Gram-Schmidt triangle); ks = {d11, d1r, d12, d22, d2r}
template <typename T>
__global__ void kk_combine(long n, const T* __restrict__ z1, T* __restrict__ x, const double* __restrict__ ks) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double y2 = ks[3] > 0 ? ks[4] / ks[3] : 0.0;  // a direction with zero image is dropped
  double y1 = ks[0] > 0 ? (ks[1] - ks[2] * y2) / ks[0] : 0.0;
  x[i] = (T)(y1 * (double)z1[i] + y2 * (double)x[i]);
}

// y = A x (float64); pads stay zero.  TX = storage type of x.
template <typename TX>
__global__ void __launch_bounds__(256) kg_apply(GridGeom g, const TX* __restrict__ x, const double* __restrict__ chat,
                                                double inv_dt, double* __restrict__ y, long s0 = 0) {
  long sl = s0 + blockIdx.x * (long)blockDim.x + threadIdx.x;  // slots [s0, 2 Nh)
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  if (!p.real) {
    y[sl] = 0;
    y[n2 + sl] = 0;
    y[2 * n2 + sl] = 0;
    return;
  }
  double v[3];
  slot_apply<double, TX>(g, c, sl, p, x, chat, inv_dt, v);
  y[sl] = v[0];
  y[n2 + sl] = v[1];
  y[2 * n2 + sl] = v[2];
}

// Knuth's two-sum: s + e == a + b exactly (s the rounded sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Float32-pair ("double-float") arithmetic for kg_apply_ff: a value is the
// unevaluated sum hi + lo of two float32.  two_prod is exact (fma); the pair
// product drops lo * lo; the pair sum renormalises with two_sum.  Each
// operation carries about 2^-48 of the operands' magnitude.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
// (sh, sl) += (ah, al) * (bh, bl)
__device__ __forceinline__ void ff_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float p, e, t;
  two_prod(ah, bh, p, e);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  two_sum(sh, p, sh, t);
  sl += t + e;
}

// y = A x for a float32 x (the mixed path's outer product, step 2 of each GCR
// iteration).  The stencil sum S - d x_k of float32 values is accumulated as
// a float32 pair (two-sum per term, the rounding error of d x_k by one fma),
// and x_k / dt + C^_k (S - d x_k) in float32-pair arithmetic, with C^ held
// as the pair (chat, chat_lo) written by the numeric setup and 1/dt as
// (idt, idt_lo): about 1e-14 of the largest term, against 1e-16 for float64
// products.  Only the last add of each component and its two widenings are
// float64: the float64 pipe (1/64 of the float32 rate here) bounded the
// float64-product version of this kernel (24 float64 operations per cell,
// conversions included; now 9).  (Widening with integer bit operations
// instead of the conversions measured slower.)
__global__ void __launch_bounds__(256) kg_apply_ff(GridGeom g, const float* __restrict__ x,
                                                   const float* __restrict__ chat, const float* __restrict__ chat_lo,
                                                   float idt, float idt_lo, double* __restrict__ y) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  if (!p.real) {
    y[sl] = 0;
    y[n2 + sl] = 0;
    y[2 * n2 + sl] = 0;
    return;
  }
  float x0 = x[sl], x1 = x[n2 + sl], x2 = x[2 * n2 + sl];
  float h0 = 0, h1 = 0, h2 = 0, l0 = 0, l1 = 0, l2 = 0, e;
  int d = for_neighbours(g, c, p, [&](long q) {
    two_sum(h0, x[q], h0, e);
    l0 += e;
    two_sum(h1, x[n2 + q], h1, e);
    l1 += e;
    two_sum(h2, x[2 * n2 + q], h2, e);
    l2 += e;
  });
  float fd = (float)d;
  float p0 = -fd * x0, p1 = -fd * x1, p2 = -fd * x2;  // -d x_k = p + q exactly
  float q0 = fmaf(-fd, x0, -p0), q1 = fmaf(-fd, x1, -p1), q2 = fmaf(-fd, x2, -p2);
  two_sum(h0, p0, h0, e);
  l0 += e + q0;
  two_sum(h1, p1, h1, e);
  l1 += e + q1;
  two_sum(h2, p2, h2, e);
  l2 += e + q2;
  float s0, s1, s2;  // the sums renormalised as pairs (s, l)
  two_sum(h0, l0, s0, l0);
  two_sum(h1, l1, s1, l1);
  two_sum(h2, l2, s2, l2);
  const float* Ch = chat + sl;
  const float* Cl = chat_lo + sl;
  float xs[3] = {x0, x1, x2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float yh, yl;
    two_prod(xs[k], idt, yh, yl);
    yl = fmaf(xs[k], idt_lo, yl);
    ff_fma(ld(Ch + (3 * k) * n2), ld(Cl + (3 * k) * n2), s0, l0, yh, yl);
    ff_fma(ld(Ch + (3 * k + 1) * n2), ld(Cl + (3 * k + 1) * n2), s1, l1, yh, yl);
    ff_fma(ld(Ch + (3 * k + 2) * n2), ld(Cl + (3 * k + 2) * n2), s2, l2, yh, yl);
    y[k * n2 + sl] = (double)yh + (double)yl;
  }
}

// y = r on the colour-0 slots [0, Nh): the product A z there when z leaves a
// block Gauss-Seidel sweep whose last half-sweep updated colour 0 with its
// (colour-1) neighbours final -- then D_k z_k = r_k - C^_k sum_j z_j, so
// (A z)_k = D_k z_k + C^_k sum_j z_j = r_k (exact up to rounding)
__global__ void kg_copy_colour0(GridGeom g, const double* __restrict__ r, double* __restrict__ y) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= g.nh) return;
  y[sl] = r[sl];
  y[n2 + sl] = r[n2 + sl];
  y[2 * n2 + sl] = r[2 * n2 + sl];
}

// r = b - A x, partial sums of |r|^2 and |b|^2
__global__ void __launch_bounds__(256) kg_residual(GridGeom g, const double* __restrict__ b,
                                                   const double* __restrict__ x, const double* __restrict__ chat,
                                                   double inv_dt, double* __restrict__ r, double* __restrict__ partial) {
  long n2 = 2 * g.nh;
  double acc[2] = {0, 0};
  for (long sl = blockIdx.x * (long)blockDim.x + threadIdx.x; sl < n2; sl += (long)gridDim.x * blockDim.x) {
    int c = (int)(sl / g.nh);
    SlotPos p = slot_pos(g, c, sl % g.nh);
    if (!p.real) {
      r[sl] = 0;
      r[n2 + sl] = 0;
      r[2 * n2 + sl] = 0;
      continue;
    }
    double v[3];
    slot_residual<double, double>(g, c, sl, p, b, x, chat, inv_dt, v);
    r[sl] = v[0];
    r[n2 + sl] = v[1];
    r[2 * n2 + sl] = v[2];
    acc[0] += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    acc[1] += b[sl] * b[sl] + b[n2 + sl] * b[n2 + sl] + b[2 * n2 + sl] * b[2 * n2 + sl];
  }
  block_reduce_store<2>(acc, partial, 2);
}

// A gated kernel does nothing when *gate == 0 (the whole grid returns at
// once): the second Gram-Schmidt pass, decided on the device, inside a
// captured graph.  gate == nullptr: always run.
__device__ __forceinline__ bool gated_off(const double* gate) { return gate && *gate == 0.0; }

// partial dots d_i = C_i . v for i in [i0, i0 + NV); SELF adds v . v and
// v . r as values NV and NV + 1.  Every index into acc is a compile-time
// constant, so acc stays in registers.
template <int NV, bool SELF = false>
__global__ void __launch_bounds__(256) kg_multidot(long n, const double* __restrict__ C, int i0,
                                                   const double* __restrict__ v, double* __restrict__ partial,
                                                   const double* __restrict__ gate = nullptr,
                                                   const double* __restrict__ r = nullptr) {
  if (gated_off(gate)) return;
  constexpr int NQ = NV + (SELF ? 2 : 0);
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0;
#pragma unroll 2  // two elements in flight per thread
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    double vt = v[t];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += C[(long)(i0 + q) * n + t] * vt;
    if constexpr (SELF) {
      acc[NV] += vt * vt;
      acc[NV + 1] += vt * r[t];
    }
  }
  block_reduce_store<NQ>(acc, partial, NQ);
}

// kg_multidot launched with NV = cnt (1 <= cnt <= NV).  The kernel is bound
// by the float64 pipe, and with NV fixed at the chunk size every launch took
// the time of a full chunk whatever cnt was: the masked-off fused
// multiply-adds still cost pipe slots.
template <int NV, bool SELF>
void launch_multidot(int cnt, cudaStream_t s, long n, const double* C, int i0, const double* v, double* partial,
                     const double* gate = nullptr, const double* r = nullptr) {
  if constexpr (NV > 1) {
    if (cnt < NV) {
      launch_multidot<NV - 1, SELF>(cnt, s, n, C, i0, v, partial, gate, r);
      return;
    }
  }
  kg_multidot<NV, SELF><<<kRedBlocks, kBlock, 0, s>>>(n, C, i0, v, partial, gate, r);
}

// v -= sum_{i<j} coef[i] C_i (coef on the device); when *rnow != 0 the same
// pass also takes the GCR step r -= rcoef v with the new v and stores the
// partial sums of |r|^2
__global__ void __launch_bounds__(256) kg_multiaxpy_r(long n, double* __restrict__ v, const double* __restrict__ C,
                                                      int j, const double* __restrict__ coef,
                                                      double* __restrict__ r, const double* __restrict__ rnow,
                                                      const double* __restrict__ rcoef,
                                                      double* __restrict__ partial,
                                                      const double* __restrict__ gate = nullptr) {
  if (gated_off(gate)) return;
  const bool upd = *rnow != 0.0;
  const double f = *rcoef;
  double acc[1] = {0};
#pragma unroll 2  // two elements in flight per thread
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    double a = v[t];
#pragma unroll 4
    for (int i = 0; i < j; ++i) a -= coef[i] * C[(long)i * n + t];
    v[t] = a;
    if (upd) {
      double b = r[t] - f * a;
      r[t] = b;
      acc[0] += b * b;
    }
  }
  if (upd) block_reduce_store<1>(acc, partial, 1);
}

// partial sums of |c|^2 and c.r
__global__ void __launch_bounds__(256) kg_dot2(long n, const double* __restrict__ c, const double* __restrict__ r,
                                               double* __restrict__ partial) {
  double acc[2] = {0, 0};
#pragma unroll 2  // two elements in flight per thread
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    double ct = c[t];
    acc[0] += ct * ct;
    acc[1] += ct * r[t];
  }
  block_reduce_store<2>(acc, partial, 2);
}

// r -= coef * c, partial |r|^2
__global__ void __launch_bounds__(256) kg_rupdate(long n, double* __restrict__ r, const double* __restrict__ c,
                                                  const double* __restrict__ coef, double* __restrict__ partial) {
  double f = *coef;
  double acc[1] = {0};
#pragma unroll 2  // two elements in flight per thread
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    double v = r[t] - f * c[t];
    r[t] = v;
    acc[0] += v * v;
  }
  block_reduce_store<1>(acc, partial, 1);
}

// x += sum_k y_k Z_k
template <typename TZ>
__global__ void __launch_bounds__(256) kg_xupdate(long n, double* __restrict__ x, const TZ* __restrict__ Z, int m,
                                                  const double* __restrict__ y) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  double a = x[t];
  for (int k = 0; k < m; ++k) a += y[k] * (double)Z[(long)k * n + t];
  x[t] = a;
}

// natural SoA <-> red-black slots (pads of the output are zeroed)
template <typename TI, typename TO>
__global__ void k_to_rb(GridGeom g, const int* __restrict__ nat_of_slot, const TI* __restrict__ in,
                        TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int k = nat_of_slot[sl];
  for (int c = 0; c < 3; ++c) out[c * n2 + sl] = k < 0 ? (TO)0 : (TO)in[c * g.n + k];
}
template <typename TI, typename TO>
__global__ void k_from_rb(GridGeom g, const int* __restrict__ nat_of_slot, const TI* __restrict__ in,
                          TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int k = nat_of_slot[sl];
  if (k < 0) return;
  for (int c = 0; c < 3; ++c) out[c * g.n + k] = (TO)in[c * n2 + sl];
}

// ---------------------------------------------------------------------------
// GCR scalars (device resident, one thread)
// ---------------------------------------------------------------------------
struct GcrScal {
  double rn2, bn2, cc, cr;         // reduction results (read by the host)
  double gjj, rcoef;               // gamma_jj, alpha_j s_j
  double cn2, pass2;               // |c|^2 before the projection; 1: run the second pass
  double d[kMaxRestart];           // dots of the current vector with C'_i
  double coef[kMaxRestart];        // projection coefficients of the update
  double gam[kMaxRestart * kMaxRestart];  // Gamma, row-major
  double alpha[kMaxRestart], s[kMaxRestart], y[kMaxRestart];
  double cq[2];                    // |c|^2 and c . r before the current projection pass
  double rnow;                     // 1: the current pass's update also takes the GCR step
};

// gamma_jj = |c|, s_j = 1/gamma_jj, alpha_j = c_j . r = s_j (c . r)
__device__ __forceinline__ void norm_coef(GcrScal* S, int j) {
  double g = sqrt(S->cc);
  S->gjj = g;
  S->gam[j * kMaxRestart + j] = g;
  double s = 1.0 / g;
  S->s[j] = s;
  S->alpha[j] = s * S->cr;
  S->rcoef = S->alpha[j] * s;
}
__global__ void k_norm_coef(GcrScal* S, int j) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  norm_coef(S, j);
}

// Gram-Schmidt coefficients from the dots d_i = C'_i . c (C'_i unnormalised,
// c_i = s_i C'_i): gamma_i = s_i d_i is added to Gamma_ij and the update
// c -= gamma_i c_i uses coef_i = gamma_i s_i.  With the c_i orthonormal,
// |c - P c|^2 = |c|^2 - sum gamma_i^2.
// After the first pass, the second is needed only when the projection removed
// more than half of |c|^2 (|c - P c| < |c|/sqrt 2): below that, rounding
// in the first pass can have left components along the c_i that a second
// pass removes ("twice is enough", Kahan-Parlett).  pass2 is set to 0 or 1.
// The pass that ends the projection (the first when no second runs) also
// takes step 4 here: |c - P c|^2 from the sum above (at least half of |c|^2
// in the first pass; in the second, P c is at rounding level), and
// (c - P c) . r = c . r, r being orthogonal to every earlier c_i; rnow = 1
// makes the projection's update take step 5 in the same pass.
__global__ void k_gs_coef(GcrScal* S, int j, int first, const double* __restrict__ gate = nullptr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (gate && *gate == 0.0) return;
  double proj = 0;
  for (int i = 0; i < j; ++i) {
    double gm = S->s[i] * S->d[i];
    S->gam[i * kMaxRestart + j] = first ? gm : S->gam[i * kMaxRestart + j] + gm;
    S->coef[i] = gm * S->s[i];
    proj += gm * gm;
  }
  double rem = S->cq[0] - proj;
  bool last = true;
  if (first) {
    S->pass2 = rem < 0.5 * S->cq[0] ? 1.0 : 0.0;
    last = S->pass2 == 0.0;
  }
  S->rnow = last ? 1.0 : 0.0;
  if (last) {
    S->cc = rem;
    S->cr = S->cq[1];
    norm_coef(S, j);
  }
}
// y = Gamma^{-1} alpha (upper triangular)
__global__ void k_backsub(GcrScal* S, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = m - 1; i >= 0; --i) {
    double a = S->alpha[i];
    for (int k = i + 1; k < m; ++k) a -= S->gam[i * kMaxRestart + k] * S->y[k];
    S->y[i] = a / S->gam[i * kMaxRestart + i];
  }
}

// m <- x / |x| per cell (the projection step), natural SoA
__global__ void k_renormalise(long n, const double* __restrict__ x, double* __restrict__ m, int* __restrict__ bad) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double a = x[k], b = x[n + k], c = x[2 * n + k];
  double s = sqrt(a * a + b * b + c * c);
  if (!(s > 0.0) || !isfinite(s)) {
    atomicExch(bad, 1);
    return;
  }
  m[k] = a / s;
  m[n + k] = b / s;
  m[2 * n + k] = c / s;
}

// rhs = m/dt - C(m) f with f = -q (0, m2, m3) + he  (explicit source terms)
__global__ void k_rhs_llg(long n, const double* __restrict__ m, double alpha, double inv_dt, double q, double he0,
                          double he1, double he2, double* __restrict__ b) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double m1 = m[k], m2 = m[n + k], m3 = m[2 * n + k];
  double f1 = he0, f2 = he1 - q * m2, f3 = he2 - q * m3;
  double mm = m1 * m1 + m2 * m2 + m3 * m3, mf = m1 * f1 + m2 * f2 + m3 * f3;
  // C(m) f = m x f + alpha (m (m.f) - |m|^2 f)
  double c1 = m2 * f3 - m3 * f2 + alpha * (m1 * mf - mm * f1);
  double c2 = m3 * f1 - m1 * f3 + alpha * (m2 * mf - mm * f2);
  double c3 = m1 * f2 - m2 * f1 + alpha * (m3 * mf - mm * f3);
  b[k] = m1 * inv_dt - c1;
  b[n + k] = m2 * inv_dt - c2;
  b[2 * n + k] = m3 * inv_dt - c3;
}

// The initial approximation of a time step's solve (the same reading as the
// oracle's step_guess): m^n and up to kStepHist earlier states s_1 (newest)
// ... s_d extrapolated one step ahead with the terms of Newton's
// backward-difference series m + D m + D^2 m + ... that keep shrinking.
// k_step_diff_norms gives the partial sums of |D^j m|^2, j = 1..d, each
// difference formed element by element with the oracle's operations
// (t_l -= t_{l+1}, j times); the host picks the order k and k_step_guess
// forms sum_{l<=k} c_l s_l, c_l = (-1)^l C(k+1, l+1).
constexpr int kStepHist = 6;
struct StepStates {
  const double* s[kStepHist + 1];  // s[0] = m^n, s[l] = m^{n-l}
};
__global__ void __launch_bounds__(256) k_step_diff_norms(long n, int d, StepStates S, double* __restrict__ partial) {
  double acc[kStepHist];
#pragma unroll
  for (int j = 0; j < kStepHist; ++j) acc[j] = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double t[kStepHist + 1];
#pragma unroll
    for (int l = 0; l <= kStepHist; ++l) t[l] = l <= d ? S.s[l][i] : 0.0;
#pragma unroll
    for (int j = 1; j <= kStepHist; ++j) {
#pragma unroll
      for (int l = 0; l + j <= kStepHist; ++l) t[l] = t[l] - t[l + 1];
      if (j <= d) acc[j - 1] += t[0] * t[0];
    }
  }
  block_reduce_store<kStepHist>(acc, partial, kStepHist);
}
struct StepCoef {
  double c[kStepHist + 1];
};
__global__ void k_step_guess(long n, int k, StepStates S, StepCoef C, double* __restrict__ x) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = C.c[0] * S.s[0][i];
  for (int l = 1; l <= k; ++l) v += C.c[l] * S.s[l][i];
  x[i] = v;
}

// *differ = 1 if a and b differ in any bit (a continued time integration is
// recognised by the field passed in being the hierarchy's last output)
__global__ void k_differ(long n, const double* __restrict__ a, const double* __restrict__ b, int* __restrict__ differ) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n && __double_as_longlong(a[i]) != __double_as_longlong(b[i])) *differ = 1;
}

// rhs = m / dt
__global__ void k_scale(long n, const double* __restrict__ m, double inv_dt, double* __restrict__ b) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = m[i] * inv_dt;
}

}  // namespace llmg
