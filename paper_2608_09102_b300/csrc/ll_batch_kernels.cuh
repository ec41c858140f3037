// Device kernels of the batched solver: assembly of the union hierarchy from
// per-instance hierarchies, the dense solves of the instances whose coarsest
// level is reached, and the GCR vector kernels with one set of scalars per
// instance.  Included by ll_solver.cu only.
#pragma once

#include "ll_kernels.cuh"

namespace llmg {

// ---------------------------------------------------------------------------
// union assembly (integer bookkeeping, once per batch)
// ---------------------------------------------------------------------------
// Local row r of one instance's level (colour-class numbering, classes
// [cs[t], cs[t+1]) for t < ncls) -> union row: off[t] + r - cs[t]; rows of an
// instance whose coarsest level this is (ncls == 0) map to off[0] + r.
// tab = {cs[0..ncls], off[0..max(ncls,1))}.
__global__ void kb_union_rowmap(int n, int ncls, const int* __restrict__ tab, int* __restrict__ map) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  if (ncls == 0) {
    map[r] = tab[1] + r;
    return;
  }
  int t = 0;
  while (t + 1 < ncls && r >= tab[t + 1]) ++t;
  map[r] = tab[ncls + 1 + t] + r - tab[t];
}

__global__ void kb_fill_int(long n, int v, int* __restrict__ p) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// level-0 slots of one instance -> union rows: colour c slots go to the
// union's class c at offset off[c]
__global__ void kb_union_slotmap(long nh, int off0, int off1, int* __restrict__ map) {
  long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= 2 * nh) return;
  map[s] = s < nh ? off0 + (int)s : off1 + (int)(s - nh);
}

// number of blocks of each union row (from one instance's BSR level)
__global__ void kb_union_rowcount(int n, const int* __restrict__ rp, const int* __restrict__ map,
                                  int* __restrict__ cnt) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) cnt[map[r]] = rp[r + 1] - rp[r];
}

// pattern of one instance's BSR level inside the union: rows keep their
// block order, columns go through the row map (monotone within an
// instance, so sorted rows stay sorted and the diagonal keeps its place)
__global__ void kb_union_pattern(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const int* __restrict__ dg, const int* __restrict__ map,
                                 const int* __restrict__ urp, int* __restrict__ ucol, int* __restrict__ udiag,
                                 int* __restrict__ bmap) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int R = map[r];
  int o = urp[R] - rp[r];
  for (int p = rp[r]; p < rp[r + 1]; ++p) {
    ucol[o + p] = map[col[p]];
    bmap[p] = o + p;
  }
  udiag[R] = o + dg[r];
}

// members of one instance's level-(l+1) rows, mapped into the union level l
__global__ void kb_union_memcount(int n, const int* __restrict__ mptr, const int* __restrict__ map,
                                  int* __restrict__ cnt) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) cnt[map[r]] = mptr[r + 1] - mptr[r];
}
__global__ void kb_union_members(int n, const int* __restrict__ mptr, const int* __restrict__ mem,
                                 const int* __restrict__ map, const int* __restrict__ fmap,
                                 const int* __restrict__ umptr, int* __restrict__ umem) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int o = umptr[map[r]] - mptr[r];
  for (int p = mptr[r]; p < mptr[r + 1]; ++p) umem[o + p] = fmap[mem[p]];
}

// union agg of one instance's level l: its rows -> union rows of level l+1
// (-1 where the instance has no aggregate, i.e. padding slots)
__global__ void kb_union_agg(long n, const int* __restrict__ agg, const int* __restrict__ map,
                             const int* __restrict__ cmap, int* __restrict__ uagg) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int a = agg[r];
  uagg[map[r]] = a < 0 ? -1 : cmap[a];
}

// level 0 of one instance as union BSR rows: the diagonal block first for
// colour 0 (all neighbours have the higher colour 1), last for colour 1
__global__ void kb_union_l0_count(GridGeom g, const int* __restrict__ map, int* __restrict__ cnt) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= 2 * g.nh) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  long nb[6];
  cnt[map[sl]] = p.real ? 1 + slot_neighbours(g, c, p, nb) : 1;
}
__global__ void kb_union_l0_pattern(GridGeom g, const int* __restrict__ map, const int* __restrict__ urp,
                                    int* __restrict__ ucol, int* __restrict__ udiag) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= 2 * g.nh) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  int R = map[sl];
  int o = urp[R];
  long nb[6];
  int d = p.real ? slot_neighbours(g, c, p, nb) : 0;
  if (c == 0) {
    udiag[R] = o;
    ucol[o++] = R;
    for (int q = 0; q < d; ++q) ucol[o++] = map[nb[q]];
  } else {
    for (int q = 0; q < d; ++q) ucol[o++] = map[nb[q]];
    udiag[R] = o;
    ucol[o] = R;
  }
}

// level-0 values of one instance (per step): off-diagonal blocks C^_k, the
// diagonal I/dt - deg C^_k, and D^-1; a padding slot gets I/dt and dt I.
// val64 is the float64 operator, valt/dinvt the V-cycle copies.
template <typename T>
__global__ void kb_union_l0_values(GridGeom g, const int* __restrict__ map, const int* __restrict__ urp,
                                   const int* __restrict__ udiag, const double* __restrict__ chat,
                                   const T* __restrict__ dinv, double inv_dt, double* __restrict__ val64,
                                   T* __restrict__ valt, T* __restrict__ dinvt) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  int R = map[sl];
  long nb[6];
  int d = p.real ? slot_neighbours(g, c, p, nb) : 0;
  double C[9], D[9];
  for (int e = 0; e < 9; ++e) C[e] = p.real ? chat[e * n2 + sl] : 0.0;
  for (int e = 0; e < 9; ++e) D[e] = ((e % 4) == 0 ? inv_dt : 0.0) - d * C[e];
  for (int q = urp[R]; q < urp[R + 1]; ++q) {
    const double* src = q == udiag[R] ? D : C;
    for (int e = 0; e < 9; ++e) {
      val64[9L * q + e] = src[e];
      if (valt) valt[9L * q + e] = (T)src[e];
    }
  }
  for (int e = 0; e < 9; ++e) dinvt[9L * R + e] = p.real ? dinv[e * n2 + sl] : ((e % 4) == 0 ? (T)(1.0 / inv_dt) : (T)0);
}

// coarse values of one instance's level (per step): blocks through bmap,
// D^-1 through the row map
template <typename TM, typename T>
__global__ void kb_union_values(int n, const int* __restrict__ rp, const int* __restrict__ bmap,
                                const int* __restrict__ map, const TM* __restrict__ val, const T* __restrict__ dinv,
                                TM* __restrict__ uval, T* __restrict__ udinv) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int p = rp[r]; p < rp[r + 1]; ++p)
    for (int e = 0; e < 9; ++e) uval[9L * bmap[p] + e] = val[9L * p + e];
  long R = map[r];
  for (int e = 0; e < 9; ++e) udinv[9 * R + e] = dinv[9L * r + e];
}

// ---- the transposed operator A^T (adjoint solves) -------------------------
// level 0: (A^T)_kk = I/dt - deg C^_k^T, (A^T)_kj = C^_j^T for a face
// neighbour j (A_kj = C^_k couples row k through its own coefficient, so the
// transpose carries the neighbour's); D^-1 transposed.  Same block order as
// kb_union_l0_pattern.
template <typename T>
__global__ void kb_union_l0_values_t(GridGeom g, const int* __restrict__ map, const int* __restrict__ urp,
                                     const double* __restrict__ chat, const T* __restrict__ dinv, double inv_dt,
                                     double* __restrict__ val64, T* __restrict__ valt, T* __restrict__ dinvt) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  int c = (int)(sl / g.nh);
  SlotPos p = slot_pos(g, c, sl % g.nh);
  int R = map[sl];
  long nb[6];
  int d = p.real ? slot_neighbours(g, c, p, nb) : 0;
  double D[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      D[3 * a + b] = (a == b ? inv_dt : 0.0) - (p.real ? d * chat[(3 * b + a) * n2 + sl] : 0.0);
  int q = urp[R];
  auto put = [&](const double* blk) {
    for (int e = 0; e < 9; ++e) {
      val64[9L * q + e] = blk[e];
      if (valt) valt[9L * q + e] = (T)blk[e];
    }
    ++q;
  };
  if (c == 0) put(D);
  for (int t = 0; t < d; ++t) {
    double Cn[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Cn[3 * a + b] = chat[(3 * b + a) * n2 + nb[t]];
    put(Cn);
  }
  if (c == 1) put(D);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      dinvt[9L * R + 3 * a + b] = p.real ? dinv[(3 * b + a) * n2 + sl] : (a == b ? (T)(1.0 / inv_dt) : (T)0);
}

// coarse levels: block position of (J, I) for every block (I, J) of a BSR
// level with a symmetric pattern (-1 if absent, which a Galerkin pattern
// built from an undirected graph never is)
__global__ void kb_transpose_pos(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 int* __restrict__ tpos) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int p = rp[r]; p < rp[r + 1]; ++p) {
    int J = col[p], f = -1;
    for (int q = rp[J]; q < rp[J + 1]; ++q)
      if (col[q] == r) f = q;
    tpos[p] = f;
  }
}
// (A^T)_IJ = (A_JI)^T through tpos and bmap; D^-1 transposed
template <typename TM, typename T>
__global__ void kb_union_values_t(int n, const int* __restrict__ rp, const int* __restrict__ bmap,
                                  const int* __restrict__ tpos, const int* __restrict__ map,
                                  const TM* __restrict__ val, const T* __restrict__ dinv, TM* __restrict__ uval,
                                  T* __restrict__ udinv, int* __restrict__ bad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int p = rp[r]; p < rp[r + 1]; ++p) {
    int t = tpos[p];
    if (t < 0) {
      atomicExch(bad, 1);
      continue;
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) uval[9L * bmap[p] + 3 * a + b] = val[9L * t + 3 * b + a];
  }
  long R = map[r];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) udinv[9 * R + 3 * a + b] = dinv[9L * r + 3 * b + a];
}

// ---- one step's vector-Jacobian product (natural SoA, float64) ------------
// xbar = (g - (u.g) u)/|x|, u = x/|x|: the transpose of the projection's
// Jacobian applied to g
__global__ void k_vjp_xbar(long n, const double* __restrict__ x, const double* __restrict__ g,
                           double* __restrict__ xbar) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double v0 = x[k], v1 = x[n + k], v2 = x[2 * n + k];
  double nrm = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  double u0 = v0 / nrm, u1 = v1 / nrm, u2 = v2 / nrm;
  double g0 = g[k], g1 = g[n + k], g2 = g[2 * n + k];
  double ug = u0 * g0 + u1 * g1 + u2 * g2;
  xbar[k] = (g0 - ug * u0) / nrm;
  xbar[n + k] = (g1 - ug * u1) / nrm;
  xbar[2 * n + k] = (g2 - ug * u2) / nrm;
}

// mbar_k = lambda_k/dt - [y x lambda + alpha((m.y) lambda + (lambda.m) y
// - 2 (lambda.y) m)]_k with y = Delta_h x, and partial sums of
// lambda.(m (m.y) - |m|^2 y) (dL/dalpha is minus their total)
__global__ void __launch_bounds__(256) k_vjp_param(int nx, int ny, int nz, const double* __restrict__ m,
                                                   const double* __restrict__ x, const double* __restrict__ lam,
                                                   double alpha, double inv_dt, double ih2,
                                                   double* __restrict__ mbar, double* __restrict__ partial) {
  long n = (long)nx * ny * nz;
  double acc[1] = {0};
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    int i = (int)(k % nx);
    long t = k / nx;
    int j = (int)(t % ny), l = (int)(t / ny);
    long nxy = (long)nx * ny;
    long nb[6];
    int d = 0;
    if (l > 0) nb[d++] = k - nxy;
    if (j > 0) nb[d++] = k - nx;
    if (i > 0) nb[d++] = k - 1;
    if (i < nx - 1) nb[d++] = k + 1;
    if (j < ny - 1) nb[d++] = k + nx;
    if (l < nz - 1) nb[d++] = k + nxy;
    double y[3];
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int q = 0; q < d; ++q) s += x[c * n + nb[q]];
      y[c] = (s - d * x[c * n + k]) * ih2;
    }
    double mk[3] = {m[k], m[n + k], m[2 * n + k]};
    double lk[3] = {lam[k], lam[n + k], lam[2 * n + k]};
    double my = mk[0] * y[0] + mk[1] * y[1] + mk[2] * y[2];
    double lm = lk[0] * mk[0] + lk[1] * mk[1] + lk[2] * mk[2];
    double ly = lk[0] * y[0] + lk[1] * y[1] + lk[2] * y[2];
    double mm = mk[0] * mk[0] + mk[1] * mk[1] + mk[2] * mk[2];
    double yxl[3] = {y[1] * lk[2] - y[2] * lk[1], y[2] * lk[0] - y[0] * lk[2], y[0] * lk[1] - y[1] * lk[0]};
    for (int c = 0; c < 3; ++c)
      mbar[c * n + k] = lk[c] * inv_dt - (yxl[c] + alpha * (my * lk[c] + lm * y[c] - 2.0 * ly * mk[c]));
    acc[0] += lm * my - mm * ly;
  }
  block_reduce_store<1>(acc, partial, 1);
}

// natural SoA vector of one instance <-> union level-0 rows (cell-major)
template <typename TI, typename TO>
__global__ void kb_union_in(GridGeom g, const int* __restrict__ nat_of_slot, const int* __restrict__ map,
                            const TI* __restrict__ in, TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= 2 * g.nh) return;
  int k = nat_of_slot[sl];
  long R = map[sl];
  for (int c = 0; c < 3; ++c) out[3 * R + c] = k < 0 ? (TO)0 : (TO)in[c * g.n + k];
}
template <typename TI, typename TO>
__global__ void kb_union_out(GridGeom g, const int* __restrict__ nat_of_slot, const int* __restrict__ map,
                             const TI* __restrict__ in, TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= 2 * g.nh) return;
  int k = nat_of_slot[sl];
  if (k < 0) return;
  long R = map[sl];
  for (int c = 0; c < 3; ++c) out[c * g.n + k] = (TO)in[3 * R + c];
}

// ---------------------------------------------------------------------------
// V-cycle pieces
// ---------------------------------------------------------------------------
// x = A_i^{-1} b for every instance i whose coarsest level this is (one task
// per instance: its rows start at row0, N = 3 x cells, column-major inverse)
template <typename T>
__global__ void kc_solve_batch(const CoarseTask* __restrict__ tasks, const T* __restrict__ b, T* __restrict__ x) {
  CoarseTask t = tasks[blockIdx.y];
  if (blockIdx.x * blockDim.x >= t.N) return;  // whole block past this task
  extern __shared__ double sb[];
  const T* bb = b + 3L * t.row0;
  for (int j = threadIdx.x; j < t.N; j += blockDim.x) sb[j] = (double)bb[j];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.N) return;
  double acc = 0.0;
  for (int j = 0; j < t.N; ++j) acc += t.ainv[(long)j * t.N + i] * sb[j];
  x[3L * t.row0 + i] = (T)acc;
}

template <typename TI, typename TO>
__global__ void k_convert(long n, const TI* __restrict__ in, TO* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}

// ---------------------------------------------------------------------------
// GCR with per-instance scalars.  Vectors are in union level-0 order; a chunk
// is an element range of one instance, one block per chunk; partial sums go
// to partial[q * nchunks + chunk] and are added per instance in chunk order.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void chunk_reduce_store(double* v, double* partial, int nvals, int nchunks) {
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
    partial[(long)threadIdx.x * nchunks + blockIdx.x] = a;
  }
}

// ((double*)&S[i])[field + q] = sum of partial[q][chunks of instance i]
__global__ void kgb_finish(const double* __restrict__ partial, int nchunks, const int* __restrict__ iptr,
                           GcrScal* __restrict__ S, int field, bool gated = false) {
  __shared__ double sh[kBlock];
  int i = blockIdx.x, q = blockIdx.y;
  if (gated && S[i].pass2 == 0.0) return;
  double a = 0;
  for (int k = iptr[i] + threadIdx.x; k < iptr[i + 1]; k += kBlock) a += partial[(long)q * nchunks + k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) reinterpret_cast<double*>(S + i)[field + q] = sh[0];
}

// gate: the second Gram-Schmidt pass of an instance runs only when its
// pass2 flag is set (see k_gs_coef); gate == nullptr: always run
__device__ __forceinline__ bool inst_off(const GcrScal* gate, int inst) { return gate && gate[inst].pass2 == 0.0; }

// dots with C_i for i in [i0, i0 + NV); SELF adds v . v as value NV (|c|^2
// before the projection).  Compile-time indices only: acc stays in registers.
template <int NV, bool SELF = false>
__global__ void __launch_bounds__(256) kgb_multidot(const Chunk* __restrict__ ch, int nchunks,
                                                    const double* __restrict__ C, long n3, int i0,
                                                    const double* __restrict__ v, double* __restrict__ partial,
                                                    const GcrScal* __restrict__ gate = nullptr) {
  Chunk k = ch[blockIdx.x];
  if (inst_off(gate, k.inst)) return;  // uniform per block: one chunk, one instance
  double acc[NV + 1];
#pragma unroll
  for (int q = 0; q <= NV; ++q) acc[q] = 0;
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    double vt = v[t];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += C[(long)(i0 + q) * n3 + t] * vt;
    if (SELF) acc[NV] += vt * vt;
  }
  chunk_reduce_store<NV + 1>(acc, partial, NV + (SELF ? 1 : 0), nchunks);
}

// kgb_multidot launched with NV = cnt (1 <= cnt <= NV), as launch_multidot
template <int NV, bool SELF>
void launch_batch_multidot(int cnt, cudaStream_t s, int nch, const Chunk* ch, const double* C, long n3, int i0,
                           const double* v, double* partial, const GcrScal* gate = nullptr) {
  if constexpr (NV > 1) {
    if (cnt < NV) {
      launch_batch_multidot<NV - 1, SELF>(cnt, s, nch, ch, C, n3, i0, v, partial, gate);
      return;
    }
  }
  kgb_multidot<NV, SELF><<<nch, kBlock, 0, s>>>(ch, nch, C, n3, i0, v, partial, gate);
}

__global__ void __launch_bounds__(256) kgb_multiaxpy(const Chunk* __restrict__ ch, double* __restrict__ v,
                                                     const double* __restrict__ C, long n3, int j,
                                                     const GcrScal* __restrict__ S,
                                                     const GcrScal* __restrict__ gate = nullptr) {
  Chunk k = ch[blockIdx.x];
  if (inst_off(gate, k.inst)) return;
  const double* coef = S[k.inst].coef;
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    double a = v[t];
    for (int i = 0; i < j; ++i) a -= coef[i] * C[(long)i * n3 + t];
    v[t] = a;
  }
}

__global__ void __launch_bounds__(256) kgb_dot2(const Chunk* __restrict__ ch, int nchunks,
                                                const double* __restrict__ c, const double* __restrict__ r,
                                                double* __restrict__ partial) {
  Chunk k = ch[blockIdx.x];
  double acc[2] = {0, 0};
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    double ct = c[t];
    acc[0] += ct * ct;
    acc[1] += ct * r[t];
  }
  chunk_reduce_store<2>(acc, partial, 2, nchunks);
}

__global__ void __launch_bounds__(256) kgb_rupdate(const Chunk* __restrict__ ch, int nchunks, double* __restrict__ r,
                                                   const double* __restrict__ c, const GcrScal* __restrict__ S,
                                                   double* __restrict__ partial) {
  Chunk k = ch[blockIdx.x];
  double f = S[k.inst].rcoef;
  double acc[1] = {0};
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    double v = r[t] - f * c[t];
    r[t] = v;
    acc[0] += v * v;
  }
  chunk_reduce_store<1>(acc, partial, 1, nchunks);
}

template <typename TZ>
__global__ void __launch_bounds__(256) kgb_xupdate(const Chunk* __restrict__ ch, double* __restrict__ x,
                                                   const TZ* __restrict__ Z, long n3, const GcrScal* __restrict__ S,
                                                   const int* __restrict__ jdone) {
  Chunk k = ch[blockIdx.x];
  int m = jdone[k.inst];
  const double* y = S[k.inst].y;
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    double a = x[t];
    for (int q = 0; q < m; ++q) a += y[q] * (double)Z[(long)q * n3 + t];
    x[t] = a;
  }
}

// y = A x on union level 0 in float64 (x stored as TX), one thread per row
template <typename TX>
__global__ void __launch_bounds__(256) kgb_apply(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                                 const double* __restrict__ val, const TX* __restrict__ x,
                                                 double* __restrict__ y) {
  int R = blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= n) return;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int p = rp[R]; p < rp[R + 1]; ++p) {
    const double* A = val + 9L * p;
    long J = 3L * col[p];
    double v0 = (double)x[J], v1 = (double)x[J + 1], v2 = (double)x[J + 2];
    a0 = fma(A[0], v0, fma(A[1], v1, fma(A[2], v2, a0)));
    a1 = fma(A[3], v0, fma(A[4], v1, fma(A[5], v2, a1)));
    a2 = fma(A[6], v0, fma(A[7], v1, fma(A[8], v2, a2)));
  }
  y[3L * R] = a0;
  y[3L * R + 1] = a1;
  y[3L * R + 2] = a2;
}

// r = b - A x on the rows of each chunk, partial |r|^2 and |b|^2
__global__ void __launch_bounds__(256) kgb_residual(const Chunk* __restrict__ ch, int nchunks,
                                                   const int* __restrict__ rp, const int* __restrict__ col,
                                                   const double* __restrict__ val, const double* __restrict__ b,
                                                   const double* __restrict__ x, double* __restrict__ r,
                                                   double* __restrict__ partial) {
  Chunk k = ch[blockIdx.x];
  double acc[2] = {0, 0};
  for (long R = k.e0 / 3 + threadIdx.x; R < k.e1 / 3; R += blockDim.x) {
    double a0 = b[3 * R], a1 = b[3 * R + 1], a2 = b[3 * R + 2];
    acc[1] += a0 * a0 + a1 * a1 + a2 * a2;
    for (int p = rp[R]; p < rp[R + 1]; ++p) {
      const double* A = val + 9L * p;
      long J = 3L * col[p];
      double v0 = x[J], v1 = x[J + 1], v2 = x[J + 2];
      a0 = fma(-A[0], v0, fma(-A[1], v1, fma(-A[2], v2, a0)));
      a1 = fma(-A[3], v0, fma(-A[4], v1, fma(-A[5], v2, a1)));
      a2 = fma(-A[6], v0, fma(-A[7], v1, fma(-A[8], v2, a2)));
    }
    r[3 * R] = a0;
    r[3 * R + 1] = a1;
    r[3 * R + 2] = a2;
    acc[0] += a0 * a0 + a1 * a1 + a2 * a2;
  }
  chunk_reduce_store<2>(acc, partial, 2, nchunks);
}

// ---------------------------------------------------------------------------
// K-cycle on a union level: the two inner GCR steps of every instance that
// has the K-cycle there, with 8 scalars per instance (ks[8 i + q], the same
// fields as the single solve's), partial dots per chunk of one instance's
// rows and per-instance sums in chunk order.  row_inst[R] is the instance of
// union row R, or -1 for rows without the K-cycle (instances whose coarsest
// level this is: their correction is the direct solve z1 itself).
// ---------------------------------------------------------------------------
template <typename T, int NQ>
__global__ void __launch_bounds__(256) kbk_dots(const Chunk* __restrict__ ch, int nchunks, const T* __restrict__ u0,
                                                const T* __restrict__ v0, const T* __restrict__ u1,
                                                const T* __restrict__ v1, double* __restrict__ partial) {
  Chunk k = ch[blockIdx.x];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0;
  for (long t = k.e0 + threadIdx.x; t < k.e1; t += blockDim.x) {
    acc[0] += (double)u0[t] * (double)v0[t];
    if (NQ > 1) acc[NQ - 1] += (double)u1[t] * (double)v1[t];
  }
  chunk_reduce_store<NQ>(acc, partial, NQ, nchunks);
}

// ks[8 i + field + q] = sum of partial[q][chunks of instance i]
__global__ void kbk_finish(const double* __restrict__ partial, int nchunks, const int* __restrict__ iptr,
                           double* __restrict__ ks, int field) {
  __shared__ double sh[kBlock];
  int i = blockIdx.x, q = blockIdx.y;
  double a = 0;
  for (int k = iptr[i] + threadIdx.x; k < iptr[i + 1]; k += kBlock) a += partial[(long)q * nchunks + k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ks[8L * i + field + q] = sh[0];
}

// y = u - (ks[8 i + num] / ks[8 i + den]) v per element of instance i (a
// zero denominator means v = 0 there: coefficient 0); rows without the
// K-cycle copy u
template <typename T>
__global__ void kbk_axpy(long n3, const int* __restrict__ row_inst, const T* u, const T* __restrict__ v,
                         const double* __restrict__ ks, int num, int den, T* y) {  // y may alias u
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n3) return;
  int i = row_inst[t / 3];
  double f = 0;
  if (i >= 0) {
    double d = ks[8L * i + den];
    f = d > 0 ? ks[8L * i + num] / d : 0.0;
  }
  y[t] = u[t] - (T)f * v[t];
}

// x = y1 z1 + y2 x per instance (as kk_combine); rows without the K-cycle
// take z1
template <typename T>
__global__ void kbk_combine(long n3, const int* __restrict__ row_inst, const T* __restrict__ z1, T* __restrict__ x,
                            const double* __restrict__ ks) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n3) return;
  int i = row_inst[t / 3];
  if (i < 0) {
    x[t] = z1[t];
    return;
  }
  const double* k = ks + 8L * i;
  double y2 = k[3] > 0 ? k[4] / k[3] : 0.0;
  double y1 = k[0] > 0 ? (k[1] - k[2] * y2) / k[0] : 0.0;
  x[t] = (T)(y1 * (double)z1[t] + y2 * (double)x[t]);
}

// per-instance scalar updates (one thread per instance, the same formulas as
// the single-instance kernels)
__global__ void kgb_gs_coef(GcrScal* S, int ninst, int j, int first) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  GcrScal& s = S[i];
  if (!first && s.pass2 == 0.0) return;  // second pass not needed for this instance
  double proj = 0;
  for (int q = 0; q < j; ++q) {
    double gm = s.s[q] * s.d[q];
    s.gam[q * kMaxRestart + j] = first ? gm : s.gam[q * kMaxRestart + j] + gm;
    s.coef[q] = gm * s.s[q];
    proj += gm * gm;
  }
  if (first) s.pass2 = (s.cn2 - proj < 0.5 * s.cn2) ? 1.0 : 0.0;
}
// as k_norm_coef; an instance that is not active keeps its residual
__global__ void kgb_norm_coef(GcrScal* S, int ninst, int j, const int* __restrict__ act) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  GcrScal& s = S[i];
  double g = sqrt(s.cc);
  s.gjj = g;
  s.gam[j * kMaxRestart + j] = g;
  double sj = 1.0 / g;
  s.s[j] = sj;
  s.alpha[j] = sj * s.cr;
  s.rcoef = act[i] ? s.alpha[j] * sj : 0.0;
}
__global__ void kgb_backsub(GcrScal* S, int ninst, const int* __restrict__ jdone) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  GcrScal& s = S[i];
  int m = jdone[i];
  for (int q = m - 1; q >= 0; --q) {
    double a = s.alpha[q];
    for (int k = q + 1; k < m; ++k) a -= s.gam[q * kMaxRestart + k] * s.y[k];
    s.y[q] = a / s.gam[q * kMaxRestart + q];
  }
}
// the scalars the host reads each iteration: {rn2, gjj} per instance
__global__ void kgb_head(const GcrScal* __restrict__ S, int ninst, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  out[2 * i] = S[i].rn2;
  out[2 * i + 1] = S[i].gjj;
}
__global__ void kgb_head2(const GcrScal* __restrict__ S, int ninst, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  out[2 * i] = S[i].rn2;
  out[2 * i + 1] = S[i].bn2;
}

}  // namespace llmg
