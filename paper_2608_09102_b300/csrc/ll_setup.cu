// Symbolic setup on the GPU: grid graph, pairwise-matching aggregation (two
// passes per level, Sec. 3.1.1), graph contraction (integer Galerkin of the
// weight graph), Jones-Plassmann colouring, BSR patterns and the slot maps of
// the Galerkin products (Eq. galerkin, Eq. Ac_direct).  Integer work only;
// results are independent of thread scheduling (atomics are used only for
// order-free operations -- counts and minima -- or are followed by a sort).
#include <limits.h>

#include <algorithm>

#include "ll_internal.cuh"
#include "ll_setup.cuh"

namespace llmg {

// ---------------------------------------------------------------------------
// exclusive prefix sum of int32 (three-phase: block scans, scan of the block
// totals, add-back), returns the total
// ---------------------------------------------------------------------------
__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ bsum, int n) {
  __shared__ int s[1024];
  int i = blockIdx.x * 1024 + threadIdx.x;
  int v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}
__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ boff, int n) {
  int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

static void scan_rec(const int* in, int* out, int n, cudaStream_t s) {
  int nb = cdiv(n, 1024);
  DBuf<int> bsum, boff;
  bsum.alloc(nb);
  boff.alloc(nb);
  k_scan_block<<<nb, 1024, 0, s>>>(in, out, bsum, n);
  LL_LAUNCHED();
  if (nb > 1) {
    scan_rec(bsum, boff, nb, s);
    k_scan_add<<<nb, 1024, 0, s>>>(out, boff, n);
    LL_LAUNCHED();
  }
  LL_CU(cudaStreamSynchronize(s));  // before the temporaries are released
}

// out[0..n) = exclusive scan of in, out[n] = total; returns the total
int exclusive_scan(const int* in, int* out, int n, cudaStream_t s) {
  if (n == 0) {
    LL_CU(cudaMemsetAsync(out, 0, sizeof(int), s));
    return 0;
  }
  scan_rec(in, out, n, s);
  int last_in = 0, last_out = 0;
  LL_CU(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  LL_CU(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  LL_CU(cudaStreamSynchronize(s));
  int total = last_in + last_out;
  LL_CU(cudaMemcpyAsync(out + n, &total, sizeof(int), cudaMemcpyHostToDevice, s));
  LL_CU(cudaStreamSynchronize(s));
  return total;
}

static int read_int(const int* d, cudaStream_t s) {
  int v = 0;
  LL_CU(cudaMemcpyAsync(&v, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  LL_CU(cudaStreamSynchronize(s));
  return v;
}

__global__ void k_fill(int* p, int v, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
static void fill(int* p, int v, long n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<<<cdiv(n, kBlock), kBlock, 0, s>>>(p, v, n);
  LL_LAUNCHED();
}

// ---------------------------------------------------------------------------
// level-0 graph: face neighbours of the grid, weight 1, natural cell order
// ---------------------------------------------------------------------------
__device__ __forceinline__ int grid_neighbours(int k, int nx, int ny, int nz, int* nb) {
  int x = k % nx, t = k / nx, y = t % ny, z = t / ny;
  int d = 0;
  long nxy = (long)nx * ny;
  if (z > 0) nb[d++] = (int)(k - nxy);
  if (y > 0) nb[d++] = k - nx;
  if (x > 0) nb[d++] = k - 1;
  if (x < nx - 1) nb[d++] = k + 1;
  if (y < ny - 1) nb[d++] = k + nx;
  if (z < nz - 1) nb[d++] = (int)(k + nxy);
  return d;
}
__global__ void k_grid_degree(int n, int nx, int ny, int nz, int* deg) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int nb[6];
  deg[k] = grid_neighbours(k, nx, ny, nz, nb);
}
__global__ void k_grid_fill(int n, int nx, int ny, int nz, const int* rp, int* col, int* w) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int nb[6];
  int d = grid_neighbours(k, nx, ny, nz, nb);
  for (int t = 0; t < d; ++t) {
    col[rp[k] + t] = nb[t];
    w[rp[k] + t] = 1;
  }
}

void build_grid_graph(int nx, int ny, int nz, DevGraph& g, cudaStream_t s) {
  int n = nx * ny * nz;
  g.n = n;
  g.rowptr.alloc(n + 1);
  DBuf<int> deg;
  deg.alloc(n);
  k_grid_degree<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, nx, ny, nz, deg);
  LL_LAUNCHED();
  g.nnz = exclusive_scan(deg, g.rowptr, n, s);
  g.col.alloc(g.nnz);
  g.w.alloc(g.nnz);
  k_grid_fill<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, nx, ny, nz, g.rowptr, g.col, g.w);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// one pass of pairwise matching (handshake rounds)
// ---------------------------------------------------------------------------
// Edge order: weight, then hash of the endpoints, then the smaller lower end,
// then the smaller upper end.  Returns true when (wa, ha, a0, a1) is larger.
__device__ __forceinline__ bool edge_better(int wa, uint32_t ha, int a0, int a1, int wb, uint32_t hb, int b0,
                                            int b1) {
  if (wa != wb) return wa > wb;
  if (ha != hb) return ha > hb;
  if (a0 != b0) return a0 < b0;
  return a1 < b1;
}

__global__ void k_maxw(int n, const int* __restrict__ rp, const int* __restrict__ w, int* __restrict__ maxw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) m = max(m, w[p]);
  maxw[i] = m;
}

// Every unmatched node picks its best unmatched candidate neighbour (an edge
// whose weight is at least a quarter of the largest weight at either end).
__global__ void k_choose(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ w,
                         const int* __restrict__ maxw, const int* __restrict__ mate, uint32_t seed,
                         int* __restrict__ best) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = -1;
  if (mate[i] < 0) {
    int bw = 0, b0 = 0, b1 = 0;
    uint32_t bh = 0;
    int mi = maxw[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = col[p], wj = w[p];
      if (mate[j] >= 0) continue;
      if (4 * wj < mi && 4 * wj < maxw[j]) continue;
      int e0 = min(i, j), e1 = max(i, j);
      uint32_t eh = pair_key((uint32_t)e0, (uint32_t)e1, seed);
      if (b < 0 || edge_better(wj, eh, e0, e1, bw, bh, b0, b1)) {
        b = j;
        bw = wj;
        bh = eh;
        b0 = e0;
        b1 = e1;
      }
    }
  }
  best[i] = b;
}

// Mutual choices become pairs.
__global__ void k_handshake(int n, const int* __restrict__ best, int* __restrict__ mate, int* __restrict__ formed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = best[i];
  if (mate[i] < 0 && b >= 0 && best[b] == i) {
    mate[i] = b;
    *formed = 1;
  }
}

// Representative of each node's group: the smaller node of its pair; a
// leftover joins the pair of its best neighbour (over all neighbours) when
// that neighbour is matched and `attach` is set.
__global__ void k_represent(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const int* __restrict__ w, const int* __restrict__ mate, uint32_t seed, int attach,
                            int* __restrict__ rep) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int mi = mate[i];
  int r = (mi >= 0 && mi < i) ? mi : i;
  if (attach && mi < 0) {
    int bj = -1, bw = 0, b0 = 0, b1 = 0;
    uint32_t bh = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = col[p], wj = w[p];
      int e0 = min(i, j), e1 = max(i, j);
      uint32_t eh = pair_key((uint32_t)e0, (uint32_t)e1, seed);
      if (bj < 0 || edge_better(wj, eh, e0, e1, bw, bh, b0, b1)) {
        bj = j;
        bw = wj;
        bh = eh;
        b0 = e0;
        b1 = e1;
      }
    }
    if (bj >= 0 && mate[bj] >= 0) r = min(bj, mate[bj]);
  }
  rep[i] = r;
}

__global__ void k_min_member(int n, const int* __restrict__ rep, int* __restrict__ minmem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMin(&minmem[rep[i]], i);
}
__global__ void k_is_first(int n, const int* __restrict__ rep, const int* __restrict__ minmem, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = minmem[rep[i]] == i ? 1 : 0;
}
__global__ void k_number(int n, const int* __restrict__ rep, const int* __restrict__ minmem,
                         const int* __restrict__ pos, int* __restrict__ group) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) group[i] = pos[minmem[rep[i]]];
}

// Number groups given by a representative array by the rank of their smallest
// member; returns the number of groups.
static int number_groups(int n, const int* rep, int* group, cudaStream_t s) {
  DBuf<int> minmem, flag, pos;
  minmem.alloc(n);
  flag.alloc(n);
  pos.alloc(n + 1);
  fill(minmem, INT_MAX, n, s);
  int nb = cdiv(n, kBlock);
  k_min_member<<<nb, kBlock, 0, s>>>(n, rep, minmem);
  LL_LAUNCHED();
  k_is_first<<<nb, kBlock, 0, s>>>(n, rep, minmem, flag);
  LL_LAUNCHED();
  int ng = exclusive_scan(flag, pos, n, s);
  k_number<<<nb, kBlock, 0, s>>>(n, rep, minmem, pos, group);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
  return ng;
}

int matching_pass(const DevGraph& g, int rounds, uint32_t seed, int attach, int* group, cudaStream_t s) {
  int n = g.n;
  if (n == 0) return 0;
  DBuf<int> maxw, mate, best, rep, formed;
  maxw.alloc(n);
  mate.alloc(n);
  best.alloc(n);
  rep.alloc(n);
  formed.alloc(1);
  int nb = cdiv(n, kBlock);
  k_maxw<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.w, maxw);
  LL_LAUNCHED();
  fill(mate, -1, n, s);
  for (int r = 0; r < rounds; ++r) {
    LL_CU(cudaMemsetAsync(formed, 0, sizeof(int), s));
    k_choose<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.col, g.w, maxw, mate, seed, best);
    LL_LAUNCHED();
    k_handshake<<<nb, kBlock, 0, s>>>(n, best, mate, formed);
    LL_LAUNCHED();
    if (!read_int(formed, s)) break;
  }
  k_represent<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.col, g.w, mate, seed, attach, rep);
  LL_LAUNCHED();
  int ng = number_groups(n, rep, group, s);
  LL_CU(cudaStreamSynchronize(s));
  return ng;
}

// ---------------------------------------------------------------------------
// members of groups (sorted ascending) and graph contraction
// ---------------------------------------------------------------------------
__global__ void k_count_members(int n, const int* __restrict__ map, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && map[i] >= 0) atomicAdd(&cnt[map[i]], 1);  // map < 0: padding slot
}
__global__ void k_place_members(int n, const int* __restrict__ map, const int* __restrict__ mptr,
                                int* __restrict__ next, int* __restrict__ mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && map[i] >= 0) {
    int g = map[i];
    mem[mptr[g] + atomicAdd(&next[g], 1)] = i;
  }
}
__global__ void k_sort_segments(int nseg, const int* __restrict__ ptr, int* __restrict__ key, int* __restrict__ v1,
                                int* __restrict__ v2) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nseg) return;
  int a = ptr[g], b = ptr[g + 1];
  for (int i = a + 1; i < b; ++i) {
    int k = key[i];
    int x1 = v1 ? v1[i] : 0, x2 = v2 ? v2[i] : 0;
    int j = i - 1;
    while (j >= a && key[j] > k) {
      key[j + 1] = key[j];
      if (v1) v1[j + 1] = v1[j];
      if (v2) v2[j + 1] = v2[j];
      --j;
    }
    key[j + 1] = k;
    if (v1) v1[j + 1] = x1;
    if (v2) v2[j + 1] = x2;
  }
}

// mptr (nc+1) and mem (n): members of each coarse node, ascending
void build_members(int n, const int* map, int nc, DBuf<int>& mptr, DBuf<int>& mem, cudaStream_t s) {
  DBuf<int> cnt, next;
  cnt.alloc(nc);
  next.alloc(nc);
  cnt.zero(s);
  next.zero(s);
  mptr.alloc(nc + 1);
  mem.alloc(n);
  k_count_members<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, map, cnt);
  LL_LAUNCHED();
  exclusive_scan(cnt, mptr, nc, s);
  k_place_members<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, map, mptr, next, mem);
  LL_LAUNCHED();
  k_sort_segments<<<cdiv(nc, kBlock), kBlock, 0, s>>>(nc, mptr, mem, nullptr, nullptr);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

__global__ void k_member_degree(int nc, const int* __restrict__ mptr, const int* __restrict__ mem,
                                const int* __restrict__ rp, int* __restrict__ d) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int s = 0;
  for (int t = mptr[I]; t < mptr[I + 1]; ++t) s += rp[mem[t] + 1] - rp[mem[t]];
  d[I] = s;
}
// gather (coarse neighbour, weight) pairs of each coarse node, sort them and
// merge duplicates in place; ucnt[I] = number of distinct neighbours
__global__ void k_contract_gather(int nc, const int* __restrict__ mptr, const int* __restrict__ mem,
                                  const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ w,
                                  const int* __restrict__ map, const int* __restrict__ sptr, int* __restrict__ sj,
                                  int* __restrict__ sw, int* __restrict__ ucnt) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int a = sptr[I], e = a;
  for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
    int i = mem[t];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int J = map[col[p]];
      if (J == I) continue;
      sj[e] = J;
      sw[e] = w[p];
      ++e;
    }
  }
  for (int i = a + 1; i < e; ++i) {  // insertion sort by neighbour
    int k = sj[i], x = sw[i], j = i - 1;
    while (j >= a && sj[j] > k) {
      sj[j + 1] = sj[j];
      sw[j + 1] = sw[j];
      --j;
    }
    sj[j + 1] = k;
    sw[j + 1] = x;
  }
  int u = a;
  for (int i = a; i < e; ++i) {
    if (u > a && sj[u - 1] == sj[i]) {
      sw[u - 1] += sw[i];
    } else {
      sj[u] = sj[i];
      sw[u] = sw[i];
      ++u;
    }
  }
  ucnt[I] = u - a;
}
__global__ void k_contract_fill(int nc, const int* __restrict__ sptr, const int* __restrict__ sj,
                                const int* __restrict__ sw, const int* __restrict__ crp, int* __restrict__ ccol,
                                int* __restrict__ cw) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int a = sptr[I], o = crp[I], u = crp[I + 1] - crp[I];
  for (int t = 0; t < u; ++t) {
    ccol[o + t] = sj[a + t];
    cw[o + t] = sw[a + t];
  }
}

// Weight graph of the coarse nodes: w_IJ = sum of the weights of the fine
// edges between I and J (I != J).
void contract_graph(const DevGraph& g, const int* map, int nc, const int* mptr, const int* mem, DevGraph& out,
                    cudaStream_t s) {
  out.n = nc;
  out.rowptr.alloc(nc + 1);
  DBuf<int> deg, sptr, sj, sw, ucnt;
  deg.alloc(nc);
  sptr.alloc(nc + 1);
  ucnt.alloc(nc);
  int nb = cdiv(nc, kBlock);
  k_member_degree<<<nb, kBlock, 0, s>>>(nc, mptr, mem, g.rowptr, deg);
  LL_LAUNCHED();
  int tot = exclusive_scan(deg, sptr, nc, s);
  sj.alloc(tot);
  sw.alloc(tot);
  k_contract_gather<<<nb, kBlock, 0, s>>>(nc, mptr, mem, g.rowptr, g.col, g.w, map, sptr, sj, sw, ucnt);
  LL_LAUNCHED();
  out.nnz = exclusive_scan(ucnt, out.rowptr, nc, s);
  out.col.alloc(out.nnz);
  out.w.alloc(out.nnz);
  k_contract_fill<<<nb, kBlock, 0, s>>>(nc, sptr, sj, sw, out.rowptr, out.col, out.w);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

__global__ void k_compose(int n, const int* __restrict__ g1, const int* __restrict__ g2, int* __restrict__ agg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) agg[i] = g2[g1[i]];
}

// One level: pass 1 (pairs), pass 2 on the pair graph (leftovers attached),
// composed.  Numbering by smallest member carries through the composition.
int aggregate_level(const DevGraph& g, int rounds, uint32_t seed, int* agg, cudaStream_t s) {
  int n = g.n;
  DBuf<int> g1, g2, mptr, mem;
  g1.alloc(n);
  int n1 = matching_pass(g, rounds, seed, 0, g1, s);
  build_members(n, g1, n1, mptr, mem, s);
  DevGraph pg;
  contract_graph(g, g1, n1, mptr, mem, pg, s);
  g2.alloc(n1);
  int n2 = matching_pass(pg, rounds, seed, 1, g2, s);
  k_compose<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, g1, g2, agg);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
  return n2;
}

// ---------------------------------------------------------------------------
// Colouring of an aggregated level: Jones-Plassmann rounds with priority
// (degree, node_key, index), then kRecolourPasses passes of iterated greedy
// recolouring (the classes visited from the highest colour down, each node
// taking the smallest colour unused by the neighbours already recoloured)
// ---------------------------------------------------------------------------
constexpr int kRecolourPasses = 4;

// does node j take precedence over node i in the rounds?
__device__ __forceinline__ bool node_beats(const int* __restrict__ rp, int j, int i, uint32_t seed) {
  int dj = rp[j + 1] - rp[j], di = rp[i + 1] - rp[i];
  if (dj != di) return dj > di;
  uint32_t hj = node_key((uint32_t)j, seed), hi = node_key((uint32_t)i, seed);
  if (hj != hi) return hj > hi;
  return j > i;
}

// smallest colour below 128 not in the two bit masks; -1 if none
__device__ __forceinline__ int first_free(unsigned long long used0, unsigned long long used1) {
  if (~used0) return __ffsll((long long)~used0) - 1;
  if (~used1) return 64 + __ffsll((long long)~used1) - 1;
  return -1;
}

__device__ __forceinline__ void mark_used(int cj, unsigned long long& used0, unsigned long long& used1) {
  if (cj >= 0 && cj < 64) used0 |= 1ull << cj;
  else if (cj >= 64 && cj < 128) used1 |= 1ull << (cj - 64);
}

__global__ void k_colour_round(int n, const int* __restrict__ rp, const int* __restrict__ col, uint32_t seed,
                               const int* __restrict__ cin, int* __restrict__ cout, int* __restrict__ left,
                               int* __restrict__ overflow) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int ci = cin[i];
  if (ci >= 0) {
    cout[i] = ci;
    return;
  }
  bool wins = true;
  unsigned long long used0 = 0, used1 = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = col[p], cj = cin[j];
    if (cj < 0) {
      if (node_beats(rp, j, i, seed)) wins = false;
    } else {
      mark_used(cj, used0, used1);
    }
  }
  if (!wins) {
    cout[i] = -1;
    atomicAdd(left, 1);
    return;
  }
  int c = first_free(used0, used1);
  if (c < 0) {
    c = 0;
    *overflow = 1;
  }
  cout[i] = c;
}

// one class of a recolouring pass: the nodes of old colour c take the
// smallest colour unused by their already recoloured neighbours (cnew >= 0)
__global__ void k_recolour_class(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const int* __restrict__ cold, int c, int* __restrict__ cnew,
                                 int* __restrict__ overflow) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cold[i] != c) return;
  unsigned long long used0 = 0, used1 = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) mark_used(cnew[col[p]], used0, used1);
  int k = first_free(used0, used1);
  if (k < 0) {
    k = 0;
    *overflow = 1;
  }
  cnew[i] = k;
}

static int max_colour(const int* colour, int n, cudaStream_t s) {
  std::vector<int> h(n);
  LL_CU(cudaMemcpyAsync(h.data(), colour, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  LL_CU(cudaStreamSynchronize(s));
  int mx = -1;
  for (int v : h) mx = std::max(mx, v);
  return mx;
}

// returns the number of colours, or -1 when more than kMaxColours are needed
int colour_graph(const DevGraph& g, uint32_t seed, int* colour, cudaStream_t s) {
  int n = g.n;
  DBuf<int> buf, left, ovf;
  buf.alloc(n);
  left.alloc(1);
  ovf.alloc(1);
  ovf.zero(s);
  fill(colour, -1, n, s);
  int* a = colour;
  int* b = buf;
  int nb = cdiv(n, kBlock);
  for (int round = 0; round <= n; ++round) {
    LL_CU(cudaMemsetAsync(left, 0, sizeof(int), s));
    k_colour_round<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.col, seed, a, b, left, ovf);
    LL_LAUNCHED();
    std::swap(a, b);
    if (read_int(left, s) == 0) break;
  }
  if (read_int(ovf, s)) return -1;
  int ncol = max_colour(a, n, s) + 1;
  for (int pass = 0; pass < kRecolourPasses; ++pass) {
    fill(b, -1, n, s);
    for (int c = ncol - 1; c >= 0; --c) {
      k_recolour_class<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.col, a, c, b, ovf);
      LL_LAUNCHED();
    }
    std::swap(a, b);
    if (read_int(ovf, s)) return -1;
    ncol = max_colour(a, n, s) + 1;
  }
  if (a != colour) LL_CU(cudaMemcpyAsync(colour, a, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  LL_CU(cudaStreamSynchronize(s));
  return ncol;
}

// Row-work key of a coarse row, by which the rows of one colour class are
// ordered so that the rows sharing a warp in the sweeps need the same number
// of block slots and few float64 lanes idle:
//  * bucketed (the per-class kernels with kRowLanes or 8 lanes per row):
//    16 x ceil(pre / kRowLanes) + ceil(deg / kRowLanes), each capped at 15;
//  * exact (the one-row-per-thread SELL-32 sweeps, where a chunk of 32 rows
//    visits as many slots as its longest row): 32 x min(pre, 31) + min(deg, 31);
// pre = neighbours of lower colour (the forward sweep's blocks), deg = all
// neighbours (the backward sweep's).
__global__ void k_row_work_keys(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const int* __restrict__ colour, int exact, int* __restrict__ key) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int pre = 0, deg = rp[i + 1] - rp[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) pre += colour[ci[p]] < colour[i];
  if (exact) {
    key[i] = 32 * min(pre, 31) + min(deg, 31);
    return;
  }
  int sp = min((pre + kRowLanes - 1) / kRowLanes, 15), sd = min((deg + kRowLanes - 1) / kRowLanes, 15);
  key[i] = 16 * sp + sd;
}

void row_work_keys(const DevGraph& g, const int* colour, bool exact, DBuf<int>& key, cudaStream_t s) {
  key.alloc(g.n);
  k_row_work_keys<<<cdiv(g.n, kBlock), kBlock, 0, s>>>(g.n, g.rowptr, g.col, colour, exact ? 1 : 0, key);
  LL_LAUNCHED();
}

// Stable counting sort of the rows by bucket b = colour * nkeys + key, in
// tiles of kSortTile rows: counts per (bucket, tile), one exclusive scan in
// bucket-major order, then every row goes to its bucket's offset for its tile
// plus its rank among the earlier rows of its tile in the same bucket.
constexpr int kSortTile = 1024;
__global__ void k_tile_counts(int n, const int* __restrict__ colour, const int* __restrict__ key, int nkeys,
                              int ntiles, int* __restrict__ cnt) {
  int i = blockIdx.x * kSortTile + threadIdx.x;
  if (i < n) atomicAdd(&cnt[(long)(colour[i] * nkeys + key[i]) * ntiles + blockIdx.x], 1);  // counts only
}
__global__ void __launch_bounds__(kSortTile) k_tile_scatter(int n, const int* __restrict__ colour,
                                                            const int* __restrict__ key, int nkeys, int ntiles,
                                                            const int* __restrict__ off, int* __restrict__ out) {
  __shared__ int bk[kSortTile];
  int i = blockIdx.x * kSortTile + threadIdx.x;
  int b = i < n ? colour[i] * nkeys + key[i] : -1;
  bk[threadIdx.x] = b;
  __syncthreads();
  if (i >= n) return;
  int rank = 0;
  for (int j = 0; j < (int)threadIdx.x; ++j) rank += bk[j] == b;
  out[off[(long)b * ntiles + blockIdx.x] + rank] = i;
}
__global__ void k_colour_counts(int n, const int* __restrict__ colour, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[colour[i]], 1);  // counts only: order-independent
}

// rows of each colour, crow[cptr[c] .. cptr[c+1]), ordered by (key, index)
void colour_classes(int n, const int* colour, int ncol, const int* key, int nkeys, DBuf<int>& cptr, DBuf<int>& crow,
                    std::vector<int>& h_cptr, cudaStream_t s) {
  int ntiles = cdiv(n, kSortTile);
  long nb = (long)ncol * nkeys * ntiles;
  if (nb >= (1L << 31) - 1) throw Status{LL_ELIMIT};
  DBuf<int> cnt, off, ccnt;
  cnt.alloc(nb);
  off.alloc(nb + 1);
  ccnt.alloc(ncol);
  crow.alloc(n);
  cnt.zero(s);
  ccnt.zero(s);
  k_tile_counts<<<ntiles, kSortTile, 0, s>>>(n, colour, key, nkeys, ntiles, cnt);
  LL_LAUNCHED();
  if (exclusive_scan(cnt, off, (int)nb, s) != n) {
    note_internal_error("bucket counts do not sum to the row count", __FILE__, __LINE__);
    throw Status{LL_ECUDA};
  }
  k_tile_scatter<<<ntiles, kSortTile, 0, s>>>(n, colour, key, nkeys, ntiles, off, crow);
  LL_LAUNCHED();
  k_colour_counts<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, colour, ccnt);
  LL_LAUNCHED();
  std::vector<int> h_cnt(ncol);
  LL_CU(cudaMemcpyAsync(h_cnt.data(), ccnt.p, ncol * sizeof(int), cudaMemcpyDeviceToHost, s));
  LL_CU(cudaStreamSynchronize(s));
  h_cptr.assign(ncol + 1, 0);
  for (int c = 0; c < ncol; ++c) h_cptr[c + 1] = h_cptr[c] + h_cnt[c];
  cptr.alloc(ncol + 1);
  LL_CU(cudaMemcpyAsync(cptr.p, h_cptr.data(), (ncol + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  LL_CU(cudaStreamSynchronize(s));
}

// The blocks of a Galerkin level in order of decreasing slot-list length
// (ties by index): the Galerkin threads take them in this order, so that the
// lanes of a warp sum lists of about the same length (the diagonal blocks'
// lists are several times longer than the others').
constexpr int kLenKeys = 64;
__global__ void k_len_keys(int n, const int* __restrict__ sptr, int* __restrict__ key, int* __restrict__ zero) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int len = sptr[p + 1] - sptr[p];
  key[p] = kLenKeys - 1 - (len < kLenKeys - 1 ? len : kLenKeys - 1);
  zero[p] = 0;
}
void order_by_length(int n, const int* sptr, DBuf<int>& perm, cudaStream_t s) {
  DBuf<int> key, zero, cptr;
  key.alloc(n);
  zero.alloc(n);
  k_len_keys<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, sptr, key, zero);
  LL_LAUNCHED();
  std::vector<int> h_cptr;
  colour_classes(n, zero, 1, key, kLenKeys, cptr, perm, h_cptr, s);
}

// ---------------------------------------------------------------------------
// BSR pattern of a coarse operator: graph neighbours plus the diagonal
// ---------------------------------------------------------------------------
__global__ void k_bsr_pattern(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                              int* __restrict__ rowptr, int* __restrict__ col, int* __restrict__ diag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  rowptr[i] = grp[i] + i;
  if (i == n) return;
  int o = grp[i] + i;
  bool placed = false;
  for (int p = grp[i]; p < grp[i + 1]; ++p) {
    if (!placed && gcol[p] > i) {
      diag[i] = o;
      col[o++] = i;
      placed = true;
    }
    col[o++] = gcol[p];
  }
  if (!placed) {
    diag[i] = o;
    col[o++] = i;
  }
}

void bsr_pattern(const DevGraph& g, DBuf<int>& rowptr, DBuf<int>& col, DBuf<int>& diag, int& nnzb, cudaStream_t s) {
  int n = g.n;
  nnzb = g.nnz + n;
  rowptr.alloc(n + 1);
  col.alloc(nnzb);
  diag.alloc(n);
  k_bsr_pattern<<<cdiv(n + 1, kBlock), kBlock, 0, s>>>(n, g.rowptr, g.col, rowptr, col, diag);
  LL_LAUNCHED();
}

// position of block column J in BSR row I (-1 if absent)
__device__ __forceinline__ int find_block(const int* __restrict__ rowptr, const int* __restrict__ col, int I, int J) {
  int a = rowptr[I], b = rowptr[I + 1];
  while (a < b) {  // binary search, columns ascending
    int m = (a + b) >> 1;
    int c = col[m];
    if (c == J) return m;
    if (c < J) a = m + 1;
    else b = m;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Galerkin slot map, level 0 -> level 1.  The level-0 operator has, per cell
// k (red-black slot), the diagonal block I/dt - deg_k Chat_k and the block
// Chat_k towards each face neighbour.  Hence
//   A_1(I,J) = delta_IJ |G_I|/dt I + sum_{k in G_I} w_kJ Chat_k,
//   w_kJ = #(neighbours of k in G_J) - delta_IJ deg_k  (an integer).
// For every slot (I,J) the list of (k, w_kJ) with w_kJ != 0 is stored,
// sorted by k.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rb_neighbours(const GridGeom g, int x, int y, int z, int* nbx, int* nby, int* nbz) {
  int d = 0;
  if (z > 0) nbx[d] = x, nby[d] = y, nbz[d++] = z - 1;
  if (y > 0) nbx[d] = x, nby[d] = y - 1, nbz[d++] = z;
  if (x > 0) nbx[d] = x - 1, nby[d] = y, nbz[d++] = z;
  if (x < g.nx - 1) nbx[d] = x + 1, nby[d] = y, nbz[d++] = z;
  if (y < g.ny - 1) nbx[d] = x, nby[d] = y + 1, nbz[d++] = z;
  if (z < g.nz - 1) nbx[d] = x, nby[d] = y, nbz[d++] = z + 1;
  return d;
}

// pass 0: count per slot; pass 1: place entries
__global__ void k_slots_l1(GridGeom g, const int* __restrict__ agg_nat, const int* __restrict__ rowptr,
                           const int* __restrict__ col, int pass, int* __restrict__ cnt, const int* __restrict__ sptr,
                           int* __restrict__ sidx, int* __restrict__ sw) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  int x = (int)(k % g.nx);
  long t = k / g.nx;
  int y = (int)(t % g.ny), z = (int)(t / g.ny);
  int I = agg_nat[k];
  int nbx[6], nby[6], nbz[6];
  int d = rb_neighbours(g, x, y, z, nbx, nby, nbz);
  int J[7], wJ[7], u = 0;
  J[u] = I;
  wJ[u++] = -d;
  for (int q = 0; q < d; ++q) {
    long l = nbx[q] + (long)g.nx * (nby[q] + (long)g.ny * nbz[q]);
    int a = agg_nat[l];
    int f = -1;
    for (int v = 0; v < u; ++v)
      if (J[v] == a) f = v;
    if (f < 0) {
      J[u] = a;
      wJ[u++] = 1;
    } else {
      wJ[f] += 1;
    }
  }
  int c = (x + y + z) & 1;
  int slot_k = (int)(c * g.nh + ((long)z * g.ny + y) * g.nxh + (x >> 1));
  for (int v = 0; v < u; ++v) {
    if (wJ[v] == 0) continue;
    int s = find_block(rowptr, col, I, J[v]);
    if (s < 0) continue;  // cannot happen: the pattern is the contracted graph
    if (pass == 0) {
      atomicAdd(&cnt[s], 1);
    } else {
      int p = sptr[s] + atomicAdd(&cnt[s], 1);
      sidx[p] = slot_k;
      sw[p] = wJ[v];
    }
  }
}

void slot_map_level1(const GridGeom& g, const int* agg_nat, const DevGraph& g1, const int* rowptr, const int* col,
                     int nnzb, DBuf<int>& sptr, DBuf<int>& sidx, DBuf<int>& sw, cudaStream_t s) {
  (void)g1;
  DBuf<int> cnt;
  cnt.alloc(nnzb);
  cnt.zero(s);
  sptr.alloc(nnzb + 1);
  int nb = cdiv(g.n, kBlock);
  k_slots_l1<<<nb, kBlock, 0, s>>>(g, agg_nat, rowptr, col, 0, cnt, nullptr, nullptr, nullptr);
  LL_LAUNCHED();
  int tot = exclusive_scan(cnt, sptr, nnzb, s);
  sidx.alloc(tot);
  sw.alloc(tot);
  cnt.zero(s);
  k_slots_l1<<<nb, kBlock, 0, s>>>(g, agg_nat, rowptr, col, 1, cnt, sptr, sidx, sw);
  LL_LAUNCHED();
  k_sort_segments<<<cdiv(nnzb, kBlock), kBlock, 0, s>>>(nnzb, sptr, sidx, sw, nullptr);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

// Galerkin slot map, level l -> l+1 (l >= 1): A_{l+1}(I',J') is the sum of the
// fine blocks A_l(I,J) with agg(I) = I', agg(J) = J'; each coarse slot lists
// its fine block positions, ascending.
__global__ void k_slots_bsr(int nf, const int* __restrict__ frp, const int* __restrict__ fcol,
                            const int* __restrict__ agg, const int* __restrict__ crp, const int* __restrict__ ccol,
                            int pass, int* __restrict__ cnt, const int* __restrict__ sptr, int* __restrict__ sidx) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nf) return;
  int Ic = agg[I];
  for (int p = frp[I]; p < frp[I + 1]; ++p) {
    int s = find_block(crp, ccol, Ic, agg[fcol[p]]);
    if (s < 0) continue;  // cannot happen: the pattern is the contracted graph
    if (pass == 0) atomicAdd(&cnt[s], 1);
    else sidx[sptr[s] + atomicAdd(&cnt[s], 1)] = p;
  }
}

void slot_map_bsr(int nf, const int* frp, const int* fcol, const int* agg, const int* crp, const int* ccol, int cnnzb,
                  DBuf<int>& sptr, DBuf<int>& sidx, cudaStream_t s) {
  DBuf<int> cnt;
  cnt.alloc(cnnzb);
  cnt.zero(s);
  sptr.alloc(cnnzb + 1);
  int nb = cdiv(nf, kBlock);
  k_slots_bsr<<<nb, kBlock, 0, s>>>(nf, frp, fcol, agg, crp, ccol, 0, cnt, nullptr, nullptr);
  LL_LAUNCHED();
  int tot = exclusive_scan(cnt, sptr, cnnzb, s);
  sidx.alloc(tot);
  cnt.zero(s);
  k_slots_bsr<<<nb, kBlock, 0, s>>>(nf, frp, fcol, agg, crp, ccol, 1, cnt, sptr, sidx);
  LL_LAUNCHED();
  k_sort_segments<<<cdiv(cnnzb, kBlock), kBlock, 0, s>>>(cnnzb, sptr, sidx, nullptr, nullptr);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// red-black slot maps of level 0
// ---------------------------------------------------------------------------
__global__ void k_rb_maps(GridGeom g, const int* __restrict__ agg_nat, int* __restrict__ agg_rb,
                          int* __restrict__ nat_of_slot) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (sl >= 2 * g.nh) return;
  int c = (int)(sl / g.nh);
  long r = sl % g.nh;
  int i = (int)(r % g.nxh);
  long row = r / g.nxh;
  int y = (int)(row % g.ny), z = (int)(row / g.ny);
  int x = 2 * i + ((c + y + z) & 1);
  if (x >= g.nx) {
    if (agg_rb) agg_rb[sl] = -1;
    nat_of_slot[sl] = -1;
    return;
  }
  long k = x + (long)g.nx * (y + (long)g.ny * z);
  if (agg_rb) agg_rb[sl] = agg_nat[k];
  nat_of_slot[sl] = (int)k;
}

void rb_maps(const GridGeom& g, const int* agg_nat, int* agg_rb, int* nat_of_slot, cudaStream_t s) {
  k_rb_maps<<<cdiv(2 * g.nh, kBlock), kBlock, 0, s>>>(g, agg_nat, agg_rb, nat_of_slot);
  LL_LAUNCHED();
}

__global__ void k_colour0_flag(int n, const int* __restrict__ mem, long nh, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = mem[i] < nh ? 1 : 0;
}
__global__ void k_members_c0(int nc, const int* __restrict__ mptr, const int* __restrict__ mem, long nh,
                             const int* __restrict__ optr, int* __restrict__ out) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int o = optr[I];
  for (int t = mptr[I]; t < mptr[I + 1]; ++t)
    if (mem[t] < nh) out[o++] = mem[t];
}
__global__ void k_count_c0(int nc, const int* __restrict__ mptr, const int* __restrict__ mem, long nh,
                           int* __restrict__ cnt) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int c = 0;
  for (int t = mptr[I]; t < mptr[I + 1]; ++t) c += mem[t] < nh;
  cnt[I] = c;
}

// members of colour 0 only (red slots are [0, nh))
void members_colour0(int nc, const int* mptr, const int* mem, long nh, DBuf<int>& optr, DBuf<int>& out,
                     cudaStream_t s) {
  DBuf<int> cnt;
  cnt.alloc(nc);
  optr.alloc(nc + 1);
  int nb = cdiv(nc, kBlock);
  k_count_c0<<<nb, kBlock, 0, s>>>(nc, mptr, mem, nh, cnt);
  LL_LAUNCHED();
  int tot = exclusive_scan(cnt, optr, nc, s);
  out.alloc(tot);
  k_members_c0<<<nb, kBlock, 0, s>>>(nc, mptr, mem, nh, optr, out);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// renumbering of a level by colour classes (rows of one colour contiguous)
// ---------------------------------------------------------------------------
__global__ void k_invert_perm(int n, const int* __restrict__ n2o, int* __restrict__ o2n) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) o2n[n2o[r]] = r;
}
__global__ void k_perm_degree(int n, const int* __restrict__ rp, const int* __restrict__ n2o, int* __restrict__ d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) d[r] = rp[n2o[r] + 1] - rp[n2o[r]];
}
__global__ void k_perm_fill(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ w,
                            const int* __restrict__ n2o, const int* __restrict__ o2n, const int* __restrict__ nrp,
                            int* __restrict__ ncol, int* __restrict__ nw) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int o = n2o[r], q = nrp[r];
  for (int p = rp[o]; p < rp[o + 1]; ++p, ++q) {
    ncol[q] = o2n[col[p]];
    nw[q] = w[p];
  }
}

// out = g with node r of out being node n2o[r] of g (columns renumbered and
// sorted ascending per row)
void permute_graph(const DevGraph& g, const int* n2o, const int* o2n, DevGraph& out, cudaStream_t s) {
  int n = g.n;
  out.n = n;
  out.nnz = g.nnz;
  out.rowptr.alloc(n + 1);
  out.col.alloc(g.nnz);
  out.w.alloc(g.nnz);
  DBuf<int> deg;
  deg.alloc(n);
  int nb = cdiv(n, kBlock);
  k_perm_degree<<<nb, kBlock, 0, s>>>(n, g.rowptr, n2o, deg);
  LL_LAUNCHED();
  exclusive_scan(deg, out.rowptr, n, s);
  k_perm_fill<<<nb, kBlock, 0, s>>>(n, g.rowptr, g.col, g.w, n2o, o2n, out.rowptr, out.col, out.w);
  LL_LAUNCHED();
  k_sort_segments<<<nb, kBlock, 0, s>>>(n, out.rowptr, out.col, out.w, nullptr);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
}

void invert_perm(int n, const int* n2o, int* o2n, cudaStream_t s) {
  k_invert_perm<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, n2o, o2n);
  LL_LAUNCHED();
}

// out[i] = m2[m1[i]] (or -1 where m1[i] < 0); m1 indexed through idx when given:
// out[i] = m2[m1[idx[i]]]
__global__ void k_map_through(int n, const int* __restrict__ idx, const int* __restrict__ m1,
                              const int* __restrict__ m2, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int j = idx ? idx[i] : i;
  int a = j < 0 ? -1 : m1[j];
  out[i] = a < 0 ? -1 : m2[a];
}
void map_through(int n, const int* idx, const int* m1, const int* m2, int* out, cudaStream_t s) {
  k_map_through<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, idx, m1, m2, out);
  LL_LAUNCHED();
}

}  // namespace llmg
