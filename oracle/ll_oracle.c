/*
 * ll_oracle.c -- plain, slow FP64 CPU oracle for the semi-implicit BDF1
 * Landau-Lifshitz linear solve by aggregation AMG + preconditioned GCR.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg do.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (each routine cites the passage it restates):
 *   - the operator of the damped semi-implicit scheme (Sec. 2.1, component
 *     form of (I + dt m^n x Delta_h + alpha dt m^n x (m^n x Delta_h)) m^{n+1}
 *     = m^n), divided through by dt, assembled as a scalar CSR matrix in the
 *     component-major unknown order [m1 (all cells); m2; m3] of Sec. 2.1;
 *   - pairwise-matching aggregation, two passes per level (Sec. 3.1), with the
 *     Boolean prolongation P of Eq. (Pagg) formed explicitly;
 *   - Galerkin coarse operators A_c = P^T A P (Eq. galerkin) by two explicit
 *     sparse matrix products;
 *   - block Gauss-Seidel smoothing (Sec. 3, "(symmetric) Gauss-Seidel"),
 *     V-cycle, dense LU at the coarsest level;
 *   - preconditioned GCR exactly as Algorithm 1 (modified Gram-Schmidt),
 *     with restarts;
 *   - the time step with projection m <- m/|m| (Sec. 4, projection step).
 *
 * Readings of points the paper leaves open are listed in the design notes of
 * the repository; the ones that change results are restated at each routine.
 */


#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small utilities                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nrows, ncols;
  int *rowptr; /* nrows+1 */
  int *col;    /* nnz, sorted ascending within each row */
  double *val; /* nnz */
} csr_t;

static void *xmalloc(size_t n) {
  void *p = malloc(n ? n : 1);
  if (!p) abort();
  return p;
}
static void *xcalloc(size_t n, size_t s) {
  void *p = calloc(n ? n : 1, s ? s : 1);
  if (!p) abort();
  return p;
}
static void csr_free(csr_t *a) {
  free(a->rowptr);
  free(a->col);
  free(a->val);
  memset(a, 0, sizeof(*a));
}

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* y = A x */
static void csr_matvec(const csr_t *a, const double *x, double *y) {
  for (int i = 0; i < a->nrows; ++i) {
    double s = 0.0;
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) s += a->val[p] * x[a->col[p]];
    y[i] = s;
  }
}

/* transpose of a CSR matrix (counting sort; keeps columns sorted) */
static csr_t csr_transpose(const csr_t *a) {
  csr_t t;
  int nnz = a->rowptr[a->nrows];
  t.nrows = a->ncols;
  t.ncols = a->nrows;
  t.rowptr = (int *)xcalloc((size_t)t.nrows + 1, sizeof(int));
  t.col = (int *)xmalloc((size_t)nnz * sizeof(int));
  t.val = (double *)xmalloc((size_t)nnz * sizeof(double));
  for (int p = 0; p < nnz; ++p) t.rowptr[a->col[p] + 1]++;
  for (int i = 0; i < t.nrows; ++i) t.rowptr[i + 1] += t.rowptr[i];
  int *next = (int *)xmalloc((size_t)t.nrows * sizeof(int));
  memcpy(next, t.rowptr, (size_t)t.nrows * sizeof(int));
  for (int i = 0; i < a->nrows; ++i)
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) {
      int q = next[a->col[p]]++;
      t.col[q] = i;
      t.val[q] = a->val[p];
    }
  free(next);
  return t;
}

/* C = A B, textbook row-by-row (Gustavson) product with a dense accumulator */
static csr_t csr_matmul(const csr_t *a, const csr_t *b) {
  csr_t c;
  c.nrows = a->nrows;
  c.ncols = b->ncols;
  c.rowptr = (int *)xcalloc((size_t)c.nrows + 1, sizeof(int));
  double *acc = (double *)xcalloc((size_t)b->ncols, sizeof(double));
  int *mark = (int *)xmalloc((size_t)b->ncols * sizeof(int));
  for (int j = 0; j < b->ncols; ++j) mark[j] = -1;
  int *cols = (int *)xmalloc((size_t)b->ncols * sizeof(int));
  size_t cap = (size_t)a->rowptr[a->nrows] + 16, nnz = 0;
  c.col = (int *)xmalloc(cap * sizeof(int));
  c.val = (double *)xmalloc(cap * sizeof(double));
  for (int i = 0; i < a->nrows; ++i) {
    int ncols = 0;
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) {
      int k = a->col[p];
      double av = a->val[p];
      for (int q = b->rowptr[k]; q < b->rowptr[k + 1]; ++q) {
        int j = b->col[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols[ncols++] = j;
        }
        acc[j] += av * b->val[q];
      }
    }
    qsort(cols, (size_t)ncols, sizeof(int), cmp_int);
    if (nnz + (size_t)ncols > cap) {
      while (nnz + (size_t)ncols > cap) cap *= 2;
      c.col = (int *)realloc(c.col, cap * sizeof(int));
      c.val = (double *)realloc(c.val, cap * sizeof(double));
      if (!c.col || !c.val) abort();
    }
    for (int t = 0; t < ncols; ++t) {
      c.col[nnz] = cols[t];
      c.val[nnz] = acc[cols[t]];
      ++nnz;
    }
    c.rowptr[i + 1] = (int)nnz;
  }
  free(acc);
  free(mark);
  free(cols);
  return c;
}

/* ------------------------------------------------------------------------ */
/* integer mixing (MurmurHash3 32-bit finaliser, a published function)        */
/* ------------------------------------------------------------------------ */

static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
/* tie-break key of the undirected edge {a,b}, a < b */
static uint32_t edge_hash(uint32_t a, uint32_t b, uint32_t seed) {
  return fmix32((a * 2654435761u) ^ b ^ seed);
}
/* colouring priority of vertex v */
static uint32_t vertex_hash(uint32_t v, uint32_t seed) {
  return fmix32((v * 2654435761u) ^ seed ^ 0x5bd1e995u);
}

/* ------------------------------------------------------------------------ */
/* grid and operator (Sec. 2.1)                                               */
/* ------------------------------------------------------------------------ */

/* Cell-centred grid, lexicographic cell index k = x + nx*(y + ny*z).  The
 * discrete Laplacian with homogeneous Neumann boundaries keeps only the face
 * neighbours that exist:  (Delta_h u)_k = sum_{l ~ k} (u_l - u_k) / h^2.
 * Returns the N x N scalar matrix L. */
static csr_t assemble_laplacian(int nx, int ny, int nz, double h) {
  int n = nx * ny * nz;
  csr_t L;
  L.nrows = L.ncols = n;
  L.rowptr = (int *)xcalloc((size_t)n + 1, sizeof(int));
  L.col = (int *)xmalloc((size_t)n * 7 * sizeof(int));
  L.val = (double *)xmalloc((size_t)n * 7 * sizeof(double));
  double ih2 = 1.0 / (h * h);
  int nnz = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int k = x + nx * (y + ny * z);
        int nb[6], deg = 0;
        if (z > 0) nb[deg++] = k - nx * ny;
        if (y > 0) nb[deg++] = k - nx;
        if (x > 0) nb[deg++] = k - 1;
        if (x < nx - 1) nb[deg++] = k + 1;
        if (y < ny - 1) nb[deg++] = k + nx;
        if (z < nz - 1) nb[deg++] = k + nx * ny;
        /* the neighbours above are in ascending order; the diagonal sits
         * between the lower and the upper ones */
        int placed = 0;
        for (int t = 0; t < deg; ++t) {
          if (!placed && nb[t] > k) {
            L.col[nnz] = k;
            L.val[nnz] = -deg * ih2;
            ++nnz;
            placed = 1;
          }
          L.col[nnz] = nb[t];
          L.val[nnz] = ih2;
          ++nnz;
        }
        if (!placed) {
          L.col[nnz] = k;
          L.val[nnz] = -deg * ih2;
          ++nnz;
        }
        L.rowptr[k + 1] = nnz;
      }
  return L;
}

/* The 3x3 coefficient that multiplies (Delta_h x)_k in row-block k:
 *   C(m) y = m x y + alpha m x (m x y) = [m]_x y + alpha (m m^T - |m|^2 I) y,
 * read off the component form of the damped scheme (Sec. 2.1): row 1 holds
 * +m2 Delta m3 - m3 Delta m2 and alpha[-(m2^2+m3^2) Delta m1 + m1 m2 Delta m2
 * + m1 m3 Delta m3], and cyclically.  All coefficients use m^n. */
static void coef_C(const double m[3], double alpha, double c[3][3]) {
  double m1 = m[0], m2 = m[1], m3 = m[2];
  /* cross-product part, [m]_x */
  double cx[3][3] = {{0.0, -m3, m2}, {m3, 0.0, -m1}, {-m2, m1, 0.0}};
  /* damping part, m x (m x .) = m m^T - |m|^2 I */
  double s = m1 * m1 + m2 * m2 + m3 * m3;
  double mm[3][3] = {{m1 * m1 - s, m1 * m2, m1 * m3},
                     {m2 * m1, m2 * m2 - s, m2 * m3},
                     {m3 * m1, m3 * m2, m3 * m3 - s}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[i][j] = cx[i][j] + alpha * mm[i][j];
}

/* Assemble A = I/dt + blockrows(C(m_k)) (L (x) I) in component-major order:
 *   A[(c,k),(c',l)] = delta_cc' delta_kl / dt + C(m_k)_{cc'} L_kl.
 * This is the paper's (I + dt m^n x Delta_h + alpha dt m^n x (m^n x Delta_h))
 * divided by dt, whose right-hand side is m^n/dt. */
static csr_t assemble_operator(int nx, int ny, int nz, double h, double alpha, double dt,
                               const double *m /* SoA, 3N */) {
  int n = nx * ny * nz;
  csr_t L = assemble_laplacian(nx, ny, nz, h);
  csr_t A;
  A.nrows = A.ncols = 3 * n;
  A.rowptr = (int *)xcalloc((size_t)3 * n + 1, sizeof(int));
  size_t cap = (size_t)3 * L.rowptr[n] * 3;
  A.col = (int *)xmalloc(cap * sizeof(int));
  A.val = (double *)xmalloc(cap * sizeof(double));
  int nnz = 0;
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < n; ++k) {
      double mk[3] = {m[k], m[n + k], m[2 * n + k]}, C[3][3];
      coef_C(mk, alpha, C);
      for (int c2 = 0; c2 < 3; ++c2)
        for (int p = L.rowptr[k]; p < L.rowptr[k + 1]; ++p) {
          int l = L.col[p];
          double v = C[c][c2] * L.val[p];
          if (c2 == c && l == k) v += 1.0 / dt;
          A.col[nnz] = c2 * n + l;
          A.val[nnz] = v;
          ++nnz;
        }
      A.rowptr[c * n + k + 1] = nnz;
    }
  csr_free(&L);
  return A;
}

/* ------------------------------------------------------------------------ */
/* aggregation (Sec. 3.1.1): two passes of pairwise matching per level        */
/* ------------------------------------------------------------------------ */

/* Weighted undirected graph without self loops (integer weights). */
typedef struct {
  int n;
  int *rowptr, *col, *w;
} graph_t;

static void graph_free(graph_t *g) {
  free(g->rowptr);
  free(g->col);
  free(g->w);
  memset(g, 0, sizeof(*g));
}

/* level-0 graph: face neighbours of the grid, weight 1 each */
static graph_t grid_graph(int nx, int ny, int nz) {
  int n = nx * ny * nz;
  graph_t g;
  g.n = n;
  g.rowptr = (int *)xcalloc((size_t)n + 1, sizeof(int));
  g.col = (int *)xmalloc((size_t)n * 6 * sizeof(int));
  g.w = (int *)xmalloc((size_t)n * 6 * sizeof(int));
  int e = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int k = x + nx * (y + ny * z);
        if (z > 0) g.col[e] = k - nx * ny, g.w[e++] = 1;
        if (y > 0) g.col[e] = k - nx, g.w[e++] = 1;
        if (x > 0) g.col[e] = k - 1, g.w[e++] = 1;
        if (x < nx - 1) g.col[e] = k + 1, g.w[e++] = 1;
        if (y < ny - 1) g.col[e] = k + nx, g.w[e++] = 1;
        if (z < nz - 1) g.col[e] = k + nx * ny, g.w[e++] = 1;
        g.rowptr[k + 1] = e;
      }
  return g;
}

/* Contract a graph by a map fine -> coarse: the weight between coarse nodes
 * I != J is the sum of the weights of the fine edges joining them (the
 * integer Galerkin product of the weight graph); edges inside an aggregate
 * disappear. */
static graph_t graph_contract(const graph_t *g, const int *map, int nc) {
  /* members of each coarse node, in ascending fine order */
  int *mptr = (int *)xcalloc((size_t)nc + 1, sizeof(int));
  int *mem = (int *)xmalloc((size_t)g->n * sizeof(int));
  for (int i = 0; i < g->n; ++i) mptr[map[i] + 1]++;
  for (int I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
  int *next = (int *)xmalloc((size_t)nc * sizeof(int));
  memcpy(next, mptr, (size_t)nc * sizeof(int));
  for (int i = 0; i < g->n; ++i) mem[next[map[i]]++] = i;
  free(next);

  graph_t c;
  c.n = nc;
  c.rowptr = (int *)xcalloc((size_t)nc + 1, sizeof(int));
  size_t cap = (size_t)g->rowptr[g->n] + 16, e = 0;
  c.col = (int *)xmalloc(cap * sizeof(int));
  c.w = (int *)xmalloc(cap * sizeof(int));
  int *acc = (int *)xcalloc((size_t)nc, sizeof(int));
  int *mark = (int *)xmalloc((size_t)nc * sizeof(int));
  for (int J = 0; J < nc; ++J) mark[J] = -1;
  int *cols = (int *)xmalloc((size_t)nc * sizeof(int));
  for (int I = 0; I < nc; ++I) {
    int ncol = 0;
    for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
      int i = mem[t];
      for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p) {
        int J = map[g->col[p]];
        if (J == I) continue;
        if (mark[J] != I) {
          mark[J] = I;
          acc[J] = 0;
          cols[ncol++] = J;
        }
        acc[J] += g->w[p];
      }
    }
    qsort(cols, (size_t)ncol, sizeof(int), cmp_int);
    for (int t = 0; t < ncol; ++t) {
      c.col[e] = cols[t];
      c.w[e] = acc[cols[t]];
      ++e;
    }
    c.rowptr[I + 1] = (int)e;
  }
  free(acc);
  free(mark);
  free(cols);
  free(mptr);
  free(mem);
  return c;
}

/* Does edge (a-b, weight wa, hash ha) beat edge (c-d, weight wc, hash hc)?
 * Edges are totally ordered by (weight, hash, -min endpoint, -max endpoint). */
static int edge_beats(int wa, uint32_t ha, int a0, int a1, int wb, uint32_t hb, int b0, int b1) {
  if (wa != wb) return wa > wb;
  if (ha != hb) return ha > hb;
  if (a0 != b0) return a0 < b0;
  return a1 < b1;
}

/* One pass of pairwise matching on graph g (Sec. 3.1.1: each level runs two
 * matching passes that prefer the strongest couplings).
 * Reading: an edge {i,j} is a candidate when it is strong for either end,
 * 4 w_ij >= max_l w_il or 4 w_ij >= max_l w_jl (threshold 1/4 of the
 * strongest coupling); rounds of handshake matching -- every unmatched node
 * points at its best unmatched candidate neighbour and mutual pointers
 * become pairs -- are repeated until a round forms no pair or `rounds`
 * rounds have run.  Leftover nodes stay singletons, unless `attach` is set:
 * then each leftover whose best neighbour (same edge order, over all
 * neighbours) is matched joins that neighbour's pair.  Groups are numbered
 * by the rank of their smallest member.  Returns the number of groups;
 * group[i] receives the group of node i. */
static int matching_pass(const graph_t *g, int rounds, uint32_t seed, int attach, int *group) {
  int n = g->n;
  int *maxw = (int *)xcalloc((size_t)n, sizeof(int));
  int *mate = (int *)xmalloc((size_t)n * sizeof(int));
  int *best = (int *)xmalloc((size_t)n * sizeof(int));
  int *newmate = (int *)xmalloc((size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) {
    mate[i] = -1;
    for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p)
      if (g->w[p] > maxw[i]) maxw[i] = g->w[p];
  }
  for (int r = 0; r < rounds; ++r) {
    /* every unmatched node picks its best unmatched strong neighbour,
     * looking only at the state at the start of the round */
    for (int i = 0; i < n; ++i) {
      best[i] = -1;
      if (mate[i] >= 0) continue;
      int bw = 0, b0 = 0, b1 = 0;
      uint32_t bh = 0;
      for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p) {
        int j = g->col[p], w = g->w[p];
        if (mate[j] >= 0) continue;
        /* strong in the view of either end (a symmetric candidate set, so
         * the largest remaining candidate edge is always a mutual choice) */
        if (4 * w < maxw[i] && 4 * w < maxw[j]) continue;
        int e0 = i < j ? i : j, e1 = i < j ? j : i;
        uint32_t eh = edge_hash((uint32_t)e0, (uint32_t)e1, seed);
        if (best[i] < 0 || edge_beats(w, eh, e0, e1, bw, bh, b0, b1)) {
          best[i] = j;
          bw = w;
          bh = eh;
          b0 = e0;
          b1 = e1;
        }
      }
    }
    /* mutual choices become pairs */
    int formed = 0;
    for (int i = 0; i < n; ++i) {
      newmate[i] = mate[i];
      if (mate[i] < 0 && best[i] >= 0 && best[best[i]] == i) {
        newmate[i] = best[i];
        formed = 1;
      }
    }
    memcpy(mate, newmate, (size_t)n * sizeof(int));
    if (!formed) break;
  }
  /* a node left unmatched joins the pair of its best neighbour, when that
   * neighbour is matched (keeps isolated leftovers from piling up as
   * singletons on coarse levels); its pair is represented by the smaller of
   * the two matched nodes */
  int *rep = (int *)xmalloc((size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) rep[i] = (mate[i] >= 0 && mate[i] < i) ? mate[i] : i;
  if (attach) {
    for (int i = 0; i < n; ++i) {
      if (mate[i] >= 0) continue;
      int bj = -1, bw = 0, b0 = 0, b1 = 0;
      uint32_t bh = 0;
      for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p) {
        int j = g->col[p], w = g->w[p];
        int e0 = i < j ? i : j, e1 = i < j ? j : i;
        uint32_t eh = edge_hash((uint32_t)e0, (uint32_t)e1, seed);
        if (bj < 0 || edge_beats(w, eh, e0, e1, bw, bh, b0, b1)) {
          bj = j;
          bw = w;
          bh = eh;
          b0 = e0;
          b1 = e1;
        }
      }
      if (bj >= 0 && mate[bj] >= 0) rep[i] = (mate[bj] < bj) ? mate[bj] : bj;
    }
  }
  /* number the groups by the rank of their smallest member */
  int *minmem = (int *)xmalloc((size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) minmem[i] = n;
  for (int i = 0; i < n; ++i)
    if (i < minmem[rep[i]]) minmem[rep[i]] = i;
  int ng = 0;
  int *gid = (int *)xmalloc((size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i)
    if (minmem[rep[i]] == i) gid[rep[i]] = ng++;
  for (int i = 0; i < n; ++i) group[i] = gid[rep[i]];
  free(gid);
  free(minmem);
  free(rep);
  free(maxw);
  free(mate);
  free(best);
  free(newmate);
  return ng;
}

/* One coarsening level: pass 1 on g (pairs and singletons), pass 2 on the
 * contracted pair graph with leftovers attached to a neighbouring pair,
 * composed, then numbered by the rank of each aggregate's smallest fine
 * member.  Aggregates hold about four nodes, the coarsening factor of a
 * little under four that Sec. 3.1.1 describes.  Returns the number of
 * aggregates. */
static int aggregate_level(const graph_t *g, int rounds, uint32_t seed, int *agg) {
  int n = g->n;
  int *g1 = (int *)xmalloc((size_t)n * sizeof(int));
  int n1 = matching_pass(g, rounds, seed, 0, g1);
  graph_t gg = graph_contract(g, g1, n1);
  int *g2 = (int *)xmalloc((size_t)(n1 > 0 ? n1 : 1) * sizeof(int));
  int n2 = matching_pass(&gg, rounds, seed, 1, g2);
  graph_free(&gg);
  int *minmem = (int *)xmalloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(int));
  for (int a = 0; a < n2; ++a) minmem[a] = n;
  for (int i = 0; i < n; ++i) {
    int a = g2[g1[i]];
    if (i < minmem[a]) minmem[a] = i;
  }
  int *rank = (int *)xmalloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(int));
  int nc = 0;
  for (int i = 0; i < n; ++i) {
    int a = g2[g1[i]];
    if (minmem[a] == i) rank[a] = nc++;
  }
  for (int i = 0; i < n; ++i) agg[i] = rank[g2[g1[i]]];
  free(g1);
  free(g2);
  free(minmem);
  free(rank);
  return nc;
}

/* Boolean prolongation of Eq. (Pagg) for the scalar unknowns, in the
 * component-major order at both levels: P[(c,i),(c,agg(i))] = 1. */
static csr_t prolongation(int n, int nc, const int *agg) {
  csr_t P;
  P.nrows = 3 * n;
  P.ncols = 3 * nc;
  P.rowptr = (int *)xmalloc(((size_t)3 * n + 1) * sizeof(int));
  P.col = (int *)xmalloc((size_t)3 * n * sizeof(int));
  P.val = (double *)xmalloc((size_t)3 * n * sizeof(double));
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < n; ++i) {
      int r = c * n + i;
      P.rowptr[r] = r;
      P.col[r] = c * nc + agg[i];
      P.val[r] = 1.0;
    }
  P.rowptr[3 * n] = 3 * n;
  return P;
}

/* ------------------------------------------------------------------------ */
/* colouring for the Gauss-Seidel smoother                                    */
/* ------------------------------------------------------------------------ */

/* Reading: on the grid the two colours are the parity of x+y+z (the 5/7-point
 * cell graph is bipartite).  On aggregated levels (the paper fixes no order
 * of the Gauss-Seidel unknowns, Sec. 3) a colouring in two stages:
 *  1. Jones-Plassmann rounds: every uncoloured node whose priority beats all
 *     its uncoloured neighbours takes the smallest colour unused by its
 *     neighbours (those nodes form an independent set).  Priority: the larger
 *     degree (number of neighbours), then the larger vertex_hash, then the
 *     larger index.
 *  2. kRecolourPasses passes of iterated greedy recolouring: the classes of
 *     the current colouring are visited from the highest colour to the
 *     lowest, and each node takes the smallest colour unused by the
 *     neighbours already visited in this pass.  Nodes of one class are not
 *     adjacent, so the order inside a class does not matter, and a pass never
 *     needs more colours than the colouring it starts from. */
enum { kRecolourPasses = 4 };

static int node_beats(const graph_t *g, int j, int i, uint32_t seed) {
  int dj = g->rowptr[j + 1] - g->rowptr[j], di = g->rowptr[i + 1] - g->rowptr[i];
  if (dj != di) return dj > di;
  uint32_t hj = vertex_hash((uint32_t)j, seed), hi = vertex_hash((uint32_t)i, seed);
  if (hj != hi) return hj > hi;
  return j > i;
}

/* smallest colour not taken by a neighbour of i (colours < 0 are free) */
static int first_free(const graph_t *g, int i, const int *c, char *used, int maxdeg) {
  memset(used, 0, (size_t)maxdeg + 2);
  for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p) {
    int cj = c[g->col[p]];
    if (cj >= 0 && cj <= maxdeg) used[cj] = 1;
  }
  int k = 0;
  while (used[k]) ++k;
  return k;
}

static int colour_graph(const graph_t *g, uint32_t seed, int *colour) {
  int n = g->n, ncol = 0;
  int *snap = (int *)xmalloc((size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i) colour[i] = -1;
  int left = n;
  int maxdeg = 0;
  for (int i = 0; i < n; ++i)
    if (g->rowptr[i + 1] - g->rowptr[i] > maxdeg) maxdeg = g->rowptr[i + 1] - g->rowptr[i];
  char *used = (char *)xcalloc((size_t)maxdeg + 2, 1);
  while (left > 0) { /* stage 1 */
    memcpy(snap, colour, (size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) {
      if (snap[i] >= 0) continue;
      int wins = 1;
      for (int p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p) {
        int j = g->col[p];
        if (snap[j] < 0 && node_beats(g, j, i, seed)) {
          wins = 0;
          break;
        }
      }
      if (!wins) continue;
      colour[i] = first_free(g, i, snap, used, maxdeg);
      if (colour[i] + 1 > ncol) ncol = colour[i] + 1;
      --left;
    }
  }
  for (int pass = 0; pass < kRecolourPasses; ++pass) { /* stage 2 */
    for (int i = 0; i < n; ++i) snap[i] = -1;
    int nnew = 0;
    for (int c = ncol - 1; c >= 0; --c)
      for (int i = 0; i < n; ++i) {
        if (colour[i] != c) continue;
        snap[i] = first_free(g, i, snap, used, maxdeg);
        if (snap[i] + 1 > nnew) nnew = snap[i] + 1;
      }
    memcpy(colour, snap, (size_t)n * sizeof(int));
    ncol = nnew;
  }
  free(snap);
  free(used);
  return ncol;
}

/* ------------------------------------------------------------------------ */
/* dense LU with partial pivoting (coarsest level "exact solution")          */
/* ------------------------------------------------------------------------ */

/* Factor the n x n row-major matrix a in place; piv[k] = row swapped into k.
 * Ties in pivot magnitude go to the lowest row.  Returns 0, or 1 if a pivot
 * is zero. */
static int lu_factor(int n, double *a, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + k]) > best) {
        best = fabs(a[(size_t)i * n + k]);
        p = i;
      }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

static void lu_solve(int n, const double *a, const int *piv, double *x) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) {
      double t = x[k];
      x[k] = x[piv[k]];
      x[piv[k]] = t;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
    x[i] /= a[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------------------ */
/* hierarchy                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rtol;
  int maxit, restart, nu_pre, nu_post, coarsest_cells, max_levels, rounds;
  uint32_t seed;
  int prec; /* 0 = V-cycle, 1 = none (plain GCR), 2 = exact dense LU of A */
  int kcycle; /* levels 1..kcycle (not the coarsest) are solved by two inner GCR steps */
  /* stagnation stop (not in the paper; a safeguard, 0 = off): at a restart,
   * stop as not converged when the true residual norm exceeds stall_ratio
   * times its value at the latest restart at least stall_window iterations
   * earlier */
  int stall_window;
  double stall_ratio;
} orc_params;

typedef struct {
  int n;       /* cells on this level */
  csr_t A;     /* 3n x 3n scalar operator, component-major */
  int *agg;    /* n -> n_{l+1} (NULL on the coarsest level) */
  csr_t P, Pt; /* explicit prolongation and its transpose */
  int ncolours;
  int *colour; /* n */
  graph_t g;   /* weight graph of this level */
} level_t;

typedef struct {
  int nx, ny, nz;
  double h, alpha, dt;
  orc_params prm;
  int nlev;
  level_t lev[64];
  double *lu; /* coarsest dense LU factors (3 n_L)^2 */
  int *piv;
  int singular;
  double *exact_lu; /* prec == 2: LU of the whole fine operator */
  int *exact_piv;
} orc_hier;

void orc_free(orc_hier *H) {
  if (!H) return;
  for (int l = 0; l < H->nlev; ++l) {
    csr_free(&H->lev[l].A);
    csr_free(&H->lev[l].P);
    csr_free(&H->lev[l].Pt);
    free(H->lev[l].agg);
    free(H->lev[l].colour);
    graph_free(&H->lev[l].g);
  }
  free(H->lu);
  free(H->piv);
  free(H->exact_lu);
  free(H->exact_piv);
  free(H);
}

static double *csr_to_dense(const csr_t *a) {
  double *d = (double *)xcalloc((size_t)a->nrows * a->ncols, sizeof(double));
  for (int i = 0; i < a->nrows; ++i)
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) d[(size_t)i * a->ncols + a->col[p]] += a->val[p];
  return d;
}

/* Build the whole hierarchy for one time step. */
orc_hier *orc_setup(int nx, int ny, int nz, double h, double alpha, double dt, const double *m,
                    const orc_params *prm) {
  orc_hier *H = (orc_hier *)xcalloc(1, sizeof(orc_hier));
  H->nx = nx;
  H->ny = ny;
  H->nz = nz;
  H->h = h;
  H->alpha = alpha;
  H->dt = dt;
  H->prm = *prm;
  int n = nx * ny * nz;
  level_t *L0 = &H->lev[0];
  L0->n = n;
  L0->A = assemble_operator(nx, ny, nz, h, alpha, dt, m);
  L0->g = grid_graph(nx, ny, nz);
  L0->colour = (int *)xmalloc((size_t)n * sizeof(int));
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) L0->colour[x + nx * (y + ny * z)] = (x + y + z) & 1;
  L0->ncolours = n > 1 ? 2 : 1;
  H->nlev = 1;
  int maxlev = prm->max_levels < 64 ? prm->max_levels : 64;
  while (H->lev[H->nlev - 1].n > prm->coarsest_cells && H->nlev < maxlev) {
    level_t *F = &H->lev[H->nlev - 1];
    int *agg = (int *)xmalloc((size_t)F->n * sizeof(int));
    int nc = aggregate_level(&F->g, prm->rounds, prm->seed, agg);
    if (3 * (long)nc > 2 * (long)F->n) { /* coarsening ratio below 1.5: stop */
      free(agg);
      break;
    }
    F->agg = agg;
    F->P = prolongation(F->n, nc, agg);
    F->Pt = csr_transpose(&F->P);
    level_t *C = &H->lev[H->nlev];
    C->n = nc;
    /* Galerkin product A_c = P^T (A P), Eq. (galerkin) */
    csr_t AP = csr_matmul(&F->A, &F->P);
    C->A = csr_matmul(&F->Pt, &AP);
    csr_free(&AP);
    C->g = graph_contract(&F->g, agg, nc);
    C->colour = (int *)xmalloc((size_t)nc * sizeof(int));
    C->ncolours = colour_graph(&C->g, prm->seed, C->colour);
    H->nlev++;
  }
  level_t *Lc = &H->lev[H->nlev - 1];
  int nn = 3 * Lc->n;
  H->lu = csr_to_dense(&Lc->A);
  H->piv = (int *)xmalloc((size_t)nn * sizeof(int));
  H->singular = lu_factor(nn, H->lu, H->piv);
  if (prm->prec == 2) {
    H->exact_lu = csr_to_dense(&L0->A);
    H->exact_piv = (int *)xmalloc((size_t)3 * n * sizeof(int));
    lu_factor(3 * n, H->exact_lu, H->exact_piv);
  }
  return H;
}

/* ------------------------------------------------------------------------ */
/* smoother, V-cycle                                                          */
/* ------------------------------------------------------------------------ */

/* Solve the 3x3 system d y = s by Gaussian elimination with partial
 * pivoting (d is overwritten). */
static void solve3(double d[3][3], double s[3], double y[3]) {
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(d[i][k]) > fabs(d[p][k])) p = i;
    if (p != k) {
      for (int j = 0; j < 3; ++j) {
        double t = d[k][j];
        d[k][j] = d[p][j];
        d[p][j] = t;
      }
      double t = s[k];
      s[k] = s[p];
      s[p] = t;
    }
    for (int i = k + 1; i < 3; ++i) {
      double l = d[i][k] / d[k][k];
      for (int j = k; j < 3; ++j) d[i][j] -= l * d[k][j];
      s[i] -= l * s[k];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double t = s[i];
    for (int j = i + 1; j < 3; ++j) t -= d[i][j] * y[j];
    y[i] = t / d[i][i];
  }
}

/* One block Gauss-Seidel sweep on level l: the cells of each colour in turn
 * (ascending colours when forward != 0, descending otherwise); each cell's
 * three unknowns are updated together by solving with the 3x3 diagonal block
 * against the residual of the other unknowns. */
static void gs_sweep(const level_t *L, const double *b, double *x, int forward) {
  int n = L->n;
  for (int t = 0; t < L->ncolours; ++t) {
    int col = forward ? t : L->ncolours - 1 - t;
    for (int k = 0; k < n; ++k) {
      if (L->colour[k] != col) continue;
      double d[3][3] = {{0}}, s[3], y[3];
      for (int c = 0; c < 3; ++c) {
        int r = c * n + k;
        s[c] = b[r];
        for (int p = L->A.rowptr[r]; p < L->A.rowptr[r + 1]; ++p) {
          int j = L->A.col[p];
          if (j % n == k) d[c][j / n] += L->A.val[p];
          else s[c] -= L->A.val[p] * x[j];
        }
      }
      solve3(d, s, y);
      for (int c = 0; c < 3; ++c) x[c * n + k] = y[c];
    }
  }
}

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void vcycle(const orc_hier *H, int l, const double *b, double *x);

/* K-cycle coarse solve (the Krylov acceleration of each level that Sec. 3.1
 * describes for AGMG): two steps of preconditioned GCR (Algorithm 1 with
 * modified Gram-Schmidt) on A_l e = r from e = 0, the cycle of level l as
 * the preconditioner. */
static void kinner(const orc_hier *H, int l, const double *r, double *e) {
  const csr_t *A = &H->lev[l].A;
  int nn = A->nrows;
  double *z1 = (double *)xmalloc((size_t)nn * sizeof(double));
  double *z2 = (double *)xmalloc((size_t)nn * sizeof(double));
  double *c1 = (double *)xmalloc((size_t)nn * sizeof(double));
  double *c2 = (double *)xmalloc((size_t)nn * sizeof(double));
  double *r1 = (double *)xmalloc((size_t)nn * sizeof(double));
  vcycle(H, l, r, z1);
  csr_matvec(A, z1, c1);
  double g11 = sqrt(dot(nn, c1, c1));
  /* A direction whose image A z vanishes (only z = 0 for a regular A)
   * contributes nothing and is dropped instead of normalised. */
  for (int i = 0; i < nn; ++i) c1[i] = g11 > 0 ? c1[i] / g11 : 0.0;
  double a1 = dot(nn, c1, r);
  for (int i = 0; i < nn; ++i) r1[i] = r[i] - a1 * c1[i];
  vcycle(H, l, r1, z2);
  csr_matvec(A, z2, c2);
  double g12 = dot(nn, c1, c2);
  for (int i = 0; i < nn; ++i) c2[i] -= g12 * c1[i];
  double g22 = sqrt(dot(nn, c2, c2));
  for (int i = 0; i < nn; ++i) c2[i] = g22 > 0 ? c2[i] / g22 : 0.0;
  double a2 = dot(nn, c2, r1);
  double y2 = g22 > 0 ? a2 / g22 : 0.0, y1 = g11 > 0 ? (a1 - g12 * y2) / g11 : 0.0;
  for (int i = 0; i < nn; ++i) e[i] = y1 * z1[i] + y2 * z2[i];
  free(z1);
  free(z2);
  free(c1);
  free(c2);
  free(r1);
}

/* V-cycle on level l for A_l x = b, starting from x = 0 (Sec. 3: smoother
 * plus coarse-grid correction, applied recursively down to an exact solve).
 * With prm.kcycle > 0 the coarse problem of levels 1..kcycle is solved by
 * kinner instead (a K-cycle). */
static void vcycle(const orc_hier *H, int l, const double *b, double *x) {
  const level_t *L = &H->lev[l];
  int nn = 3 * L->n;
  if (l == H->nlev - 1) {
    memcpy(x, b, (size_t)nn * sizeof(double));
    lu_solve(nn, H->lu, H->piv, x);
    return;
  }
  memset(x, 0, (size_t)nn * sizeof(double));
  for (int s = 0; s < H->prm.nu_pre; ++s) gs_sweep(L, b, x, 1);
  double *r = (double *)xmalloc((size_t)nn * sizeof(double));
  csr_matvec(&L->A, x, r);
  for (int i = 0; i < nn; ++i) r[i] = b[i] - r[i];
  int nc = 3 * H->lev[l + 1].n;
  double *bc = (double *)xmalloc((size_t)nc * sizeof(double));
  double *xc = (double *)xmalloc((size_t)nc * sizeof(double));
  csr_matvec(&L->Pt, r, bc); /* restriction = P^T */
  if (l + 1 < H->nlev - 1 && l + 1 <= H->prm.kcycle) kinner(H, l + 1, bc, xc);
  else vcycle(H, l + 1, bc, xc);
  csr_matvec(&L->P, xc, r); /* prolongation */
  for (int i = 0; i < nn; ++i) x[i] += r[i];
  for (int s = 0; s < H->prm.nu_post; ++s) gs_sweep(L, b, x, 0);
  free(r);
  free(bc);
  free(xc);
}

static void precondition(const orc_hier *H, const double *r, double *z) {
  int nn = 3 * H->lev[0].n;
  if (H->prm.prec == 1) {
    memcpy(z, r, (size_t)nn * sizeof(double));
  } else if (H->prm.prec == 2) {
    memcpy(z, r, (size_t)nn * sizeof(double));
    lu_solve(nn, H->exact_lu, H->exact_piv, z);
  } else {
    vcycle(H, 0, r, z);
  }
}

/* ------------------------------------------------------------------------ */
/* preconditioned GCR, Algorithm 1                                            */
/* ------------------------------------------------------------------------ */


/* Status codes shared in meaning with the library's header. */
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_BREAKDOWN = 2 };

/* Solve A u = b from the initial guess in x (overwritten by the solution).
 * Algorithm 1 with restarts of length prm.restart: the residual recurrence
 * r_j = r_{j-1} - alpha_j c_j drives the stopping test ||r_j|| < rtol ||b||,
 * and the solution u = u_0 + Z (Gamma^{-1} a) is formed after the loop.
 * Reading of the printed update u_m = Z Gamma^{-1} a: it omits u_0, exact
 * only for u_0 = 0, so u_0 is added.  After each cycle the true residual
 * b - A u decides convergence; another cycle runs if it fails.
 * history (optional, length maxit+1) gets the recurrence residual norms.
 * Returns a status; *iters = preconditioner applications, *relres = true
 * ||b - A u|| / ||b||. */
int orc_solve(const orc_hier *H, const double *b, double *x, double rtol, int *iters, double *relres,
              double *history) {
  const csr_t *A = &H->lev[0].A;
  int nn = A->nrows, total = 0, status = ORC_NOT_CONVERGED;
  int mmax = H->prm.restart;
  double nb = sqrt(dot(nn, b, b));
  double *r = (double *)xmalloc((size_t)nn * sizeof(double));
  double *Z = (double *)xmalloc((size_t)nn * mmax * sizeof(double));
  double *C = (double *)xmalloc((size_t)nn * mmax * sizeof(double));
  double *gam = (double *)xcalloc((size_t)mmax * mmax, sizeof(double));
  double *a = (double *)xcalloc((size_t)mmax, sizeof(double));
  double *y = (double *)xcalloc((size_t)mmax, sizeof(double));
  /* true residual norms at the restarts so far, for the stagnation stop */
  int nbound = 0;
  int *bound_it = (int *)xmalloc((size_t)(H->prm.maxit + 2) * sizeof(int));
  double *bound_nr = (double *)xmalloc((size_t)(H->prm.maxit + 2) * sizeof(double));
  if (nb == 0.0) {
    memset(x, 0, (size_t)nn * sizeof(double));
    *iters = 0;
    *relres = 0.0;
    status = ORC_OK;
    goto done;
  }
  for (;;) {
    /* r_0 = b - A u_0 (true residual) */
    csr_matvec(A, x, r);
    for (int i = 0; i < nn; ++i) r[i] = b[i] - r[i];
    double nr = sqrt(dot(nn, r, r));
    if (history && total == 0) history[0] = nr / nb;
    if (!(nr == nr)) {
      status = ORC_BREAKDOWN;
      break;
    }
    if (nr < rtol * nb) {
      status = ORC_OK;
      break;
    }
    if (total >= H->prm.maxit) break;
    if (H->prm.stall_window > 0) {
      int k = nbound - 1;
      while (k >= 0 && bound_it[k] > total - H->prm.stall_window) --k;
      if (k >= 0 && nr > H->prm.stall_ratio * bound_nr[k]) break; /* stagnated: not converged */
    }
    bound_it[nbound] = total;
    bound_nr[nbound++] = nr;
    int m = mmax;
    if (m > H->prm.maxit - total) m = H->prm.maxit - total;
    int done_j = 0, broke = 0;
    for (int j = 0; j < m; ++j) {
      double *zj = Z + (size_t)j * nn, *cj = C + (size_t)j * nn;
      precondition(H, r, zj);              /* step 1 */
      csr_matvec(A, zj, cj);               /* step 2 */
      for (int i = 0; i < j; ++i) {        /* step 3: modified Gram-Schmidt */
        const double *ci = C + (size_t)i * nn;
        double g = dot(nn, ci, cj);        /* (a) */
        gam[(size_t)i * mmax + j] = g;
        for (int t = 0; t < nn; ++t) cj[t] -= g * ci[t]; /* (b) */
      }
      double gjj = sqrt(dot(nn, cj, cj));  /* step 4 */
      gam[(size_t)j * mmax + j] = gjj;
      ++total;
      if (!(gjj > 0.0) || !(gjj < INFINITY)) {
        broke = 1;
        break;
      }
      for (int t = 0; t < nn; ++t) cj[t] /= gjj;
      a[j] = dot(nn, cj, r);               /* step 5 */
      for (int t = 0; t < nn; ++t) r[t] -= a[j] * cj[t];
      done_j = j + 1;
      double nrj = sqrt(dot(nn, r, r));
      if (history) history[total] = nrj / nb;
      if (nrj < rtol * nb) break;          /* step 6 */
    }
    /* u = u_0 + Z (Gamma^{-1} a), back substitution on the upper triangle */
    for (int i = done_j - 1; i >= 0; --i) {
      double s = a[i];
      for (int k = i + 1; k < done_j; ++k) s -= gam[(size_t)i * mmax + k] * y[k];
      y[i] = s / gam[(size_t)i * mmax + i];
    }
    for (int k = 0; k < done_j; ++k) {
      const double *zk = Z + (size_t)k * nn;
      for (int t = 0; t < nn; ++t) x[t] += y[k] * zk[t];
    }
    if (broke) {
      status = ORC_BREAKDOWN;
      break;
    }
  }
  *iters = total;
  csr_matvec(A, x, r);
  for (int i = 0; i < nn; ++i) r[i] = b[i] - r[i];
  *relres = sqrt(dot(nn, r, r)) / nb;
done:
  free(bound_it);
  free(bound_nr);
  free(r);
  free(Z);
  free(C);
  free(gam);
  free(a);
  free(y);
  return status;
}

/* ------------------------------------------------------------------------ */
/* time stepping with projection                                             */
/* ------------------------------------------------------------------------ */

/* The initial approximation u_0 of each step's solve (Algorithm 1 takes it
 * as an input; the paper does not fix it for the time loop).  Reading: the
 * states m^n, m^{n-1}, ... extrapolated one step ahead with the terms of
 * Newton's backward-difference series m^n + D m^n + D^2 m^n + ... that keep
 * shrinking, D^j m^n being the j-th backward difference over the d earlier
 * states this call has (d <= ORC_STEP_HIST): D m^n whenever d >= 1, then
 * D^j m^n for j = 2, 3, ... while |D^j m^n| < |D^{j-1} m^n| (Euclidean
 * norms over all components; the squares are compared).  With the terms up
 * to D^k the sum is the polynomial extrapolation of degree k through
 * m^n ... m^{n-k}: sum_{l=0..k} (-1)^l C(k+1, l+1) m^{n-l}, O(dt^{k+1}) from
 * the new solution while the series converges.  prev[j] holds m^{n-1-j}. */
#define ORC_STEP_HIST 6

static int step_order(int n3, int d, const double *m, double *const *prev) {
  if (d == 0) return 0;
  double s2[ORC_STEP_HIST + 1] = {0};
  for (int i = 0; i < n3; ++i) {
    double t[ORC_STEP_HIST + 1];
    t[0] = m[i];
    for (int l = 1; l <= d; ++l) t[l] = prev[l - 1][i];
    for (int j = 1; j <= d; ++j) {  /* t[0] becomes D^j m^n */
      for (int l = 0; l + j <= d; ++l) t[l] = t[l] - t[l + 1];
      s2[j] += t[0] * t[0];
    }
  }
  int k = 1;
  for (int j = 2; j <= d && s2[j] < s2[j - 1]; ++j) k = j;
  return k;
}

static void step_guess(int n3, int d, const double *m, double *const *prev, double *x) {
  int k = step_order(n3, d, m, prev);
  double c[ORC_STEP_HIST + 1];
  for (int l = 0; l <= k; ++l) { /* (-1)^l C(k+1, l+1) */
    double b = 1.0;
    for (int q = 0; q <= l; ++q) b = b * (double)(k + 1 - q) / (double)(q + 1);
    c[l] = (l % 2 ? -1.0 : 1.0) * b;
  }
  for (int i = 0; i < n3; ++i) {
    double v = c[0] * m[i];
    for (int l = 1; l <= k; ++l) v += c[l] * prev[l - 1][i];
    x[i] = v;
  }
}

/* the initial approximation alone, for the tests: prev holds d states of n3
 * values each, newest first; returns the order k it used */
int orc_step_guess(int n3, int d, const double *m, const double *prev, double *x) {
  double *p[ORC_STEP_HIST];
  if (d < 0 || d > ORC_STEP_HIST) return -1;
  for (int j = 0; j < d; ++j) p[j] = (double *)prev + (size_t)j * n3;
  step_guess(n3, d, m, p, x);
  return step_order(n3, d, m, p);
}

/* push m^n onto the history (prev[0] newest); returns the new depth */
static int step_push(int n3, int d, const double *m, double **prev) {
  double *t = prev[ORC_STEP_HIST - 1];
  for (int j = ORC_STEP_HIST - 1; j > 0; --j) prev[j] = prev[j - 1];
  prev[0] = t;
  memcpy(prev[0], m, (size_t)n3 * sizeof(double));
  return d < ORC_STEP_HIST ? d + 1 : ORC_STEP_HIST;
}

/* n_steps steps of the semi-implicit scheme: m~ = m^n, b = m^n/dt, solve
 * from the guess of step_guess, then m^{n+1} = x/|x| per cell when
 * project != 0. */
int orc_step(double *m, int n_steps, int nx, int ny, int nz, double h, double alpha, double dt,
             const orc_params *prm, int project, int *iters_per_step, double *relres_per_step) {
  int n = nx * ny * nz, worst = ORC_OK;
  double *b = (double *)xmalloc((size_t)3 * n * sizeof(double));
  double *x = (double *)xmalloc((size_t)3 * n * sizeof(double));
  double *prev[ORC_STEP_HIST];
  for (int j = 0; j < ORC_STEP_HIST; ++j) prev[j] = (double *)xmalloc((size_t)3 * n * sizeof(double));
  int depth = 0;
  for (int s = 0; s < n_steps; ++s) {
    orc_hier *H = orc_setup(nx, ny, nz, h, alpha, dt, m, prm);
    for (int i = 0; i < 3 * n; ++i) b[i] = m[i] / dt;
    step_guess(3 * n, depth, m, prev, x);
    depth = step_push(3 * n, depth, m, prev);
    int it = 0;
    double rr = 0.0;
    int st = orc_solve(H, b, x, prm->rtol, &it, &rr, NULL);
    if (st > worst) worst = st;
    if (iters_per_step) iters_per_step[s] = it;
    if (relres_per_step) relres_per_step[s] = rr;
    for (int k = 0; k < n; ++k) {
      double v0 = x[k], v1 = x[n + k], v2 = x[2 * n + k];
      double nrm = project ? sqrt(v0 * v0 + v1 * v1 + v2 * v2) : 1.0;
      m[k] = v0 / nrm;
      m[n + k] = v1 / nrm;
      m[2 * n + k] = v2 / nrm;
    }
    orc_free(H);
  }
  free(b);
  free(x);
  for (int j = 0; j < ORC_STEP_HIST; ++j) free(prev[j]);
  return worst;
}

/* The full model's explicit source terms (the LLG scheme at the end of
 * Sec. 2.1, no stray field): with f = -q (m2 e2 + m3 e3) + he the step solves
 * (I/dt + eps C(m^n) Delta_h) m^{n+1} = m^n/dt - C(m^n) f^n.  The exchange
 * factor eps is folded into the spacing (h/sqrt(eps)).  Same loop as orc_step
 * otherwise. */
int orc_step_llg(double *m, int n_steps, int nx, int ny, int nz, double h, double alpha, double dt,
                 const orc_params *prm, double q, const double *he, int *iters_per_step,
                 double *relres_per_step) {
  int n = nx * ny * nz, worst = ORC_OK;
  double *b = (double *)xmalloc((size_t)3 * n * sizeof(double));
  double *x = (double *)xmalloc((size_t)3 * n * sizeof(double));
  double *prev[ORC_STEP_HIST];
  for (int j = 0; j < ORC_STEP_HIST; ++j) prev[j] = (double *)xmalloc((size_t)3 * n * sizeof(double));
  int depth = 0;
  for (int s = 0; s < n_steps; ++s) {
    orc_hier *H = orc_setup(nx, ny, nz, h, alpha, dt, m, prm);
    for (int k = 0; k < n; ++k) {
      double mk[3] = {m[k], m[n + k], m[2 * n + k]}, C[3][3];
      double f[3] = {he[0], he[1] - q * mk[1], he[2] - q * mk[2]};
      coef_C(mk, alpha, C);
      for (int c = 0; c < 3; ++c) {
        double cf = C[c][0] * f[0] + C[c][1] * f[1] + C[c][2] * f[2];
        b[c * n + k] = mk[c] / dt - cf;
      }
    }
    step_guess(3 * n, depth, m, prev, x);
    depth = step_push(3 * n, depth, m, prev);
    int it = 0;
    double rr = 0.0;
    int st = orc_solve(H, b, x, prm->rtol, &it, &rr, NULL);
    if (st > worst) worst = st;
    if (iters_per_step) iters_per_step[s] = it;
    if (relres_per_step) relres_per_step[s] = rr;
    for (int k = 0; k < n; ++k) {
      double v0 = x[k], v1 = x[n + k], v2 = x[2 * n + k];
      double nrm = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      m[k] = v0 / nrm;
      m[n + k] = v1 / nrm;
      m[2 * n + k] = v2 / nrm;
    }
    orc_free(H);
  }
  free(b);
  free(x);
  for (int j = 0; j < ORC_STEP_HIST; ++j) free(prev[j]);
  return worst;
}

/* ------------------------------------------------------------------------ */
/* accessors for the test harness                                             */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* differentiation of the time step (adjoint)                                 */
/* ------------------------------------------------------------------------ */

/* Hierarchy of the transposed operator A^T: the aggregation, colouring and
 * transfers of A's hierarchy, every level operator transposed.  Since
 * (P^T A P)^T = P^T A^T P these are the Galerkin operators of A^T, and the
 * smoother, cycle and GCR of Sec. 3 then act on A^T unchanged. */
orc_hier *orc_setup_adjoint(int nx, int ny, int nz, double h, double alpha, double dt, const double *m,
                            const orc_params *prm) {
  orc_hier *H = orc_setup(nx, ny, nz, h, alpha, dt, m, prm);
  for (int l = 0; l < H->nlev; ++l) {
    csr_t t = csr_transpose(&H->lev[l].A);
    csr_free(&H->lev[l].A);
    H->lev[l].A = t;
  }
  level_t *Lc = &H->lev[H->nlev - 1];
  int nn = 3 * Lc->n;
  free(H->lu);
  H->lu = csr_to_dense(&Lc->A);
  H->singular = lu_factor(nn, H->lu, H->piv);
  if (prm->prec == 2) {
    int n0 = 3 * H->lev[0].n;
    free(H->exact_lu);
    H->exact_lu = csr_to_dense(&H->lev[0].A);
    lu_factor(n0, H->exact_lu, H->exact_piv);
  }
  return H;
}

/* Vector-Jacobian product of one step.  The step takes m = m^n to
 * m^{n+1}_k = x_k / |x_k| with A(m) x = m/dt (m~ = m^n); given x and
 * g = dL/dm^{n+1} it returns mbar = dL/dm^n and abar = dL/dalpha:
 *   xbar_k = (g_k - (u_k . g_k) u_k) / |x_k|,  u = x/|x|   (projection)
 *   A^T lambda = xbar                                     (adjoint solve)
 *   mbar_k = lambda_k/dt - [ y_k x lambda_k
 *            + alpha ((m_k . y_k) lambda_k + (lambda_k . m_k) y_k
 *                     - 2 (lambda_k . y_k) m_k) ]
 *   abar = - sum_k lambda_k . (m_k (m_k . y_k) - |m_k|^2 y_k)
 * with y = Delta_h x per component: the derivative of
 * lambda^T (b - A x) with b = m/dt and (A x)_k = x_k/dt + C(m_k) y_k. */
int orc_step_vjp(int nx, int ny, int nz, double h, double alpha, double dt, const orc_params *prm,
                 const double *m, const double *x, const double *g, double *mbar, double *abar, int *iters,
                 double *relres) {
  int n = nx * ny * nz;
  double *xbar = (double *)xmalloc((size_t)3 * n * sizeof(double));
  double *lam = (double *)xcalloc((size_t)3 * n, sizeof(double));
  double *y = (double *)xmalloc((size_t)3 * n * sizeof(double));
  for (int k = 0; k < n; ++k) {
    double v[3] = {x[k], x[n + k], x[2 * n + k]};
    double nrm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double u[3] = {v[0] / nrm, v[1] / nrm, v[2] / nrm};
    double ug = u[0] * g[k] + u[1] * g[n + k] + u[2] * g[2 * n + k];
    for (int c = 0; c < 3; ++c) xbar[c * n + k] = (g[c * n + k] - ug * u[c]) / nrm;
  }
  orc_hier *H = orc_setup_adjoint(nx, ny, nz, h, alpha, dt, m, prm);
  int st = orc_solve(H, xbar, lam, prm->rtol, iters, relres, NULL);
  orc_free(H);
  csr_t L = assemble_laplacian(nx, ny, nz, h);
  for (int c = 0; c < 3; ++c) csr_matvec(&L, x + (size_t)c * n, y + (size_t)c * n);
  csr_free(&L);
  double a = 0.0;
  for (int k = 0; k < n; ++k) {
    double mk[3] = {m[k], m[n + k], m[2 * n + k]};
    double yk[3] = {y[k], y[n + k], y[2 * n + k]};
    double lk[3] = {lam[k], lam[n + k], lam[2 * n + k]};
    double my = mk[0] * yk[0] + mk[1] * yk[1] + mk[2] * yk[2];
    double lm = lk[0] * mk[0] + lk[1] * mk[1] + lk[2] * mk[2];
    double ly = lk[0] * yk[0] + lk[1] * yk[1] + lk[2] * yk[2];
    double mm = mk[0] * mk[0] + mk[1] * mk[1] + mk[2] * mk[2];
    double yxl[3] = {yk[1] * lk[2] - yk[2] * lk[1], yk[2] * lk[0] - yk[0] * lk[2], yk[0] * lk[1] - yk[1] * lk[0]};
    for (int c = 0; c < 3; ++c)
      mbar[c * n + k] = lk[c] / dt - (yxl[c] + alpha * (my * lk[c] + lm * yk[c] - 2.0 * ly * mk[c]));
    a += lm * my - mm * ly;
  }
  *abar = -a;
  free(xbar);
  free(lam);
  free(y);
  return st;
}

int orc_nlevels(const orc_hier *H) { return H->nlev; }
int orc_level_cells(const orc_hier *H, int l) { return H->lev[l].n; }
int orc_level_nnz(const orc_hier *H, int l) { return H->lev[l].A.rowptr[H->lev[l].A.nrows]; }
int orc_level_ncolours(const orc_hier *H, int l) { return H->lev[l].ncolours; }
int orc_singular(const orc_hier *H) { return H->singular; }
void orc_level_csr(const orc_hier *H, int l, int *rowptr, int *col, double *val) {
  const csr_t *A = &H->lev[l].A;
  memcpy(rowptr, A->rowptr, ((size_t)A->nrows + 1) * sizeof(int));
  memcpy(col, A->col, (size_t)A->rowptr[A->nrows] * sizeof(int));
  memcpy(val, A->val, (size_t)A->rowptr[A->nrows] * sizeof(double));
}
void orc_level_agg(const orc_hier *H, int l, int *agg) {
  memcpy(agg, H->lev[l].agg, (size_t)H->lev[l].n * sizeof(int));
}
void orc_level_colours(const orc_hier *H, int l, int *colour) {
  memcpy(colour, H->lev[l].colour, (size_t)H->lev[l].n * sizeof(int));
}
int orc_level_graph_nnz(const orc_hier *H, int l) { return H->lev[l].g.rowptr[H->lev[l].n]; }
void orc_level_graph(const orc_hier *H, int l, int *rowptr, int *col, int *w) {
  const graph_t *g = &H->lev[l].g;
  memcpy(rowptr, g->rowptr, ((size_t)g->n + 1) * sizeof(int));
  memcpy(col, g->col, (size_t)g->rowptr[g->n] * sizeof(int));
  memcpy(w, g->w, (size_t)g->rowptr[g->n] * sizeof(int));
}
void orc_apply(const orc_hier *H, int l, const double *x, double *y) { csr_matvec(&H->lev[l].A, x, y); }
void orc_smooth(const orc_hier *H, int l, const double *b, double *x, int forward) {
  gs_sweep(&H->lev[l], b, x, forward);
}
void orc_vcycle(const orc_hier *H, const double *r, double *z) { vcycle(H, 0, r, z); }
void orc_vcycle_level(const orc_hier *H, int l, const double *r, double *z) { vcycle(H, l, r, z); }
void orc_kinner(const orc_hier *H, int l, const double *r, double *e) { kinner(H, l, r, e); }
void orc_coarse_solve(const orc_hier *H, double *x) {
  lu_solve(3 * H->lev[H->nlev - 1].n, H->lu, H->piv, x);
}

/* y = A x for the operator of Sec. 2.1 alone (no hierarchy): assembles the
 * CSR matrix and multiplies; used for residual checks at full size. */
void orc_operator_apply(int nx, int ny, int nz, double h, double alpha, double dt, const double *m,
                        const double *x, double *y) {
  csr_t A = assemble_operator(nx, ny, nz, h, alpha, dt, m);
  csr_matvec(&A, x, y);
  csr_free(&A);
}

/* Aggregates of the grid graph alone (level 0 -> 1), for full-size checks. */
int orc_grid_aggregates(int nx, int ny, int nz, int rounds, uint32_t seed, int *agg) {
  graph_t g = grid_graph(nx, ny, nz);
  int nc = aggregate_level(&g, rounds, seed, agg);
  graph_free(&g);
  return nc;
}

/* Aggregation of an arbitrary weighted graph (for tests of the rule). */
int orc_aggregate_graph(int n, const int *rowptr, const int *col, const int *w, int rounds, uint32_t seed,
                        int *agg) {
  graph_t g;
  g.n = n;
  g.rowptr = (int *)rowptr;
  g.col = (int *)col;
  g.w = (int *)w;
  return aggregate_level(&g, rounds, seed, agg);
}
int orc_matching_pass(int n, const int *rowptr, const int *col, const int *w, int rounds, uint32_t seed,
                      int attach, int *group) {
  graph_t g;
  g.n = n;
  g.rowptr = (int *)rowptr;
  g.col = (int *)col;
  g.w = (int *)w;
  return matching_pass(&g, rounds, seed, attach, group);
}
int orc_colour_graph(int n, const int *rowptr, const int *col, uint32_t seed, int *colour) {
  graph_t g;
  g.n = n;
  g.rowptr = (int *)rowptr;
  g.col = (int *)col;
  g.w = NULL;
  return colour_graph(&g, seed, colour);
}
uint32_t orc_edge_hash(uint32_t a, uint32_t b, uint32_t seed) { return edge_hash(a, b, seed); }
uint32_t orc_vertex_hash(uint32_t v, uint32_t seed) { return vertex_hash(v, seed); }
