// Batched solves of many independent instances (ll_mg_batch_*).
//
// Every instance gets its own hierarchy (the same aggregation, colouring and
// Galerkin operators as a single solve).  The batch then concatenates the
// instances level by level into one union hierarchy: union level l holds the
// rows of every instance that has a level l, colour class by colour class
// (class t of the union = class t of every instance, instance after
// instance), followed by the rows of the instances whose coarsest level l is.
// Instances are never coupled, so one launch per colour class smooths every
// instance at once and the V-cycle of the single solver runs unchanged on the
// union; level 0 is a BSR level here (red and black slots as its two
// classes).  The dense coarsest solves of all instances that end at level l
// are one launch.  GCR runs in lockstep with one set of scalars per instance
// (Algorithm 1 per instance); an instance that has converged keeps its
// residual and stops contributing to its solution.
//
// Included by ll_solver.cu after the single-instance solver.
#pragma once

struct ll_mg_batch {
  ll_mg_params prm;
  int ninst = 0;
  bool owns = true;  // false: a compacted sub-batch sharing its parent's instance hierarchies
  std::map<std::vector<int>, ll_mg_batch*> children;  // sub-batches by instance subset
  bool transposed = false;  // the instances' A^T (adjoint solves)
  cudaStream_t user = nullptr;
  cudaEvent_t entry_ev = nullptr;
  std::vector<ll_mg_hierarchy*> inst;
  ll_mg_hierarchy* U = nullptr;  // union hierarchy; its stream is the batch's
  // rmap[i][l]: rows of instance i's level l (l = 0: red-black slots) -> union rows
  // bmap[i][l] (l >= 1): blocks of instance i's level l -> union blocks
  std::vector<std::vector<llmg::DBuf<int>*>> rmap, bmap, tmap;  // tmap: transposed block positions
  llmg::DBuf<int> bad;
  std::vector<std::vector<int>> eoff;  // union row of instance i's coarsest level (per level, -1 if not ending)
  int S0 = 0;                          // union rows of level-0 class 0
  std::vector<int> off0;               // union row of instance i's first colour-0 slot
  // GCR workspace in union level-0 order (3 doubles per row)
  long n3 = 0;
  llmg::DBuf<double> Z64, C, r, xw, bw, partial, head;
  llmg::DBuf<float> Z32;
  llmg::DBuf<GcrScal> scal;
  llmg::DBuf<Chunk> chunks;
  int nchunks = 0;
  llmg::DBuf<int> iptr, act, jdone;
  double* h_head = nullptr;  // pinned, 2 per instance
  int* h_flags = nullptr;    // pinned staging of act / jdone
  cudaGraphExec_t graphs[llmg::kMaxRestart] = {nullptr};
  long long graph_kernels[llmg::kMaxRestart] = {0};
  // a batch of groups (ll_mg_batch_setup_groups): each group is a batch of
  // its own, with its own parameters; this batch then has no union (U null)
  std::vector<ll_mg_batch*> groups;
  std::vector<std::vector<int>> gidx;  // instances of each group, ascending
  ~ll_mg_batch() {
    for (auto* g : groups) delete g;
    if (U && U->s) cudaStreamSynchronize(U->s);
    for (auto& g : graphs)
      if (g) cudaGraphExecDestroy(g);
    for (auto& v : rmap)
      for (auto* b : v) delete b;
    for (auto& v : bmap)
      for (auto* b : v) delete b;
    for (auto& v : tmap)
      for (auto* b : v) delete b;
    if (h_head) cudaFreeHost(h_head);
    if (h_flags) cudaFreeHost(h_flags);
    for (auto& c : children) delete c.second;
    if (owns)
      for (auto* H : inst) delete H;
    if (entry_ev) cudaEventDestroy(entry_ev);
    delete U;
  }
};

namespace {

constexpr long kChunkElems = 3 * 2048;  // elements of one GCR chunk (one block)
constexpr int kFieldRn2 = 0, kFieldBn2 = 1, kFieldCc = 2;
constexpr int kFieldD = (int)(offsetof(GcrScal, d) / sizeof(double));
constexpr int kFieldCn2 = (int)(offsetof(GcrScal, cn2) / sizeof(double));

void batch_enter(ll_mg_batch* B) {
  if (!B->U) {  // a batch of groups: each group waits for the caller's stream
    for (auto* g : B->groups) batch_enter(g);
    return;
  }
  LL_CU(cudaEventRecord(B->entry_ev, B->user));
  LL_CU(cudaStreamWaitEvent(B->U->s, B->entry_ev, 0));
}

// exclusive scan of per-row counts into a row pointer (n + 1 entries)
int scan_counts(llmg::DBuf<int>& cnt, llmg::DBuf<int>& ptr, int n, cudaStream_t s) {
  ptr.alloc(n + 1);
  return exclusive_scan(cnt, ptr, n, s);
}

// the union hierarchy's structure: row maps, patterns, members, aggregates
void batch_symbolic(ll_mg_batch* B) {
  ll_mg_hierarchy* U = B->U;
  cudaStream_t s = U->s;
  int ni = B->ninst;
  int nlev = 0;
  for (auto* H : B->inst) nlev = std::max(nlev, H->nlev);
  U->nlev = nlev;
  B->rmap.assign(ni, std::vector<DBuf<int>*>(nlev, nullptr));
  B->bmap.assign(ni, std::vector<DBuf<int>*>(nlev, nullptr));
  B->tmap.assign(ni, std::vector<DBuf<int>*>(nlev, nullptr));
  B->eoff.assign(ni, std::vector<int>(nlev, -1));
  // ---- row maps, level 0: class c = every instance's colour-c slots
  B->off0.assign(ni, 0);
  long s0 = 0;
  for (int i = 0; i < ni; ++i) {
    B->off0[i] = (int)s0;
    s0 += B->inst[i]->g.nh;
  }
  if (2 * s0 >= (1L << 30)) throw Status{LL_ELIMIT};
  B->S0 = (int)s0;
  {
    CLevel& L = U->lev[0];
    L.n = (int)(2 * s0);
    L.ncol = 2;
    L.cs = {0, (int)s0, (int)(2 * s0)};
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      B->rmap[i][0] = new DBuf<int>();
      B->rmap[i][0]->alloc(H->n2);
      kb_union_slotmap<<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g.nh, B->off0[i], (int)s0 + B->off0[i],
                                                             *B->rmap[i][0]);
      LL_LAUNCHED();
    }
  }
  // ---- row maps, levels >= 1
  for (int l = 1; l < nlev; ++l) {
    CLevel& L = U->lev[l];
    int K = 0;
    for (auto* H : B->inst)
      if (H->nlev - 1 > l) K = std::max(K, H->lev[l].ncol);
    std::vector<std::vector<int>> off(ni, std::vector<int>(std::max(K, 1), 0));
    L.cs.assign(K + 1, 0);
    int row = 0;
    for (int t = 0; t < K; ++t) {
      L.cs[t] = row;
      for (int i = 0; i < ni; ++i) {
        ll_mg_hierarchy* H = B->inst[i];
        if (H->nlev - 1 > l && t < H->lev[l].ncol) {
          off[i][t] = row;
          row += H->lev[l].cs[t + 1] - H->lev[l].cs[t];
        }
      }
    }
    L.cs[K] = row;
    L.ncol = K;
    std::vector<CoarseTask> tasks;
    int maxN = 0;
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev - 1 == l) {
        B->eoff[i][l] = row;
        tasks.push_back({row, 3 * H->lev[l].n, H->ainv.p});
        maxN = std::max(maxN, 3 * H->lev[l].n);
        row += H->lev[l].n;
      }
    }
    L.n = row;
    if (l <= B->prm.kcycle && l < nlev - 1) {  // K-cycle tables of this level
      std::vector<Chunk> ch;
      std::vector<int> ip(1, 0), ri(L.n, -1);
      for (int i = 0; i < ni; ++i) {
        ll_mg_hierarchy* H = B->inst[i];
        if (H->nlev - 1 > l)
          for (int t = 0; t < H->lev[l].ncol; ++t) {
            int r0 = off[i][t], r1 = r0 + H->lev[l].cs[t + 1] - H->lev[l].cs[t];
            for (int r = r0; r < r1; ++r) ri[r] = i;
            for (long e = 3L * r0; e < 3L * r1; e += kChunkElems) ch.push_back({i, e, std::min(3L * r1, e + kChunkElems)});
          }
        ip.push_back((int)ch.size());
      }
      U->knch[l] = (int)ch.size();
      U->kchunks[l].alloc(ch.size());
      U->kiptr[l].alloc(ip.size());
      U->krow_inst[l].alloc(ri.size());
      if (!ch.empty())
        LL_CU(cudaMemcpyAsync(U->kchunks[l].p, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
      LL_CU(cudaMemcpyAsync(U->kiptr[l].p, ip.data(), ip.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      LL_CU(cudaMemcpyAsync(U->krow_inst[l].p, ri.data(), ri.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      LL_CU(cudaStreamSynchronize(s));  // the host tables go out of scope
    }
    U->uc_n[l] = (int)tasks.size();
    U->uc_maxN[l] = maxN;
    if (!tasks.empty()) {
      U->uc_tasks[l].alloc(tasks.size());
      LL_CU(cudaMemcpyAsync(U->uc_tasks[l].p, tasks.data(), tasks.size() * sizeof(CoarseTask),
                            cudaMemcpyHostToDevice, s));
      std::vector<int> ptr(1, 0);
      for (auto& t : tasks) ptr.push_back(ptr.back() + t.N);
      U->uc_ptr[l].alloc(ptr.size());
      LL_CU(cudaMemcpyAsync(U->uc_ptr[l].p, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      LL_CU(cudaStreamSynchronize(s));  // ptr goes out of scope
    }
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev <= l) continue;
      CLevel& Li = H->lev[l];
      bool ending = H->nlev - 1 == l;
      int ncls = ending ? 0 : Li.ncol;
      std::vector<int> tab;
      if (ending) {
        tab = {0, B->eoff[i][l]};
      } else {
        tab.assign(Li.cs.begin(), Li.cs.begin() + ncls + 1);
        for (int t = 0; t < ncls; ++t) tab.push_back(off[i][t]);
      }
      DBuf<int> dtab;
      dtab.alloc(tab.size());
      LL_CU(cudaMemcpyAsync(dtab.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      B->rmap[i][l] = new DBuf<int>();
      B->rmap[i][l]->alloc(Li.n);
      kb_union_rowmap<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, ncls, dtab, *B->rmap[i][l]);
      LL_LAUNCHED();
      LL_CU(cudaStreamSynchronize(s));  // dtab and tab go out of scope
    }
  }
  // ---- patterns
  for (int l = 0; l < nlev; ++l) {
    CLevel& L = U->lev[l];
    DBuf<int> cnt;
    cnt.alloc(L.n + 1);
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev <= l) continue;
      if (l == 0) {
        kb_union_l0_count<<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, *B->rmap[i][0], cnt);
      } else {
        CLevel& Li = H->lev[l];
        kb_union_rowcount<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.rowptr, *B->rmap[i][l], cnt);
      }
      LL_LAUNCHED();
    }
    L.nnzb = scan_counts(cnt, L.rowptr, L.n, s);
    L.col.alloc(L.nnzb);
    L.diag.alloc(L.n);
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev <= l) continue;
      if (l == 0) {
        kb_union_l0_pattern<<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, *B->rmap[i][0], L.rowptr, L.col, L.diag);
      } else {
        CLevel& Li = H->lev[l];
        B->bmap[i][l] = new DBuf<int>();
        B->bmap[i][l]->alloc(Li.nnzb);
        kb_union_pattern<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.rowptr, Li.col, Li.diag, *B->rmap[i][l],
                                                               L.rowptr, L.col, L.diag, *B->bmap[i][l]);
        if (B->transposed) {
          LL_LAUNCHED();
          B->tmap[i][l] = new DBuf<int>();
          B->tmap[i][l]->alloc(Li.nnzb);
          kb_transpose_pos<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.rowptr, Li.col, *B->tmap[i][l]);
        }
      }
      LL_LAUNCHED();
    }
  }
  // ---- members of level l in level l-1, aggregates of level l-1 in level l
  for (int l = 1; l < nlev; ++l) {
    CLevel& L = U->lev[l];
    CLevel& F = U->lev[l - 1];
    DBuf<int> cnt;
    cnt.alloc(L.n + 1);
    F.agg.alloc(F.n);
    kb_fill_int<<<cdiv(F.n, kBlock), kBlock, 0, s>>>(F.n, -1, F.agg);
    LL_LAUNCHED();
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev <= l) continue;
      CLevel& Li = H->lev[l];
      kb_union_memcount<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.mptr, *B->rmap[i][l], cnt);
      LL_LAUNCHED();
    }
    int nm = scan_counts(cnt, L.mptr, L.n, s);
    L.mem.alloc(nm);
    for (int i = 0; i < ni; ++i) {
      ll_mg_hierarchy* H = B->inst[i];
      if (H->nlev <= l) continue;
      CLevel& Li = H->lev[l];
      kb_union_members<<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.mptr, Li.mem, *B->rmap[i][l],
                                                             *B->rmap[i][l - 1], L.mptr, L.mem);
      LL_LAUNCHED();
      const int* fagg = l == 1 ? H->agg0.p : H->lev[l - 1].agg.p;
      long fn = l == 1 ? H->n2 : H->lev[l - 1].n;
      kb_union_agg<<<cdiv(fn, kBlock), kBlock, 0, s>>>(fn, fagg, *B->rmap[i][l - 1], *B->rmap[i][l], F.agg);
      LL_LAUNCHED();
    }
  }
  LL_CU(cudaStreamSynchronize(s));
  // ---- host counts of the work models (profiling)
  for (int l = 0; l < nlev; ++l) {
    CLevel& L = U->lev[l];
    std::vector<int> rp(L.n + 1), dg(L.n);
    LL_CU(cudaMemcpy(rp.data(), L.rowptr.p, (L.n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    LL_CU(cudaMemcpy(dg.data(), L.diag.p, L.n * sizeof(int), cudaMemcpyDeviceToHost));
    L.pre_blk.assign(L.ncol, 0);
    L.off_blk.assign(L.ncol, 0);
    for (int c = 0; c < L.ncol; ++c)
      for (int I = L.cs[c]; I < L.cs[c + 1]; ++I) {
        L.pre_blk[c] += dg[I] - rp[I];
        L.off_blk[c] += rp[I + 1] - rp[I] - 1;
      }
    L.res_blk = 0;
    for (int I = 0; I < (L.ncol > 0 ? L.cs[L.ncol - 1] : 0); ++I)
      L.res_blk += B->prm.nu_pre == 1 ? rp[I + 1] - dg[I] - 1 : rp[I + 1] - rp[I];
  }
}

void batch_allocate(ll_mg_batch* B) {
  ll_mg_hierarchy* U = B->U;
  bool mixed = B->prm.precision != LL_FP64;
  for (int l = 0; l < U->nlev; ++l) {
    CLevel& L = U->lev[l];
    if (l == 0 || !mixed) L.val64.alloc(9L * L.nnzb);  // level 0: also the float64 outer operator
    if (mixed) {
      L.val32.alloc(9L * L.nnzb);
      L.dinv32.alloc(9L * L.n);
      L.x32.alloc(3L * L.n);
      L.b32.alloc(3L * L.n);
      L.r32.alloc(3L * L.n);
    } else {
      L.dinv64.alloc(9L * L.n);
      L.x64.alloc(3L * L.n);
      L.b64.alloc(3L * L.n);
      L.r64.alloc(3L * L.n);
    }
  }
  int ni = B->ninst;
  // K-cycle vectors and scalars (levels 1..kcycle that are not the coarsest)
  int kmax = 0;
  for (int l = 1; l < U->nlev - 1 && l <= B->prm.kcycle; ++l) {
    for (int q = 0; q < 4; ++q) {
      if (mixed) U->lev[l].k32[q].alloc(3L * U->lev[l].n);
      else U->lev[l].k64[q].alloc(3L * U->lev[l].n);
    }
    kmax = std::max(kmax, U->knch[l]);
  }
  U->kninst = ni;
  U->kscal_u.alloc((size_t)8 * ni * U->nlev);
  U->kscal_u.zero(U->s);
  U->partial.alloc((size_t)2 * std::max(kmax, 1));
  B->n3 = 3L * U->lev[0].n;
  int m = B->prm.restart;
  if (mixed) B->Z32.alloc((size_t)m * B->n3);
  else B->Z64.alloc((size_t)m * B->n3);
  B->C.alloc((size_t)m * B->n3);
  B->r.alloc(B->n3);
  B->xw.alloc(B->n3);
  B->bw.alloc(B->n3);
  // chunks: instance-major, each instance's colour-0 rows then colour-1 rows
  std::vector<Chunk> ch;
  std::vector<int> ip(1, 0);
  for (int i = 0; i < ni; ++i) {
    long nh = B->inst[i]->g.nh;
    for (long base : {(long)B->off0[i], (long)B->S0 + B->off0[i]}) {
      long e0 = 3 * base, e1 = 3 * (base + nh);
      for (long e = e0; e < e1; e += kChunkElems) ch.push_back({i, e, std::min(e1, e + kChunkElems)});
    }
    ip.push_back((int)ch.size());
  }
  B->nchunks = (int)ch.size();
  B->chunks.alloc(ch.size());
  LL_CU(cudaMemcpyAsync(B->chunks.p, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, U->s));
  B->iptr.alloc(ip.size());
  LL_CU(cudaMemcpyAsync(B->iptr.p, ip.data(), ip.size() * sizeof(int), cudaMemcpyHostToDevice, U->s));
  B->partial.alloc((size_t)(kDotChunk + 1) * B->nchunks);  // dots plus |c|^2
  B->scal.alloc(ni);
  B->scal.zero(U->s);
  B->head.alloc(2 * ni);
  B->act.alloc(ni);
  B->jdone.alloc(ni);
  LL_CU(cudaMallocHost((void**)&B->h_head, 2 * ni * sizeof(double)));
  LL_CU(cudaMallocHost((void**)&B->h_flags, ni * sizeof(int)));
  LL_CU(cudaStreamSynchronize(U->s));
}

// The union's small levels (from the first with at most kTailCells rows, K
// levels excluded) run in one thread-block-cluster kernel, as a single
// instance's do, with every instance's dense solve at the level where it
// ends (off with LLMG_NO_TAIL=1).
void batch_tail(ll_mg_batch* B) { setup_tail(B->U); }

// numeric values of the union from the instances' numeric setups
template <typename T, typename TM>
void batch_values(ll_mg_batch* B) {
  ll_mg_hierarchy* U = B->U;
  cudaStream_t s = U->s;
  for (auto* H : B->inst) LL_CU(cudaStreamSynchronize(H->s));
  bool mixed = !std::is_same<T, double>::value;
  if (B->transposed) B->bad.zero(s);
  for (int i = 0; i < B->ninst; ++i) {
    ll_mg_hierarchy* H = B->inst[i];
    CLevel& L0 = U->lev[0];
    T* valt = mixed ? (T*)L0.val32.p : (T*)nullptr;
    if (B->transposed)
      kb_union_l0_values_t<T><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, *B->rmap[i][0], L0.rowptr, H->chat64,
                                                                    H->dinv0<T>(), 1.0 / H->dt, L0.val64, valt,
                                                                    L0.dinv<T>());
    else
      kb_union_l0_values<T><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, *B->rmap[i][0], L0.rowptr, L0.diag,
                                                                  H->chat64, H->dinv0<T>(), 1.0 / H->dt, L0.val64,
                                                                  valt, L0.dinv<T>());
    LL_LAUNCHED();
    for (int l = 1; l < H->nlev; ++l) {
      CLevel& Li = H->lev[l];
      CLevel& L = U->lev[l];
      if (B->transposed)
        kb_union_values_t<TM, T><<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(
            Li.n, Li.rowptr, *B->bmap[i][l], *B->tmap[i][l], *B->rmap[i][l], Li.valm<TM>(), Li.dinv<T>(),
            L.valm<TM>(), L.dinv<T>(), B->bad);
      else
        kb_union_values<TM, T><<<cdiv(Li.n, kBlock), kBlock, 0, s>>>(Li.n, Li.rowptr, *B->bmap[i][l],
                                                                     *B->rmap[i][l], Li.valm<TM>(), Li.dinv<T>(),
                                                                     L.valm<TM>(), L.dinv<T>());
      LL_LAUNCHED();
    }
  }
  if (B->transposed) {
    int bad = 0;
    LL_CU(cudaMemcpyAsync(&bad, B->bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CU(cudaStreamSynchronize(s));
    if (bad) {  // a pattern without its transpose: not a Galerkin level
      note_internal_error("union pattern without its transpose", __FILE__, __LINE__);
      throw Status{LL_ECUDA};
    }
  }
  LL_CU(cudaStreamSynchronize(s));
}

void batch_refresh(ll_mg_batch* B) {
  if (B->prm.precision == LL_MIXED_FP32) batch_values<float, float>(B);
  else batch_values<double, double>(B);
}

void batch_finish(ll_mg_batch* B, int nvals, int field, bool gated = false, int row0 = 0) {
  kgb_finish<<<dim3(B->ninst, nvals), kBlock, 0, B->U->s>>>(B->partial.p + (size_t)row0 * B->nchunks, B->nchunks,
                                                             B->iptr, B->scal, field, gated);
  LL_LAUNCHED();
}

// one lockstep GCR iteration j of every instance (no host interaction)
template <typename T, typename TM>
void batch_iteration_body(ll_mg_batch* B, int j) {
  ll_mg_hierarchy* U = B->U;
  cudaStream_t s = U->s;
  CLevel& L0 = U->lev[0];
  long n3 = B->n3;
  int ni = B->ninst, nch = B->nchunks;
  GcrScal* S = B->scal.p;
  T* Zbase = std::is_same<T, double>::value ? (T*)B->Z64.p : (T*)B->Z32.p;
  T* zj = Zbase + (size_t)j * n3;
  double* cj = B->C.p + (size_t)j * n3;
  k_convert<double, T><<<cdiv(n3, kBlock), kBlock, 0, s>>>(n3, B->r, L0.b<T>());  // step 1
  LL_LAUNCHED();
  vcycle_coarse<T, TM>(U, 0, false);
  LL_CU(cudaMemcpyAsync(zj, L0.x<T>(), n3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
  kgb_apply<T><<<cdiv(L0.n, kBlock), kBlock, 0, s>>>(L0.n, L0.rowptr, L0.col, L0.val64, zj, cj);  // step 2
  LL_LAUNCHED();
  for (int pass = 0; pass < 2 && j > 0; ++pass) {  // step 3: CGS, second pass per instance when needed
    const GcrScal* gate = pass == 0 ? nullptr : S;
    for (int i0 = 0; i0 < j; i0 += kDotChunk) {
      int cnt = std::min(kDotChunk, j - i0);
      bool self = pass == 0 && i0 == 0;
      if (self)
        launch_batch_multidot<kDotChunk, true>(cnt, s, nch, B->chunks, B->C, n3, i0, cj, B->partial);
      else
        launch_batch_multidot<kDotChunk, false>(cnt, s, nch, B->chunks, B->C, n3, i0, cj, B->partial, gate);
      LL_LAUNCHED();
      batch_finish(B, cnt, kFieldD + i0, pass == 1);
      if (self) batch_finish(B, 1, kFieldCn2, false, cnt);
    }
    kgb_gs_coef<<<cdiv(ni, 64), 64, 0, s>>>(S, ni, j, pass == 0);
    LL_LAUNCHED();
    kgb_multiaxpy<<<nch, kBlock, 0, s>>>(B->chunks, cj, B->C, n3, j, S, gate);
    LL_LAUNCHED();
  }
  kgb_dot2<<<nch, kBlock, 0, s>>>(B->chunks, nch, cj, B->r, B->partial);  // step 4
  LL_LAUNCHED();
  batch_finish(B, 2, kFieldCc);
  kgb_norm_coef<<<cdiv(ni, 64), 64, 0, s>>>(S, ni, j, B->act);
  LL_LAUNCHED();
  kgb_rupdate<<<nch, kBlock, 0, s>>>(B->chunks, nch, B->r, cj, S, B->partial);  // step 5
  LL_LAUNCHED();
  batch_finish(B, 1, kFieldRn2);
  kgb_head<<<cdiv(ni, 64), 64, 0, s>>>(S, ni, B->head);
  LL_LAUNCHED();
  LL_CU(cudaMemcpyAsync(B->h_head, B->head.p, 2 * ni * sizeof(double), cudaMemcpyDeviceToHost, s));
}

template <typename T, typename TM>
void batch_run_iteration(ll_mg_batch* B, int j) {
  cudaStream_t s = B->U->s;
  if (!B->U->use_graphs) {
    batch_iteration_body<T, TM>(B, j);
  } else {
    if (!B->graphs[j]) {
      cudaGraph_t graph;
      long long before = t_launches;
      LL_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      try {
        batch_iteration_body<T, TM>(B, j);
      } catch (Status) {
        cudaStreamEndCapture(s, &graph);
        throw;
      }
      LL_CU(cudaStreamEndCapture(s, &graph));
      cudaError_t e = cudaGraphInstantiate(&B->graphs[j], graph, 0);
      cudaGraphDestroy(graph);
      LL_CU(e);
      B->graph_kernels[j] = t_launches - before;
      g_launches.fetch_sub(B->graph_kernels[j]);
    }
    LL_CU(cudaGraphLaunch(B->graphs[j], s));
    g_launches.fetch_add(B->graph_kernels[j]);
  }
  LL_CU(cudaStreamSynchronize(s));
}

void batch_upload(ll_mg_batch* B, const std::vector<int>& v, int* dst) {
  std::copy(v.begin(), v.end(), B->h_flags);
  LL_CU(cudaMemcpyAsync(dst, B->h_flags, v.size() * sizeof(int), cudaMemcpyHostToDevice, B->U->s));
  LL_CU(cudaStreamSynchronize(B->U->s));  // h_flags is reused
}

void batch_true_residual(ll_mg_batch* B) {
  ll_mg_hierarchy* U = B->U;
  CLevel& L0 = U->lev[0];
  kgb_residual<<<B->nchunks, kBlock, 0, U->s>>>(B->chunks, B->nchunks, L0.rowptr, L0.col, L0.val64, B->bw, B->xw,
                                                B->r, B->partial);
  LL_LAUNCHED();
  batch_finish(B, 2, kFieldRn2);
  kgb_head2<<<cdiv(B->ninst, 64), 64, 0, U->s>>>(B->scal, B->ninst, B->head);
  LL_LAUNCHED();
  LL_CU(cudaMemcpyAsync(B->h_head, B->head.p, 2 * B->ninst * sizeof(double), cudaMemcpyDeviceToHost, U->s));
  LL_CU(cudaStreamSynchronize(U->s));
}

// The solve's state of one instance, kept across sub-batches.
struct InstState {
  int total = 0;              // GCR iterations so far
  int st = LL_NOT_CONVERGED;  // final status once done
  int done = 0;               // 0 running, 1 finished, 2 finished with a zero right-hand side (x = 0)
  double relres = 0;
  bool paused = false;        // stopped at a restart boundary to continue in a smaller sub-batch
  StallHist stall;            // true residual norms at its restarts (stagnation stop)
};

// GCR (Algorithm 1) on every instance in lockstep, restarts of prm.restart;
// per instance the same decisions as the single solve.  With compact, the
// solve pauses at a restart boundary once the instances still iterating
// hold under half of the union's rows: they continue in a sub-batch of their
// own, from their current iterate, exactly as a restart would.
template <typename T, typename TM>
void batch_gcr(ll_mg_batch* B, double rtol, std::vector<InstState*>& S, bool compact) {
  ll_mg_hierarchy* U = B->U;
  cudaStream_t s = U->s;
  int ni = B->ninst;
  long n3 = B->n3;
  T* Zbase = std::is_same<T, double>::value ? (T*)B->Z64.p : (T*)B->Z32.p;
  std::vector<int> act(ni, 0), jd(ni, 0);
  std::vector<double> bnorm(ni, 0.0);
  long rows_all = 0;
  for (int i = 0; i < ni; ++i) rows_all += B->inst[i]->n2;
  for (;;) {
    batch_true_residual(B);
    int running = 0;
    long rows_running = 0;
    int tmin = 1 << 30;
    for (int i = 0; i < ni; ++i) {
      act[i] = 0;
      InstState& q = *S[i];
      int& total = q.total;
      int& st = q.st;
      int& done = q.done;
      if (done) continue;
      double rn2 = B->h_head[2 * i];
      bnorm[i] = sqrt(B->h_head[2 * i + 1]);
      if (bnorm[i] == 0.0) {  // zero right-hand side: x = 0 below
        st = LL_OK;
        done = 2;
      } else if (!isfinite(rn2)) {
        st = LL_BREAKDOWN;
        done = 1;
      } else if (sqrt(rn2) < rtol * bnorm[i]) {
        st = LL_OK;
        done = 1;
      } else if (total >= B->prm.maxit || q.stall.stalled(B->prm, total, sqrt(rn2))) {
        done = 1;
      } else {
        act[i] = 1;
        ++running;
        rows_running += B->inst[i]->n2;
        tmin = std::min(tmin, total);
      }
    }
    if (running == 0) break;
    if (compact && 2 * rows_running < rows_all) {
      for (int i = 0; i < ni; ++i) S[i]->paused = act[i] != 0;
      break;
    }
    int m = std::min(B->prm.restart, B->prm.maxit - tmin);
    std::fill(jd.begin(), jd.end(), 0);
    batch_upload(B, act, B->act);
    std::vector<int> cyc = act;  // still iterating in this cycle
    for (int j = 0; j < m; ++j) {
      batch_run_iteration<T, TM>(B, j);
      bool changed = false;
      int left = 0;
      for (int i = 0; i < ni; ++i) {
        if (!cyc[i]) continue;
        InstState& q = *S[i];
        ++q.total;
        double rn2 = B->h_head[2 * i], gjj = B->h_head[2 * i + 1];
        if (!(gjj > 0.0) || !isfinite(gjj) || !isfinite(rn2)) {
          q.st = LL_BREAKDOWN;
          q.done = 1;
          cyc[i] = 0;
          changed = true;
          continue;
        }
        jd[i] = j + 1;
        if (sqrt(rn2) < rtol * bnorm[i] || q.total >= B->prm.maxit) {  // step 6
          cyc[i] = 0;
          changed = true;
          continue;
        }
        ++left;
      }
      if (left == 0) break;
      if (changed) batch_upload(B, cyc, B->act);
    }
    batch_upload(B, jd, B->jdone);
    kgb_backsub<<<cdiv(ni, 64), 64, 0, s>>>(B->scal, ni, B->jdone);
    LL_LAUNCHED();
    kgb_xupdate<T><<<B->nchunks, kBlock, 0, s>>>(B->chunks, B->xw, Zbase, n3, B->scal, B->jdone);
    LL_LAUNCHED();
  }
  batch_true_residual(B);
  for (int i = 0; i < ni; ++i) {
    if (S[i]->paused || !S[i]->done) continue;
    double bn = sqrt(B->h_head[2 * i + 1]);
    S[i]->relres = bn > 0 ? sqrt(B->h_head[2 * i]) / bn : 0.0;
  }
}

// the union hierarchy and workspace of a set of instance hierarchies
void batch_build(ll_mg_batch* B) {
  B->U = new ll_mg_hierarchy();
  ll_mg_hierarchy* U = B->U;
  U->prm = B->prm;
  U->union_mode = true;
  U->tail_first = -1;
  U->user = B->user;
  LL_CU(cudaStreamCreateWithFlags(&U->s, cudaStreamNonBlocking));
  LL_CU(cudaEventCreateWithFlags(&U->entry_ev, cudaEventDisableTiming));
  const char* ng = getenv("LLMG_NO_GRAPHS");
  U->use_graphs = !(ng && ng[0] == '1');
}

// the sub-batch of B's instances `sub` (ascending), built once and kept
ll_mg_batch* batch_child(ll_mg_batch* B, const std::vector<int>& sub) {
  auto it = B->children.find(sub);
  if (it != B->children.end()) return it->second;
  ll_mg_batch* C = new ll_mg_batch();
  try {
    C->prm = B->prm;
    C->ninst = (int)sub.size();
    C->owns = false;
    C->transposed = B->transposed;
    if (C->transposed) C->bad.alloc(1);
    C->user = B->U->s;
    LL_CU(cudaEventCreateWithFlags(&C->entry_ev, cudaEventDisableTiming));
    for (int i : sub) C->inst.push_back(B->inst[i]);
    batch_build(C);
    batch_symbolic(C);
    batch_allocate(C);
    batch_tail(C);
    batch_refresh(C);
  } catch (...) {
    delete C;
    throw;
  }
  B->children[sub] = C;
  return C;
}

int batch_solve(ll_mg_batch* B, const double* const* rhs, double* const* x, double rtol, int* iters, double* relres,
                int* status) {
  if (rtol <= 0) rtol = B->prm.rtol;
  const char* nc = getenv("LLMG_BATCH_NO_COMPACT");
  bool compact = !(nc && nc[0] == '1');
  int ni = B->ninst;
  std::vector<InstState> state(ni);
  ll_mg_batch* cur = B;
  std::vector<int> idx(ni);
  for (int i = 0; i < ni; ++i) idx[i] = i;
  for (;;) {
    cudaStream_t s = cur->U->s;
    for (int k = 0; k < cur->ninst; ++k) {
      ll_mg_hierarchy* H = cur->inst[k];
      kb_union_in<double, double><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, H->nat_of_slot, *cur->rmap[k][0],
                                                                        rhs[idx[k]], cur->bw);
      LL_LAUNCHED();
      kb_union_in<double, double><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, H->nat_of_slot, *cur->rmap[k][0],
                                                                        x[idx[k]], cur->xw);
      LL_LAUNCHED();
    }
    std::vector<InstState*> sp(cur->ninst);
    for (int k = 0; k < cur->ninst; ++k) sp[k] = &state[idx[k]];
    // a sub-batch of one instance would only move its rows; stop compacting there
    if (cur->prm.precision == LL_MIXED_FP32) batch_gcr<float, float>(cur, rtol, sp, compact && cur->ninst > 1);
    else batch_gcr<double, double>(cur, rtol, sp, compact && cur->ninst > 1);
    std::vector<int> sub;
    for (int k = 0; k < cur->ninst; ++k) {
      ll_mg_hierarchy* H = cur->inst[k];
      double* xo = x[idx[k]];
      if (sp[k]->done == 2) {  // zero right-hand side: the solution is zero
        LL_CU(cudaMemsetAsync(xo, 0, 3 * H->g.n * sizeof(double), s));
      } else {
        kb_union_out<double, double><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(H->g, H->nat_of_slot,
                                                                           *cur->rmap[k][0], cur->xw, xo);
        LL_LAUNCHED();
      }
      if (sp[k]->paused) {
        sp[k]->paused = false;
        sub.push_back(idx[k]);
      }
    }
    LL_CU(cudaStreamSynchronize(s));
    if (sub.empty()) break;
    cur = batch_child(B, sub);
    idx = sub;
  }
  int worst = LL_OK;
  for (int i = 0; i < ni; ++i) {
    if (iters) iters[i] = state[i].total;
    if (relres) relres[i] = state[i].relres;
    if (status) status[i] = state[i].st;
    if (state[i].st == LL_BREAKDOWN) worst = LL_BREAKDOWN;
    else if (state[i].st == LL_NOT_CONVERGED && worst == LL_OK) worst = LL_NOT_CONVERGED;
  }
  return worst;
}

int batch_create(int count, const double* const* m, const double* alpha, const double* dt, const double* h,
                 const ll_grid* grids, const ll_mg_params* p, void* stream, ll_mg_batch** out,
                 bool transposed = false) {
  ll_mg_batch* B = nullptr;
  try {
    B = new ll_mg_batch();
    ll_mg_default_params(&B->prm);
    if (p) B->prm = *p;
    B->transposed = transposed;
    if (transposed) B->bad.alloc(1);
    B->ninst = count;
    B->user = (cudaStream_t)stream;
    LL_CU(cudaEventCreateWithFlags(&B->entry_ev, cudaEventDisableTiming));
    batch_build(B);
    ll_mg_hierarchy* U = B->U;
    batch_enter(B);
    LL_CU(cudaStreamSynchronize(U->s));  // the callers' fields are ready
    ll_mg_params ip = B->prm;
    for (int i = 0; i < count; ++i) {
      ll_mg_hierarchy* H = nullptr;
      int rc = create(m[i], alpha[i], dt[i], h[i], grids[i], &ip, nullptr, &H, false);
      if (rc != LL_OK) throw Status{rc};
      B->inst.push_back(H);
      if (H->nlev < 2) throw Status{LL_EINVAL};  // too small to coarsen: solve it alone
    }
    batch_symbolic(B);
    batch_allocate(B);
    batch_tail(B);
    batch_refresh(B);
    *out = B;
    return LL_OK;
  } catch (Status st) {
    delete B;
    return st.code;
  } catch (std::bad_alloc&) {
    delete B;
    return LL_ENOMEM;
  }
}

// ---------------------------------------------------------------------------
// batches of groups: instances with different parameters (the autotuner's
// choice per class of instances) are split into groups of equal parameters;
// each group is a batch of its own, and the groups are solved concurrently,
// one host thread and one stream per group.
// ---------------------------------------------------------------------------
bool same_params(const ll_mg_params& a, const ll_mg_params& b) {
  return a.rtol == b.rtol && a.maxit == b.maxit && a.restart == b.restart && a.nu_pre == b.nu_pre &&
         a.nu_post == b.nu_post && a.coarsest_cells == b.coarsest_cells && a.max_levels == b.max_levels &&
         a.rounds == b.rounds && a.seed == b.seed && a.precision == b.precision && a.kcycle == b.kcycle &&
         a.coarse_lanes == b.coarse_lanes && a.coarse_block == b.coarse_block &&
         a.stall_window == b.stall_window && (a.stall_window == 0 || a.stall_ratio == b.stall_ratio);
}

int batch_create_groups(int count, const double* const* m, const double* alpha, const double* dt, const double* h,
                        const ll_grid* grids, const ll_mg_params* p, void* stream, ll_mg_batch** out) {
  std::vector<int> gof(count, -1);
  std::vector<ll_mg_params> gp;
  std::vector<std::vector<int>> gidx;
  for (int i = 0; i < count; ++i) {
    int g = 0;
    while (g < (int)gp.size() && !same_params(gp[g], p[i])) ++g;
    if (g == (int)gp.size()) {
      gp.push_back(p[i]);
      gidx.emplace_back();
    }
    gidx[g].push_back(i);
  }
  if (gp.size() == 1) return batch_create(count, m, alpha, dt, h, grids, &gp[0], stream, out);
  ll_mg_batch* B = new ll_mg_batch();
  B->prm = gp[0];
  B->ninst = count;
  B->user = (cudaStream_t)stream;
  B->gidx = gidx;
  for (size_t g = 0; g < gp.size(); ++g) {
    std::vector<const double*> mg;
    std::vector<double> ag, dg, hg;
    std::vector<ll_grid> gg;
    for (int i : gidx[g]) {
      mg.push_back(m[i]);
      ag.push_back(alpha[i]);
      dg.push_back(dt[i]);
      hg.push_back(h[i]);
      gg.push_back(grids[i]);
    }
    ll_mg_batch* G = nullptr;
    int rc = batch_create((int)gidx[g].size(), mg.data(), ag.data(), dg.data(), hg.data(), gg.data(), &gp[g],
                          stream, &G);
    if (rc != LL_OK) {
      delete B;
      return rc;
    }
    B->groups.push_back(G);
  }
  *out = B;
  return LL_OK;
}

// run fn(group, its instance indices) for every group, one host thread per
// group; returns the first failure (negative status) or the worst outcome
// (a failing group's CUDA error text is passed on to the calling thread)
template <typename F>
int for_groups(ll_mg_batch* B, F fn) {
  int ng = (int)B->groups.size();
  std::vector<int> rc(ng, LL_OK);
  std::vector<std::string> err(ng);
  std::vector<std::thread> th;
  for (int g = 0; g < ng; ++g)
    th.emplace_back([&, g]() {
      try {
        rc[g] = fn(B->groups[g], B->gidx[g]);
      } catch (Status st) {
        rc[g] = st.code;
      } catch (std::bad_alloc&) {
        rc[g] = LL_ENOMEM;
      }
      if (rc[g] < 0) err[g] = t_cuda_error;
    });
  for (auto& t : th) t.join();
  int worst = LL_OK;
  for (int g = 0; g < ng; ++g)
    if (rc[g] < 0) {
      snprintf(t_cuda_error, sizeof t_cuda_error, "%s", err[g].c_str());
      return rc[g];
    }
  for (int r : rc) worst = std::max(worst, r);
  return worst;
}

}  // namespace
