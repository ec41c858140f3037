// Hierarchy, numeric setup, V-cycle, GCR and the C ABI of the sm_103a
// aggregation-multigrid solver (see include/ll_mg.h for the contract).
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <type_traits>

#include "ll_internal.cuh"
#include "ll_kernels.cuh"
#include "ll_setup.cuh"
#include "ll_tail.cuh"
#include "ll_batch_kernels.cuh"

#include <atomic>
#include <thread>

namespace llmg {

// kernels launched: in total (all threads), and by the calling thread (the
// kernels a graph capture records are counted on the capturing thread, so
// that concurrent captures on other threads do not enter its count)
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}

// the calling thread's last failed CUDA call, for ll_last_cuda_error
static thread_local char t_cuda_error[160] = "";
void note_cuda_error(cudaError_t e, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(t_cuda_error, sizeof t_cuda_error, "%s (%s) at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e),
           base ? base + 1 : file, line);
}
void note_internal_error(const char* what, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(t_cuda_error, sizeof t_cuda_error, "%s at %s:%d", what, base ? base + 1 : file, line);
}

struct CLevel {  // an aggregated level l >= 1 (3x3 BSR operator)
  int n = 0, nnzb = 0, ncol = 0;
  // in the aggregation's own numbering (rank of the smallest member)
  DevGraph graph;                   // integer weight graph
  DBuf<int> colour;                 // Jones-Plassmann colour of each cell
  DBuf<int> agg_orig;               // this level -> next level
  // renumbering by colour: new cell r is cell n2o[r]; colour c owns the new
  // range [cs[c], cs[c+1])
  DBuf<int> n2o, o2n;
  std::vector<int> cs;
  // below: new numbering
  DBuf<int> rowptr, col, diag;      // BSR pattern
  DBuf<int> prow;                   // row of each block
  DBuf<int> sptr, sidx, sw;         // Galerkin slot map from the finer level
  DBuf<int> gperm;                  // blocks by decreasing slot-list length (Galerkin thread order)
  DBuf<int> mptr, mem;              // members in the finer level (level 1: red-black slots)
  DBuf<int> mptr0, mem0;            // level 1: colour-0 slots only
  DBuf<int> agg;                    // this level -> next level
  // host counts for the algorithmic work of the kernels (profiling only)
  std::vector<long long> pre_blk, off_blk;  // per colour class: prefix / off-diagonal blocks
  long long res_blk = 0;                    // blocks the residual reads (rows before the last colour)
  DBuf<double> val64, dinv64;
  // SELL-32 copy of the off-diagonal blocks (float64 levels whose colour
  // classes are large; the layout is described at ks_sweep)
  bool sell = false;
  long sgroups = 0;        // slot groups
  DBuf<int> soff, sgc;     // slot-group offset of each chunk; chunk of each slot group
  DBuf<int> scol;          // column of each slot (-1: padding)
  DBuf<double> sval;       // block entries of each slot
  DBuf<float> val32, dinv32;
  DBuf<__nv_bfloat16> val16;        // bfloat16 storage of the operator (LL_MIXED_BF16)
  DBuf<double> x64, b64, r64;
  DBuf<float> x32, b32, r32;
  DBuf<double> k64[4];  // K-cycle vectors: r, z1, c1, c2
  DBuf<float> k32[4];
  template <typename T> T* kv(int i);
  template <typename T> T* val();
  template <typename TM> TM* valm();  // operator values in storage type TM
  template <typename T> T* dinv();
  template <typename T> T* x();
  template <typename T> T* b();
  template <typename T> T* r();
};
template <> double* CLevel::val<double>() { return val64; }
template <> float* CLevel::val<float>() { return val32; }
template <> double* CLevel::valm<double>() { return val64; }
template <> float* CLevel::valm<float>() { return val32; }
template <> __nv_bfloat16* CLevel::valm<__nv_bfloat16>() { return val16; }
template <> double* CLevel::dinv<double>() { return dinv64; }
template <> float* CLevel::dinv<float>() { return dinv32; }
template <> double* CLevel::x<double>() { return x64; }
template <> float* CLevel::x<float>() { return x32; }
template <> double* CLevel::b<double>() { return b64; }
template <> float* CLevel::b<float>() { return b32; }
template <> double* CLevel::kv<double>(int i) { return k64[i]; }
template <> float* CLevel::kv<float>(int i) { return k32[i]; }
template <> double* CLevel::r<double>() { return r64; }
template <> float* CLevel::r<float>() { return r32; }

}  // namespace llmg

using namespace llmg;

struct ll_mg_hierarchy {
  ll_mg_params prm;
  cudaStream_t s = nullptr;     // the library's own stream (capturable)
  cudaStream_t user = nullptr;  // the caller's stream
  cudaEvent_t entry_ev = nullptr;
  GridGeom g;
  double alpha = 0, dt = 1, h = 1;
  int nlev = 1;
  long n2 = 0, n3 = 0;
  // level 0
  DevGraph graph0;
  DBuf<int> agg_nat0, agg0, nat_of_slot;
  DBuf<double> chat64, dinv64;
  DBuf<float> chat32, dinv32;
  DBuf<float> chatlo;  // mixed: C^ - chat32 (the pair (chat32, chatlo) of kg_apply_ff)
  DBuf<float> m32;  // m~ per slot: the float32 level-0 kernels form C and D^-1 from it
  DBuf<double> r0tmp64;  // colour-0 residual of the level-0 restriction (float64 path)
  bool sell_ok = false;  // large float64 classes may use the SELL-32 sweeps (not in batches)
  // time-stepping history for the steps' initial approximations: up to
  // kStepHist states before the last output (step_h[(step_i + j) % kStepHist]
  // holds the j-th newest, j < step_depth) and the last output itself
  // (step_last), valid when step_hist is set; step_norms: the squared norms
  // of the backward differences
  DBuf<double> step_h[kStepHist], step_last, step_norms;
  DBuf<int> step_differ;
  int step_i = 0, step_depth = 0;
  bool step_hist = false;
  CLevel lev[kMaxLevels];
  // coarsest dense LU and its inverse (column-major)
  int ncoarse3 = 0;
  int gj_cluster = 0;  // CTAs of the coarsest inverse's cluster (0: not chosen yet)
  DBuf<double> lu, ainv;
  DBuf<int> perm, lu_status, flag;
  // GCR workspace (red-black layout, 3*n2 doubles per vector)
  DBuf<double> Z64, C, r, xw, bw, partial;
  DBuf<float> Z32;
  DBuf<GcrScal> scal;
  DBuf<double> kscal;  // K-cycle scalars, 8 per level
  double* h_head = nullptr;  // pinned copy of the first scalars
  // time-step workspace (natural layout)
  DBuf<double> stepb, stepx;
  DBuf<double> hostm;  // device copy of a host field (ll_mg_step_host), allocated on first use
  // the small coarse levels as one cluster kernel
  int tail_first = -1;  // first tail level, -1: no tail
  int tail_cluster = 0;
  DBuf<TailArgs<double, double>> tail64;
  DBuf<TailArgs<float, float>> tail32;
  DBuf<TailArgs<float, __nv_bfloat16>> tail16;
  template <typename T, typename TM> DBuf<TailArgs<T, TM>>& tail();
  // single-level hierarchies: cell-major scratch of the direct solve
  DBuf<double> single_b, single_x;
  // union hierarchy of a batch: level 0 is a BSR level too, and the
  // instances whose coarsest level is l are solved densely at level l
  bool union_mode = false;
  DBuf<CoarseTask> uc_tasks[kMaxLevels];
  DBuf<int> uc_ptr[kMaxLevels];  // running sums of the tasks' sizes N
  int uc_n[kMaxLevels] = {0}, uc_maxN[kMaxLevels] = {0};
  // union hierarchies with the K-cycle: per K level, element chunks of the
  // rows of every instance that has the K-cycle there (instance-major), the
  // chunk range of each instance, the instance of each row (-1: none), and 8
  // scalars per instance and level
  int kninst = 0;
  DBuf<Chunk> kchunks[kMaxLevels];
  DBuf<int> kiptr[kMaxLevels], krow_inst[kMaxLevels];
  int knch[kMaxLevels] = {0};
  DBuf<double> kscal_u;
  // kernel timing (ll_mg_profile)
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pairs[LL_NUM_KINDS];
  double prof_ms[LL_NUM_KINDS] = {0};
  long long prof_n[LL_NUM_KINDS] = {0};  // kernel launches timed
  double prof_flops[LL_NUM_KINDS] = {0}, prof_bytes[LL_NUM_KINDS] = {0};
  long long l0_cells[2] = {0, 0};  // real cells of each colour
  double tail_flops = 0, tail_bytes = 0;  // one launch of the cluster tail
  cudaEvent_t event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      LL_CU(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
  // CUDA graphs of the GCR iterations (one per position j in a cycle)
  bool use_graphs = true;
  int capturing = -1;  // j of the iteration being captured, or -1
  double graph_dt = 0;
  cudaGraphExec_t graphs[kMaxRestart] = {nullptr};
  unsigned graph_mask[kMaxRestart] = {0};
  long long graph_kernels[kMaxRestart] = {0};
  struct GPair {
    int kind;
    cudaEvent_t b, e;
    double flops, bytes;
    int nl;  // kernel launches between b and e
  };
  std::vector<GPair> gpairs[kMaxRestart];
  void drop_graph(int j) {
    if (graphs[j]) cudaGraphExecDestroy(graphs[j]);
    graphs[j] = nullptr;
    for (auto& q : gpairs[j]) {
      cudaEventDestroy(q.b);
      cudaEventDestroy(q.e);
    }
    gpairs[j].clear();
  }
  ~ll_mg_hierarchy() {
    if (s) cudaStreamSynchronize(s);
    for (int j = 0; j < kMaxRestart; ++j) drop_graph(j);
    if (h_head) cudaFreeHost(h_head);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (entry_ev) cudaEventDestroy(entry_ev);
    if (s) cudaStreamDestroy(s);
  }
  template <typename T> T* chat();
  template <typename T> T* dinv0();
  template <typename T> T* Z();
};
template <> double* ll_mg_hierarchy::chat<double>() { return chat64; }
template <> float* ll_mg_hierarchy::chat<float>() { return chat32; }
template <> double* ll_mg_hierarchy::dinv0<double>() { return dinv64; }
template <> float* ll_mg_hierarchy::dinv0<float>() { return dinv32; }
template <> DBuf<TailArgs<double, double>>& ll_mg_hierarchy::tail<double, double>() { return tail64; }
template <> DBuf<TailArgs<float, float>>& ll_mg_hierarchy::tail<float, float>() { return tail32; }
template <> DBuf<TailArgs<float, __nv_bfloat16>>& ll_mg_hierarchy::tail<float, __nv_bfloat16>() { return tail16; }
template <> double* ll_mg_hierarchy::Z<double>() { return Z64; }
template <> float* ll_mg_hierarchy::Z<float>() { return Z32; }

namespace {

// brackets the launches in its scope with CUDA events when their kind is timed
struct ProfScope {
  ll_mg_hierarchy* H;
  int kind;
  cudaEvent_t b = nullptr;
  double flops, bytes;  // algorithmic work of the launches in the scope
  int nl;               // kernel launches in the scope
  ProfScope(ll_mg_hierarchy* h, int k, double f = 0, double by = 0, int n = 1)
      : H(h), kind(k), flops(f), bytes(by), nl(n) {
    if (kind >= LL_NUM_KINDS || !(H->prof_mask & (1u << kind))) return;
    if (H->capturing < 0) {
      H->prof_flops[kind] += flops;
      H->prof_bytes[kind] += bytes;
    }
    if (H->capturing >= 0) {  // inside a graph: event-record nodes of its own
      LL_CU(cudaEventCreate(&b));
      LL_CU(cudaEventRecordWithFlags(b, H->s, cudaEventRecordExternal));
    } else {
      b = H->event();
      LL_CU(cudaEventRecord(b, H->s));
    }
  }
  ~ProfScope() noexcept(false) {
    if (!b) return;
    if (H->capturing >= 0) {
      cudaEvent_t e;
      LL_CU(cudaEventCreate(&e));
      LL_CU(cudaEventRecordWithFlags(e, H->s, cudaEventRecordExternal));
      H->gpairs[H->capturing].push_back({kind, b, e, flops, bytes, nl});
    } else {
      cudaEvent_t e = H->event();
      LL_CU(cudaEventRecord(e, H->s));
      H->prof_pairs[kind].push_back({b, e});
      H->prof_n[kind] += nl;
    }
  }
};

// make the library stream wait for the work already queued on the caller's
void enter(ll_mg_hierarchy* H) {
  LL_CU(cudaEventRecord(H->entry_ev, H->user));
  LL_CU(cudaStreamWaitEvent(H->s, H->entry_ev, 0));
}
#define LL_PROF(kind) ProfScope prof_scope_(H, kind)
#define LL_PROFW(kind, flops, bytes) ProfScope prof_scope_(H, kind, flops, bytes)
#define LL_PROFN(kind, flops, bytes, n) ProfScope prof_scope_(H, kind, flops, bytes, n)

// launch on the library stream, counted
template <typename... KP, typename... A>
void launch_k(ll_mg_hierarchy* H, void (*k)(KP...), long grid, int block, A... args) {
  k<<<(unsigned)grid, block, 0, H->s>>>(args...);
  LL_LAUNCHED();
}
// as launch_k, as a programmatic dependent of the kernel before it: the
// kernel may start while that one finishes, and waits for it
// (griddepcontrol.wait) before it reads what that kernel wrote
template <typename... KP, typename... A>
void launch_pdl(ll_mg_hierarchy* H, void (*k)(KP...), long grid, int block, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(block);
  cfg.stream = H->s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  LL_CU(cudaLaunchKernelEx(&cfg, k, ((KP)args)...));
  LL_LAUNCHED();
}

// lanes per block row in the per-class BSR kernels.  The float64 sweeps are
// bound by the float64 pipe, where idle lanes cost issue slots, so 4 lanes
// keep short rows busy; the float32 sweeps are latency-bound, and 8 lanes
// halve each row's chain of dependent loads (measured: -19 % sweep time).
template <typename T> constexpr int lanes();
template <> constexpr int lanes<double>() { return kRowLanes; }
template <> constexpr int lanes<float>() { return 2 * kRowLanes; }
// A launch over fewer rows than this fills only part of the GPU and lasts as
// long as one row's chain of dependent loads; 8 lanes per row then halve the
// chain in float64 too (issue slots are not the limit there).
constexpr int kWideLaneRows = 20000;
// SELL-32 sweeps: float64 levels whose average colour class has at least
// kSellLevelClass rows keep a SELL-32 copy, and their classes of at least
// kSellMinRows rows sweep on it with 1, 2 or 4 lanes per row (sell_lanes)
constexpr int kSellLevelClass = 20000;
constexpr int kSellMinRows = 20000;
constexpr int kSellRows1 = 40000, kSellRows2 = 8000;
constexpr int kSellBlock = 128;
constexpr int kSellUnroll = 2;
// lanes per row of a SELL-32 sweep of a class of `rows` rows: few lanes keep
// the float64 pipe busy with useful multiply-adds (no idle slots, no group
// sum); more lanes shorten each row's chain where the class is too small to
// fill the GPU with one-lane rows
template <int MODE>
int sell_lanes(long rows) {
  if (rows >= kSellRows1) return MODE == 0 ? 1 : 2;
  if (rows >= kSellRows2) return 2;
  return 4;
}
template <typename T>
bool wide_lanes(long rows) {
  return lanes<T>() >= 8 || rows < kWideLaneRows;
}
constexpr int kDotChunk = 8;
constexpr int kGalerkinSortBlocks = 200000;  // float64 Galerkin levels >= 2 with this many blocks: ordered threads
// Coarse-level kernels use small blocks: a colour class of a small level then
// spreads over many SMs instead of queueing on the float64 units of one.
constexpr int kCoarseBlock = 64;
// tail levels with at most this many cells run on one CTA (see k_coarse_tail);
// float32 ones up to 500 (the 467-cell level 6 of the 128^3 hierarchy: mixed
// tail -3 %, while float64 phases on one SM's float64 pipe took +8 %)
template <typename T> constexpr int kSoloCells = 200;
template <> constexpr int kSoloCells<float> = 500;
constexpr int kTailCells = 5000;  // levels at or below this size run in the cluster tail
constexpr int kMaxCoarsestCells = 2048;

void check_flag(ll_mg_hierarchy* H, int code) {
  int v = 0;
  LL_CU(cudaMemcpyAsync(&v, H->flag.p, sizeof(int), cudaMemcpyDeviceToHost, H->s));
  LL_CU(cudaStreamSynchronize(H->s));
  if (v) throw Status{code};
}

// SELL-32 pattern of a level from its BSR pattern (see ks_sweep): chunk
// widths, their offsets, the chunk of each slot group, the slots' columns
void sell_build(CLevel& C, cudaStream_t s) {
  int nch = cdiv(C.n, kSell);
  DBuf<int> w;
  w.alloc(nch);
  k_sell_width<<<cdiv(nch, kBlock), kBlock, 0, s>>>(C.n, C.rowptr, w);
  LL_LAUNCHED();
  C.soff.alloc(nch + 1);
  C.sgroups = exclusive_scan(w, C.soff, nch, s);
  C.sgc.alloc(C.sgroups);
  k_sell_groups<<<cdiv(nch, kBlock), kBlock, 0, s>>>(nch, C.soff, C.sgc);
  LL_LAUNCHED();
  C.scol.alloc(C.sgroups * kSell);
  if (C.sgroups > 0) {
    k_sell_cols<<<cdiv(C.sgroups * kSell, kBlock), kBlock, 0, s>>>(C.sgroups, C.n, C.sgc, C.soff, C.rowptr, C.diag,
                                                                   C.col, C.scol);
    LL_LAUNCHED();
  }
  LL_CU(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// symbolic setup (once per grid): aggregation, patterns, colours, slot maps
// ---------------------------------------------------------------------------
void symbolic(ll_mg_hierarchy* H) {
  cudaStream_t s = H->s;
  const GridGeom& g = H->g;
  const ll_mg_params& p = H->prm;
  build_grid_graph(g.nx, g.ny, g.nz, H->graph0, s);
  H->nlev = 1;
  const DevGraph* cur = &H->graph0;
  int ncur = (int)g.n;
  // aggregation and colouring in the aggregation's own numbering
  while (ncur > p.coarsest_cells && H->nlev < p.max_levels) {
    int l = H->nlev - 1;
    DBuf<int>& agg = l == 0 ? H->agg_nat0 : H->lev[l].agg_orig;
    agg.alloc(ncur);
    int nc = aggregate_level(*cur, p.rounds, p.seed, agg, s);
    if (3L * nc > 2L * ncur) {  // coarsening ratio below 1.5: stop here
      agg.release();
      break;
    }
    CLevel& C = H->lev[l + 1];
    C.n = nc;
    {
      DBuf<int> mptr, mem;
      build_members(ncur, agg, nc, mptr, mem, s);
      contract_graph(*cur, agg, nc, mptr, mem, C.graph, s);
    }
    C.colour.alloc(nc);
    C.ncol = colour_graph(C.graph, p.seed, C.colour, s);
    if (C.ncol < 0) throw Status{LL_ELIMIT};
    // the SELL-32 sweeps where the average colour class is large
    C.sell = H->sell_ok && (long)nc >= (long)kSellLevelClass * C.ncol;
    {
      DBuf<int> cptr, key;
      row_work_keys(C.graph, C.colour, C.sell, key, s);
      colour_classes(nc, C.colour, C.ncol, key, C.sell ? kRowKeysExact : kRowKeys, cptr, C.n2o, C.cs, s);
    }
    C.o2n.alloc(nc);
    invert_perm(nc, C.n2o, C.o2n, s);
    H->nlev++;
    cur = &C.graph;
    ncur = nc;
  }
  int ncoarse = H->nlev == 1 ? (int)g.n : H->lev[H->nlev - 1].n;
  if (ncoarse > kMaxCoarsestCells) throw Status{LL_ELIMIT};
  H->nat_of_slot.alloc(H->n2);
  if (H->nlev == 1) {
    rb_maps(g, nullptr, nullptr, H->nat_of_slot, s);
    LL_CU(cudaStreamSynchronize(s));
    return;
  }
  // operators, transfers and slot maps in the colour-class numbering
  for (int l = 1; l < H->nlev; ++l) {
    CLevel& C = H->lev[l];
    DevGraph gn;
    permute_graph(C.graph, C.n2o, C.o2n, gn, s);
    bsr_pattern(gn, C.rowptr, C.col, C.diag, C.nnzb, s);
    C.prow.alloc(C.nnzb);
    k_block_rows<<<cdiv(C.n, kBlock), kBlock, 0, s>>>(C.n, C.rowptr, C.prow);
    LL_LAUNCHED();
    LL_CU(cudaStreamSynchronize(s));
  }
  CLevel& L1 = H->lev[1];
  {
    DBuf<int> agg_rb_orig, agg_nat_new;
    agg_rb_orig.alloc(H->n2);
    rb_maps(g, H->agg_nat0, agg_rb_orig, H->nat_of_slot, s);
    H->agg0.alloc(H->n2);
    map_through((int)H->n2, nullptr, agg_rb_orig, L1.o2n, H->agg0, s);
    agg_nat_new.alloc(g.n);
    map_through((int)g.n, nullptr, H->agg_nat0, L1.o2n, agg_nat_new, s);
    slot_map_level1(g, agg_nat_new, L1.graph, L1.rowptr, L1.col, L1.nnzb, L1.sptr, L1.sidx, L1.sw, s);
  }
  build_members((int)H->n2, H->agg0, L1.n, L1.mptr, L1.mem, s);  // red-black slots
  members_colour0(L1.n, L1.mptr, L1.mem, g.nh, L1.mptr0, L1.mem0, s);
  for (int l = 1; l + 1 < H->nlev; ++l) {
    CLevel& F = H->lev[l];
    CLevel& C = H->lev[l + 1];
    F.agg.alloc(F.n);
    map_through(F.n, F.n2o, F.agg_orig, C.o2n, F.agg, s);
    build_members(F.n, F.agg, C.n, C.mptr, C.mem, s);
    slot_map_bsr(F.n, F.rowptr, F.col, F.agg, C.rowptr, C.col, C.nnzb, C.sptr, C.sidx, s);
  }
  // float64 Galerkin products of the large levels >= 2 by slot-list length
  // (level 2 at 128^3: 0.64 -> 0.35 ms); level 1 and the small levels keep
  // the row order, whose loads share cache lines (level 1 sorted: 0.67 ->
  // 1.01 ms), and so do float32 products, whose divergence costs little
  if (H->prm.precision == LL_FP64)
    for (int l = 2; l < H->nlev; ++l)
      if (H->lev[l].nnzb >= kGalerkinSortBlocks)
        order_by_length(H->lev[l].nnzb, H->lev[l].sptr, H->lev[l].gperm, s);
  for (int l = 1; l < H->nlev; ++l)
    if (H->lev[l].sell) sell_build(H->lev[l], s);
  LL_CU(cudaStreamSynchronize(s));
}

void allocate(ll_mg_hierarchy* H) {
  bool mixed = H->prm.precision != LL_FP64;  // float32 V-cycle
  long n2 = H->n2;
  H->chat64.alloc(9 * n2);
  if (mixed) {
    H->chat32.alloc(9 * n2);
    H->chatlo.alloc(9 * n2);
    H->dinv32.alloc(9 * n2);
    H->m32.alloc(3 * n2);
  } else {
    H->dinv64.alloc(9 * n2);
    if (H->nlev > 1) H->r0tmp64.alloc(3 * H->g.nh);
  }
  for (int l = 1; l < H->nlev; ++l) {
    CLevel& C = H->lev[l];
    if (mixed) {  // float32 Galerkin levels (bfloat16 copies of them for LL_MIXED_BF16)
      C.val32.alloc(9L * C.nnzb);
      if (H->prm.precision == LL_MIXED_BF16) C.val16.alloc(9L * C.nnzb);
      C.dinv32.alloc(9L * C.n);
      C.x32.alloc(3L * C.n);
      C.b32.alloc(3L * C.n);
      C.r32.alloc(3L * C.n);
    } else {
      C.val64.alloc(9L * C.nnzb);
      C.dinv64.alloc(9L * C.n);
      C.x64.alloc(3L * C.n);
      C.b64.alloc(3L * C.n);
      C.r64.alloc(3L * C.n);
      if (C.sell) C.sval.alloc(9L * kSell * C.sgroups);
    }
  }
  for (int l = 1; l < H->nlev - 1 && l <= H->prm.kcycle; ++l)
    for (int q = 0; q < 4; ++q) {
      if (mixed) H->lev[l].k32[q].alloc(3L * H->lev[l].n);
      else H->lev[l].k64[q].alloc(3L * H->lev[l].n);
    }
  H->kscal.alloc(8 * kMaxLevels);
  int nc = H->nlev == 1 ? (int)H->g.n : H->lev[H->nlev - 1].n;
  H->ncoarse3 = 3 * nc;
  H->lu.alloc((size_t)H->ncoarse3 * H->ncoarse3);
  H->ainv.alloc((size_t)H->ncoarse3 * H->ncoarse3);
  H->perm.alloc(H->ncoarse3);
  H->lu_status.alloc(1);
  H->flag.alloc(1);
  int m = H->prm.restart;
  long n3 = H->n3;
  if (mixed) {
    H->Z32.alloc((size_t)m * n3);
  } else {
    H->Z64.alloc((size_t)m * n3);
  }
  H->C.alloc((size_t)m * n3);
  H->r.alloc(n3);
  H->xw.alloc(n3);
  H->bw.alloc(n3);
  H->partial.alloc((size_t)(kMaxRestart + 2) * kRedBlocks);
  H->scal.alloc(1);
  H->scal.zero(H->s);
  LL_CU(cudaMallocHost((void**)&H->h_head, 8 * sizeof(double)));
  H->stepb.alloc(3 * H->g.n);
  H->stepx.alloc(3 * H->g.n);
  if (H->nlev == 1) {
    H->single_b.alloc(H->ncoarse3);
    H->single_x.alloc(H->ncoarse3);
  }
}

// algorithmic work of coarse sweeps and residuals (the models in ll_mg.h)
inline double sweep_flops(long long blocks, long long rows) { return 18.0 * blocks + 15.0 * rows; }
inline double sweep_bytes(long long blocks, long long rows, int w, int wm) {
  return (9.0 * wm + 3.0 * w + 4) * blocks + (15.0 * w + 8) * rows;
}

template <typename T, typename TM>
void fill_tail(ll_mg_hierarchy* H, DBuf<TailArgs<T, TM>>& dst) {
  TailArgs<T, TM> A;
  A.first = H->tail_first;
  A.last = H->nlev - 1;
  A.solo_first = A.last;  // the coarsest level at least
  while (A.solo_first > A.first && H->lev[A.solo_first - 1].n <= kSoloCells<T>) --A.solo_first;
  A.nu_pre = H->prm.nu_pre;
  A.nu_post = H->prm.nu_post;
  A.uni = H->union_mode;
  A.N = H->union_mode ? 0 : H->ncoarse3;
  A.ainv = H->union_mode ? nullptr : H->ainv.p;
  for (int l = A.first; l <= A.last; ++l) {
    CLevel& C = H->lev[l];
    TailLevel<T, TM>& L = A.L[l];
    L.n = C.n;
    L.ncol = C.ncol;
    L.nnzb = C.nnzb;
    L.nmem = l > A.first ? (int)C.mem.n : 0;
    for (int c = 0; c <= C.ncol && c <= kTailMaxColours; ++c) L.cs[c] = C.cs[c];
    L.rowptr = C.rowptr;
    L.diag = C.diag;
    L.col = C.col;
    L.val = C.valm<TM>();
    L.dinv = C.dinv<T>();
    L.x = C.x<T>();
    L.b = C.b<T>();
    L.r = C.r<T>();
    L.agg = C.agg;
    L.mptr = C.mptr;
    L.mem = C.mem;
    if (H->union_mode) {
      L.nuc = H->uc_n[l];
      L.uc = H->uc_tasks[l];
      L.ucptr = H->uc_ptr[l];
    }
  }
  int w = (int)sizeof(T), wm = (int)sizeof(TM);
  H->tail_flops = H->tail_bytes = 0;
  for (int l = A.first; l < A.last; ++l) {
    CLevel& C = H->lev[l];
    for (int c = 0; c < C.ncol; ++c) {
      long long rows = C.cs[c + 1] - C.cs[c];
      if (c > 0) {
        H->tail_flops += sweep_flops(C.pre_blk[c], rows);
        H->tail_bytes += sweep_bytes(C.pre_blk[c], rows, w, wm);
      }
      H->tail_flops += sweep_flops(C.off_blk[c], rows);
      H->tail_bytes += sweep_bytes(C.off_blk[c], rows, w, wm);
    }
    long long rrows = C.ncol > 0 ? C.cs[C.ncol - 1] : 0;
    H->tail_flops += sweep_flops(C.res_blk, rrows);
    H->tail_bytes += sweep_bytes(C.res_blk, rrows, w, wm);
  }
  H->tail_flops += 2.0 * H->ncoarse3 * H->ncoarse3;  // zero for a union (its dense solves are not counted)
  H->tail_bytes += 8.0 * H->ncoarse3 * H->ncoarse3;
  dst.alloc(1);
  LL_CU(cudaMemcpyAsync(dst.p, &A, sizeof(A), cudaMemcpyHostToDevice, H->s));
  LL_CU(cudaStreamSynchronize(H->s));
}

// Decide whether the small coarse levels run as one cluster kernel: the
// cluster must be schedulable (16 CTAs, else 8) and every tail level must
// have at most kTailMaxColours colours.
template <typename T, typename TM>
void setup_tail_for(ll_mg_hierarchy* H) {
  auto kern = k_coarse_tail<T, TM, 4>;
  for (int cl : {16, 8}) {
    if (cl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cl;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0) {
      H->tail_cluster = cl;
      break;
    }
    cudaGetLastError();
  }
  if (H->tail_cluster == 0) {
    H->tail_first = -1;
    return;
  }
  fill_tail<T, TM>(H, H->tail<T, TM>());
}

// host counts behind the algorithmic flop and byte models of the kernels
void setup_counts(ll_mg_hierarchy* H) {
  const GridGeom& g = H->g;
  for (long row = 0; row < (long)g.ny * g.nz; ++row) {
    int y = (int)(row % g.ny), z = (int)(row / g.ny);
    for (int c = 0; c < 2; ++c) H->l0_cells[c] += (g.nx - ((c + y + z) & 1) + 1) / 2;
  }
  for (int l = 1; l < H->nlev; ++l) {
    CLevel& C = H->lev[l];
    std::vector<int> rp(C.n + 1), dg(C.n);
    LL_CU(cudaMemcpy(rp.data(), C.rowptr.p, (C.n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    LL_CU(cudaMemcpy(dg.data(), C.diag.p, C.n * sizeof(int), cudaMemcpyDeviceToHost));
    C.pre_blk.assign(C.ncol, 0);
    C.off_blk.assign(C.ncol, 0);
    for (int c = 0; c < C.ncol; ++c)
      for (int I = C.cs[c]; I < C.cs[c + 1]; ++I) {
        C.pre_blk[c] += dg[I] - rp[I];
        C.off_blk[c] += rp[I + 1] - rp[I] - 1;
      }
    C.res_blk = 0;  // blocks the residual reads (one forward sweep: the higher colours' only)
    for (int I = 0; I < (C.ncol > 0 ? C.cs[C.ncol - 1] : 0); ++I)
      C.res_blk += H->prm.nu_pre == 1 ? rp[I + 1] - dg[I] - 1 : rp[I + 1] - rp[I];
  }
}

void setup_tail(ll_mg_hierarchy* H) {
  H->tail_first = -1;
  const char* nt = getenv("LLMG_NO_TAIL");
  if ((nt && nt[0] == '1') || H->nlev < 2) return;
  for (int l = 1; l < H->nlev; ++l)
    if (H->lev[l].n <= kTailCells) {
      H->tail_first = l;
      break;
    }
  if (H->tail_first >= 0 && H->tail_first <= H->prm.kcycle) H->tail_first = H->prm.kcycle + 1;  // K levels stay out
  if (H->tail_first < 0 || H->tail_first >= H->nlev) {
    H->tail_first = -1;
    return;
  }
  for (int l = H->tail_first; l < H->nlev; ++l)
    if (H->lev[l].ncol > kTailMaxColours) {
      H->tail_first = -1;
      return;
    }
  if (H->prm.precision == LL_MIXED_BF16) setup_tail_for<float, __nv_bfloat16>(H);
  else if (H->prm.precision == LL_MIXED_FP32) setup_tail_for<float, float>(H);
  else setup_tail_for<double, double>(H);
}

template <typename T, typename TM>
void launch_tail(ll_mg_hierarchy* H) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(H->tail_cluster);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = H->s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = H->tail_cluster;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  LL_CU(cudaLaunchKernelEx(&cfg, k_coarse_tail<T, TM, 4>, (const TailArgs<T, TM>*)H->tail<T, TM>().p));
  count_launch();
}

// Float64 FMA throughput probe: kProbeChains independent multiply-add chains
// per thread (enough in flight to cover the float64 pipe's latency), no
// memory traffic; the sum is stored only under a condition the compiler
// cannot decide, so the chains are not removed.
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(double* sink, long long iters) {
  double a[kProbeChains];
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) a[q] = 1e-3 * (threadIdx.x + q);
  const double mul = 0.9999999, add = 1e-9;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = fma(a[q], mul, add);
  }
  double t = 0;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) t += a[q];
  if (t == -1.0) sink[0] = t;
}

// dense level-0 operator (single-level hierarchies), unknown 3k + c, k natural
__global__ void k_dense_from_l0(GridGeom g, const double* __restrict__ chat64, double inv_dt,
                                double* __restrict__ a) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  long N = 3 * g.n;
  int x = (int)(k % g.nx);
  long t = k / g.nx;
  int y = (int)(t % g.ny), z = (int)(t / g.ny);
  int c = (x + y + z) & 1;
  long sl = c * g.nh + ((long)z * g.ny + y) * g.nxh + (x >> 1);
  long n2 = 2 * g.nh;
  double C[9];
  for (int e = 0; e < 9; ++e) C[e] = chat64[e * n2 + sl];
  for (int r = 0; r < 3; ++r)
    for (long j = 0; j < N; ++j) a[(3 * k + r) * N + j] = 0.0;
  long nb[6];
  int d = 0;
  if (z > 0) nb[d++] = k - (long)g.nx * g.ny;
  if (y > 0) nb[d++] = k - g.nx;
  if (x > 0) nb[d++] = k - 1;
  if (x < g.nx - 1) nb[d++] = k + 1;
  if (y < g.ny - 1) nb[d++] = k + g.nx;
  if (z < g.nz - 1) nb[d++] = k + (long)g.nx * g.ny;
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc) {
      a[(3 * k + r) * N + 3 * k + cc] = -d * C[3 * r + cc] + (r == cc ? inv_dt : 0.0);
      for (int q = 0; q < d; ++q) a[(3 * k + r) * N + 3 * nb[q] + cc] = C[3 * r + cc];
    }
}

// red-black SoA <-> cell-major natural vector (single-level hierarchies)
template <typename TI, typename TO>
__global__ void k_rb_to_cellmajor(GridGeom g, const int* __restrict__ nat, const TI* __restrict__ in,
                                  TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2 || nat[sl] < 0) return;
  long k = nat[sl];
  for (int c = 0; c < 3; ++c) out[3 * k + c] = (TO)in[c * n2 + sl];
}
template <typename TI, typename TO>
__global__ void k_cellmajor_to_rb(GridGeom g, const int* __restrict__ nat, const TI* __restrict__ in,
                                  TO* __restrict__ out) {
  long sl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n2 = 2 * g.nh;
  if (sl >= n2) return;
  long k = nat[sl];
  for (int c = 0; c < 3; ++c) out[c * n2 + sl] = k < 0 ? (TO)0 : (TO)in[3 * k + c];
}

// ---------------------------------------------------------------------------
// numeric setup (every time step)
// ---------------------------------------------------------------------------
// Numeric setup for m~ = m (coefficients, Galerkin levels, coarsest inverse),
// queued on the hierarchy's stream without waiting; numeric_check() then
// reads the two failure flags.  A batch queues every instance first.
void numeric_launch(ll_mg_hierarchy* H, const double* m) {
  LL_PROF(LL_KIND_NUMERIC);
  cudaStream_t s = H->s;
  const GridGeom& g = H->g;
  bool mixed = H->prm.precision != LL_FP64;  // float32 V-cycle
  H->flag.zero(s);
  double ih2 = 1.0 / (H->h * H->h), inv_dt = 1.0 / H->dt;
  int nb = cdiv(H->n2, kBlock);
  if (mixed)
    k0_coef<float><<<nb, kBlock, 0, s>>>(g, m, H->alpha, H->dt, ih2, H->chat64, H->chat32, H->dinv32, H->flag,
                                         H->m32, H->chatlo);
  else
    k0_coef<double><<<nb, kBlock, 0, s>>>(g, m, H->alpha, H->dt, ih2, H->chat64, nullptr, H->dinv64, H->flag);
  LL_LAUNCHED();
  for (int l = 1; l < H->nlev; ++l) {
    CLevel& C = H->lev[l];
    int nb = cdiv(C.nnzb, 128);
    if (mixed) {  // the float32 preconditioner's levels in float32 from chat32
      if (l == 1)
        k_galerkin_l1_blk<float><<<nb, 128, 0, s>>>(C.nnzb, C.gperm, C.prow, C.col, C.sptr, C.sidx, C.sw, C.mptr,
                                                    H->n2, H->chat32, (float)inv_dt, C.val32);
      else
        k_galerkin_bsr_blk<float><<<nb, 128, 0, s>>>(C.nnzb, C.gperm, C.sptr, C.sidx, H->lev[l - 1].val32, C.val32);
      LL_LAUNCHED();
      k_block_dinv<float><<<cdiv(C.n, 128), 128, 0, s>>>(C.n, C.diag, C.val32, C.dinv32, H->flag);
      LL_LAUNCHED();
      if (H->prm.precision == LL_MIXED_BF16) {
        k_cast_bf16<<<cdiv(9L * C.nnzb, kBlock), kBlock, 0, s>>>(9L * C.nnzb, C.val32, C.val16);
        LL_LAUNCHED();
      }
      continue;
    }
    if (l == 1)
      k_galerkin_l1_blk<double><<<nb, 128, 0, s>>>(C.nnzb, C.gperm, C.prow, C.col, C.sptr, C.sidx, C.sw, C.mptr,
                                                   H->n2, H->chat64, inv_dt, C.val64);
    else
      k_galerkin_bsr_blk<double><<<nb, 128, 0, s>>>(C.nnzb, C.gperm, C.sptr, C.sidx, H->lev[l - 1].val64, C.val64);
    LL_LAUNCHED();
    k_block_dinv<double><<<cdiv(C.n, 128), 128, 0, s>>>(C.n, C.diag, C.val64, C.dinv64, H->flag);
    LL_LAUNCHED();
    if (C.sell && C.sgroups > 0) {
      k_sell_values<<<cdiv(C.sgroups * kSell, kBlock), kBlock, 0, s>>>(C.sgroups, C.n, C.sgc, C.soff, C.rowptr,
                                                                        C.diag, C.val64, C.sval);
      LL_LAUNCHED();
    }
  }
  // coarsest dense LU
  int N = H->ncoarse3;
  if (H->nlev == 1) {
    k_dense_from_l0<<<cdiv(g.n, 64), 64, 0, s>>>(g, H->chat64, inv_dt, H->lu);
  } else {
    CLevel& C = H->lev[H->nlev - 1];
    if (mixed)
      k_dense_from_bsr<float><<<cdiv(C.n, 64), 64, 0, s>>>(C.n, C.rowptr, C.col, C.val32, H->lu);
    else
      k_dense_from_bsr<double><<<cdiv(C.n, 64), 64, 0, s>>>(C.n, C.rowptr, C.col, C.val64, H->lu);
  }
  LL_LAUNCHED();
  if (N <= kGjMax) {  // Gauss-Jordan on one cluster, the columns spread over its CTAs
    // 16 CTAs where a cluster of that size can be scheduled, else 8
    auto config = [&](int P, cudaLaunchConfig_t& cfg, cudaLaunchAttribute& at) {
      int W = cdiv(N, P);
      cfg = {};
      cfg.gridDim = dim3(P);
      cfg.blockDim = dim3(32 * W);
      cfg.dynamicSmemBytes = sizeof(double) * ((size_t)W * N + 2 * (N + 1));
      cfg.stream = s;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = P;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
    };
    // The kernel's dynamic shared-memory limit is one value for the whole
    // process, set to what the largest case (N = kGjMax on 8 CTAs) needs:
    // hierarchies of several host threads (the groups of a batch) set it
    // concurrently, and a per-N value could be lowered by another thread
    // between its setting and this thread's launch.
    constexpr int kGjSmemMax = (int)sizeof(double) * ((kGjMax / 8) * kGjMax + 2 * (kGjMax + 1));
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at;
    if (H->gj_cluster == 0) {
      H->gj_cluster = 8;
      config(16, cfg, at);
      int nclusters = 0;
      if (cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
          cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, kGjSmemMax) ==
              cudaSuccess &&
          cudaOccupancyMaxActiveClusters(&nclusters, k_gj_inverse, &cfg) == cudaSuccess && nclusters > 0)
        H->gj_cluster = 16;
      cudaGetLastError();
    }
    config(H->gj_cluster, cfg, at);
    LL_CU(cudaFuncSetAttribute(k_gj_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, kGjSmemMax));
    LL_CU(cudaLaunchKernelEx(&cfg, k_gj_inverse, N, (const double*)H->lu.p, H->ainv.p, H->lu_status.p));
    LL_LAUNCHED();
  } else {
    k_lu_factor<<<1, 1024, 0, s>>>(N, H->lu, H->perm, H->lu_status);
    LL_LAUNCHED();
    k_lu_inverse<<<cdiv(N, 128), 128, 0, s>>>(N, H->lu, H->perm, H->ainv);
    LL_LAUNCHED();
  }
}

// singular diagonal block (level 0 or a Galerkin level) or singular coarsest
// matrix: LL_SINGULAR_COARSE
void numeric_check(ll_mg_hierarchy* H) {
  int v[2] = {0, 0};
  LL_CU(cudaMemcpyAsync(&v[0], H->flag.p, sizeof(int), cudaMemcpyDeviceToHost, H->s));
  LL_CU(cudaMemcpyAsync(&v[1], H->lu_status.p, sizeof(int), cudaMemcpyDeviceToHost, H->s));
  LL_CU(cudaStreamSynchronize(H->s));
  if (v[0] || v[1]) throw Status{LL_SINGULAR_COARSE};
}

void numeric(ll_mg_hierarchy* H, const double* m) {
  numeric_launch(H, m);
  numeric_check(H);
}

// ---------------------------------------------------------------------------
// V-cycle (Sec. 3): pre-smoothing, residual, restriction, coarse correction,
// prolongation, post-smoothing; x = 0 initially on every level
// ---------------------------------------------------------------------------
template <typename T>
void coarse_solve(ll_mg_hierarchy* H, const T* b, T* x) {
  int N = H->ncoarse3;
  LL_PROFW(LL_KIND_COARSEST, 2.0 * N * N, 8.0 * N * N);
  kc_solve<T><<<cdiv(N, 32), 32, N * sizeof(double), H->s>>>(N, H->ainv, b, x);
  LL_LAUNCHED();
}

// Launch shape of the per-class coarse kernels: the parameters' coarse_lanes
// and coarse_block when set (the batch autotuner's choice), else the
// defaults above.
inline int coarse_block(const ll_mg_hierarchy* H) {
  return H->prm.coarse_block > 0 ? H->prm.coarse_block : kCoarseBlock;
}
template <typename T>
int sweep_lanes(const ll_mg_hierarchy* H, long rows) {
  return H->prm.coarse_lanes > 0 ? H->prm.coarse_lanes : (wide_lanes<T>(rows) ? 8 : kRowLanes);
}
template <typename T>
int residual_lanes(const ll_mg_hierarchy* H) {
  return H->prm.coarse_lanes > 0 ? H->prm.coarse_lanes : lanes<T>();
}

// one colour class of level l: rows [cs[t], cs[t+1])
// work model of one class sweep
template <typename T, typename TM, int MODE>
void class_work(const CLevel& L, int t, double& flops, double& bytes) {
  int rows = L.cs[t + 1] - L.cs[t];
  long long blk = MODE == 0 ? L.pre_blk[t] : L.off_blk[t];
  flops += rows > 0 ? sweep_flops(blk, rows) : 0.0;
  bytes += rows > 0 ? sweep_bytes(blk, rows, (int)sizeof(T), (int)sizeof(TM)) : 0.0;
}

// one colour class of level l: rows [cs[t], cs[t+1]); timed on its own
// unless the caller times a group of classes (timed = false)
template <typename T, typename TM, int MODE>
void sweep_class(ll_mg_hierarchy* H, int l, int t, bool timed = true) {
  CLevel& L = H->lev[l];
  int r0 = L.cs[t], r1 = L.cs[t + 1];
  if (r1 <= r0) return;
  double f = 0, by = 0;
  if (timed) class_work<T, TM, MODE>(L, t, f, by);
  ProfScope prof_scope_(H, timed ? LL_KIND_BSR_SMOOTH : LL_NUM_KINDS, f, by);
  if constexpr (std::is_same<T, double>::value && std::is_same<TM, double>::value) {
    if (L.sell && r1 - r0 >= kSellMinRows) {  // on the SELL-32 copy
      long rows = cdiv((long)(r1 - (r0 & ~(kSell - 1))), kSell) * kSell;  // whole chunks
      auto go = [&](auto kern, int G) {
        launch_k(H, kern, cdiv(rows * G, kSellBlock), kSellBlock, r0, r1, (const int*)L.rowptr, (const int*)L.diag,
                 (const int*)L.soff, (const int*)L.scol, (const double*)L.sval, (const double*)L.dinv64,
                 (const double*)L.b64, L.x64.p);
      };
      switch (sell_lanes<MODE>(r1 - r0)) {
        case 1: go(ks_sweep<MODE, 1, kSellUnroll>, 1); break;
        case 2: go(ks_sweep<MODE, 2, kSellUnroll>, 2); break;
        default: go(ks_sweep<MODE, 4, kSellUnroll>, 4); break;
      }
      return;
    }
  }
  int blk = coarse_block(H);
  // the float32 sweeps overlap their start with the kernel before them (PDL);
  // measured: float32 step -1.8 %, float64 no gain (its large classes are
  // bound by the float64 pipe)
  constexpr bool pdl = std::is_same<T, float>::value;
  auto go = [&](auto kern, int G) {
    if (pdl)
      launch_pdl(H, kern, cdiv((long)(r1 - r0) * G, blk), blk, r0, r1, (const int*)L.rowptr, (const int*)L.diag,
                 (const int*)L.col, (const TM*)L.valm<TM>(), (const T*)L.dinv<T>(), (const T*)L.b<T>(), L.x<T>());
    else
      launch_k(H, kern, cdiv((long)(r1 - r0) * G, blk), blk, r0, r1, (const int*)L.rowptr, (const int*)L.diag,
               (const int*)L.col, (const TM*)L.valm<TM>(), (const T*)L.dinv<T>(), (const T*)L.b<T>(), L.x<T>());
  };
  if (sweep_lanes<T>(H, r1 - r0) == 8) go(kb_sweep<T, TM, 8, MODE, pdl>, 8);
  else go(kb_sweep<T, TM, kRowLanes, MODE, pdl>, kRowLanes);
}

// one full plain block-GS sweep of level l (colours ascending or descending)
template <typename T, typename TM>
void smooth_level(ll_mg_hierarchy* H, int l, bool forward) {
  CLevel& L = H->lev[l];
  for (int k = 0; k < L.ncol; ++k) sweep_class<T, TM, 1>(H, l, forward ? k : L.ncol - 1 - k);
}

// V-cycle below level 0.  On entry b_l holds the restricted residual and,
// when pre-smoothing is on, x_l already holds the colour-0 rows of the first
// forward sweep (written by the restriction into this level).
template <typename T, typename TM>
void vcycle_coarse(ll_mg_hierarchy* H, int l, bool init0_done = true);

// The coarse problem of level l (a K level): two GCR steps from zero,
// preconditioned by the cycle of level l (the same formulas as the oracle's
// K-cycle).  On entry L.b holds the restricted residual r and x holds the
// first colour of the first forward sweep; on exit L.x is the correction.
template <typename T, typename TM>
void kinner(ll_mg_hierarchy* H, int l) {
  CLevel& L = H->lev[l];
  cudaStream_t s = H->s;
  long n3 = 3L * L.n;
  int nb = cdiv(n3, kBlock), nbs = cdiv((long)L.n * lanes<T>(), kCoarseBlock);
  double* ks = H->kscal.p + 8 * l;
  T *kr = L.kv<T>(0), *kz1 = L.kv<T>(1), *kc1 = L.kv<T>(2), *kc2 = L.kv<T>(3);
  double kflops = 18.0 * L.nnzb + 8.0 * n3, kbytes = (double)L.nnzb * (9 * sizeof(TM) + 4 + 3 * sizeof(T)) + 4.0 * n3 * sizeof(T);
  {
    LL_PROFW(LL_KIND_BSR_OTHER, 0.0, 2.0 * n3 * sizeof(T));
    LL_CU(cudaMemcpyAsync(kr, L.b<T>(), n3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  vcycle_coarse<T, TM>(H, l, true);  // z1 = B r
  {  // c1 = A z1; d11 = c1.c1, d1r = c1.r; r1 = r - (d1r/d11) c1 (into L.b)
    LL_PROFW(LL_KIND_BSR_OTHER, kflops, kbytes);
    LL_CU(cudaMemcpyAsync(kz1, L.x<T>(), n3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    kb_spmv<T, TM, lanes<T>()><<<nbs, kCoarseBlock, 0, s>>>(L.n, L.rowptr, L.col, L.valm<TM>(), kz1, kc1);
    LL_LAUNCHED();
    kd_dots<T, 2><<<kRedBlocks, kBlock, 0, s>>>(n3, kc1, kc1, kc1, kr, H->partial);
    LL_LAUNCHED();
    k_finish<<<2, kBlock, 0, s>>>(H->partial, ks);
    LL_LAUNCHED();
    kk_axpy<T><<<nb, kBlock, 0, s>>>(n3, kr, kc1, ks, 1, 0, L.b<T>());
    LL_LAUNCHED();
  }
  vcycle_coarse<T, TM>(H, l, false);  // z2 = B r1 (in L.x)
  {  // c2 = A z2 - (d12/d11) c1; d22 = c2.c2, d2r = c2.r1; x = y1 z1 + y2 z2
    LL_PROFW(LL_KIND_BSR_OTHER, kflops + 4.0 * n3, kbytes + 3.0 * n3 * sizeof(T));
    kb_spmv<T, TM, lanes<T>()><<<nbs, kCoarseBlock, 0, s>>>(L.n, L.rowptr, L.col, L.valm<TM>(), L.x<T>(), kc2);
    LL_LAUNCHED();
    kd_dots<T, 1><<<kRedBlocks, kBlock, 0, s>>>(n3, kc1, kc2, nullptr, nullptr, H->partial);
    LL_LAUNCHED();
    k_finish<<<1, kBlock, 0, s>>>(H->partial, ks + 2);
    LL_LAUNCHED();
    kk_axpy<T><<<nb, kBlock, 0, s>>>(n3, kc2, kc1, ks, 2, 0, kc2);
    LL_LAUNCHED();
    kd_dots<T, 2><<<kRedBlocks, kBlock, 0, s>>>(n3, kc2, kc2, kc2, L.b<T>(), H->partial);
    LL_LAUNCHED();
    k_finish<<<2, kBlock, 0, s>>>(H->partial, ks + 3);
    LL_LAUNCHED();
    kk_combine<T><<<nb, kBlock, 0, s>>>(n3, kz1, L.x<T>(), ks);
    LL_LAUNCHED();
  }
}

// The K-cycle on level l of a batch's union hierarchy: kinner's steps for
// every instance that has the K-cycle on this level, with each instance's
// own scalars (dots summed per instance over its chunks in a fixed order).
// Rows of instances whose coarsest level this is keep the direct solve.
template <typename T, typename TM>
void kinner_union(ll_mg_hierarchy* H, int l) {
  CLevel& L = H->lev[l];
  cudaStream_t s = H->s;
  long n3 = 3L * L.n;
  int nb = cdiv(n3, kBlock), nbs = cdiv((long)L.n * lanes<T>(), kCoarseBlock);
  double* ks = H->kscal_u.p + (size_t)8 * H->kninst * l;
  const Chunk* ch = H->kchunks[l];
  const int* ip = H->kiptr[l];
  const int* ri = H->krow_inst[l];
  int nch = H->knch[l];
  T *kr = L.kv<T>(0), *kz1 = L.kv<T>(1), *kc1 = L.kv<T>(2), *kc2 = L.kv<T>(3);
  auto dots = [&](auto nq, const T* u0, const T* v0, const T* u1, const T* v1, int field) {
    constexpr int NQ = decltype(nq)::value;
    if (nch == 0) return;
    kbk_dots<T, NQ><<<nch, kBlock, 0, s>>>(ch, nch, u0, v0, u1, v1, H->partial);
    LL_LAUNCHED();
    kbk_finish<<<dim3(H->kninst, NQ), kBlock, 0, s>>>(H->partial, nch, ip, ks, field);
    LL_LAUNCHED();
  };
  {
    LL_PROF(LL_KIND_BSR_OTHER);
    LL_CU(cudaMemcpyAsync(kr, L.b<T>(), n3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  vcycle_coarse<T, TM>(H, l, true);  // z1 = B r
  {  // c1 = A z1; d11 = c1.c1, d1r = c1.r; r1 = r - (d1r/d11) c1 (into L.b)
    LL_PROF(LL_KIND_BSR_OTHER);
    LL_CU(cudaMemcpyAsync(kz1, L.x<T>(), n3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    kb_spmv<T, TM, lanes<T>()><<<nbs, kCoarseBlock, 0, s>>>(L.n, L.rowptr, L.col, L.valm<TM>(), kz1, kc1);
    LL_LAUNCHED();
    dots(std::integral_constant<int, 2>(), kc1, kc1, kc1, kr, 0);
    kbk_axpy<T><<<nb, kBlock, 0, s>>>(n3, ri, kr, kc1, ks, 1, 0, L.b<T>());
    LL_LAUNCHED();
  }
  vcycle_coarse<T, TM>(H, l, false);  // z2 = B r1 (in L.x)
  {  // c2 = A z2 - (d12/d11) c1; d22 = c2.c2, d2r = c2.r1; x = y1 z1 + y2 z2
    LL_PROF(LL_KIND_BSR_OTHER);
    kb_spmv<T, TM, lanes<T>()><<<nbs, kCoarseBlock, 0, s>>>(L.n, L.rowptr, L.col, L.valm<TM>(), L.x<T>(), kc2);
    LL_LAUNCHED();
    dots(std::integral_constant<int, 1>(), kc1, kc2, nullptr, nullptr, 2);
    kbk_axpy<T><<<nb, kBlock, 0, s>>>(n3, ri, kc2, kc1, ks, 2, 0, kc2);
    LL_LAUNCHED();
    dots(std::integral_constant<int, 2>(), kc2, kc2, kc2, L.b<T>(), 3);
    kbk_combine<T><<<nb, kBlock, 0, s>>>(n3, ri, kz1, L.x<T>(), ks);
    LL_LAUNCHED();
  }
}

// the coarse problem of level l: a K level's two inner steps, or one cycle
template <typename T, typename TM>
void coarse_problem(ll_mg_hierarchy* H, int l) {
  if (l <= H->prm.kcycle && l < H->nlev - 1) {
    if (H->union_mode) kinner_union<T, TM>(H, l);
    else kinner<T, TM>(H, l);
  } else {
    vcycle_coarse<T, TM>(H, l, true);
  }
}

// union hierarchies: dense solves of the instances whose coarsest level is l
template <typename T>
void union_coarse(ll_mg_hierarchy* H, int l) {
  if (H->uc_n[l] == 0) return;
  CLevel& L = H->lev[l];
  LL_PROF(LL_KIND_COARSEST);
  kc_solve_batch<T><<<dim3(cdiv(H->uc_maxN[l], 32), H->uc_n[l]), 32, H->uc_maxN[l] * sizeof(double), H->s>>>(
      H->uc_tasks[l], L.b<T>(), L.x<T>());
  LL_LAUNCHED();
}

template <typename T, typename TM>
void vcycle_coarse(ll_mg_hierarchy* H, int l, bool init0_done) {
  CLevel& L = H->lev[l];
  cudaStream_t s = H->s;
  if (H->union_mode && l == H->nlev - 1) {
    union_coarse<T>(H, l);
    return;
  }
  if (l == H->tail_first) {
    LL_PROFW(LL_KIND_COARSE_TAIL, H->tail_flops, H->tail_bytes);
    launch_tail<T, TM>(H);
    return;
  }
  if (l == H->nlev - 1) {
    coarse_solve<T>(H, L.b<T>(), L.x<T>());
    return;
  }
  CLevel& N = H->lev[l + 1];
  int K = L.ncol, nu_pre = H->prm.nu_pre, nu_post = H->prm.nu_post;
  if (nu_pre == 0) {
    LL_PROF(LL_KIND_BSR_OTHER);
    k_zero<T><<<cdiv(3L * L.n, kBlock), kBlock, 0, s>>>(3L * L.n, L.x<T>());
    LL_LAUNCHED();
  }
  for (int sweep = 0; sweep < nu_pre; ++sweep) {  // one timing scope per sweep of the level
    int t0 = (sweep == 0 && init0_done) ? 1 : 0;
    double f = 0, by = 0;
    int nl = 0;
    for (int t = t0; t < K; ++t) {
      if (sweep == 0) class_work<T, TM, 0>(L, t, f, by);
      else class_work<T, TM, 1>(L, t, f, by);
      nl += L.cs[t + 1] > L.cs[t];
    }
    LL_PROFN(LL_KIND_BSR_SMOOTH, f, by, nl);
    for (int t = t0; t < K; ++t) {
      if (sweep == 0) sweep_class<T, TM, 0>(H, l, t, false);
      else sweep_class<T, TM, 1>(H, l, t, false);
    }
  }
  {
    int skip_from = nu_pre >= 1 ? L.cs[K - 1] : L.n;  // the last forward colour has zero residual
    long long rblk = nu_pre >= 1 ? L.res_blk : (long long)L.nnzb;
    LL_PROFW(LL_KIND_BSR_OTHER, sweep_flops(rblk, skip_from),
             sweep_bytes(rblk, skip_from, (int)sizeof(T), (int)sizeof(TM)));
    int init_end = (nu_pre >= 1 && l + 1 < H->nlev - 1) ? N.cs[1] : 0;
    if (skip_from > 0) {
      int blk = coarse_block(H), G = residual_lanes<T>(H);
      auto go = [&](auto gc, auto suffix) {
        constexpr int GG = decltype(gc)::value;
        launch_k(H, kb_residual<T, TM, GG, decltype(suffix)::value>, cdiv((long)skip_from * GG, blk), blk,
                 skip_from, (const int*)L.rowptr, (const int*)L.diag, (const int*)L.col, (const TM*)L.valm<TM>(),
                 (const T*)L.b<T>(), (const T*)L.x<T>(), L.r<T>());
      };
      // right after one forward sweep: the higher colours' part only
      if (nu_pre == 1) {
        if (G == 8) go(std::integral_constant<int, 8>(), std::true_type());
        else go(std::integral_constant<int, kRowLanes>(), std::true_type());
      } else {
        if (G == 8) go(std::integral_constant<int, 8>(), std::false_type());
        else go(std::integral_constant<int, kRowLanes>(), std::false_type());
      }
    }
    launch_k(H, kb_restrict<T>, cdiv(N.n, coarse_block(H)), coarse_block(H), N.n, (const int*)N.mptr,
             (const int*)N.mem, skip_from, (const T*)L.r<T>(), N.b<T>(), init_end, (const T*)N.dinv<T>(), N.x<T>());
  }
  if (H->union_mode) union_coarse<T>(H, l);  // rows past the colour classes
  coarse_problem<T, TM>(H, l + 1);
  // the correction x += P e in one pass, then plain sweeps: on this part a
  // prolongation fused into the first backward sweep (x + e formed for every
  // block that reads a lower colour) measured 5 % slower per float64 step
  // (float64 adds per block, one more dependent gather in each row's chain)
  {
    int w = (int)sizeof(T);
    LL_PROFW(LL_KIND_BSR_OTHER, 3.0 * L.n, (4.0 + 9.0 * w) * L.n);
    kb_prolong<T><<<cdiv(L.n, kBlock), kBlock, 0, s>>>(L.n, L.agg, N.x<T>(), L.x<T>());
    LL_LAUNCHED();
  }
  for (int sweep = 0; sweep < nu_post; ++sweep) {
    double f = 0, by = 0;
    int nl = 0;
    for (int t = 0; t < K; ++t) {
      class_work<T, TM, 1>(L, t, f, by);
      nl += L.cs[t + 1] > L.cs[t];
    }
    LL_PROFN(LL_KIND_BSR_SMOOTH, f, by, nl);
    for (int k = 0; k < K; ++k) sweep_class<T, TM, 1>(H, l, K - 1 - k, false);
  }
}

// z = V-cycle(r) on level 0; r float64 red-black, z red-black in T
template <typename T, typename TM>
void vcycle(ll_mg_hierarchy* H, const double* r, T* z) {
  cudaStream_t s = H->s;
  const GridGeom& g = H->g;
  if (H->nlev == 1) {  // the whole problem is the coarsest level
    k_rb_to_cellmajor<double, double><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(g, H->nat_of_slot, r, H->single_b);
    LL_LAUNCHED();
    coarse_solve<double>(H, H->single_b, H->single_x);
    k_cellmajor_to_rb<double, T><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(g, H->nat_of_slot, H->single_x, z);
    LL_LAUNCHED();
    return;
  }
  CLevel& L1 = H->lev[1];
  const T* chat = H->chat<T>();
  const T* dinv = H->dinv0<T>();
  T inv_dt = (T)(1.0 / H->dt);
  int nb = cdiv(g.nh, kBlock);
  // float32 V-cycle: C and D^-1 formed in the kernels from m~ (OnFly)
  OnFly q{H->m32.p, (float)H->alpha, (float)(1.0 / (H->h * H->h)), (float)(1.0 / H->dt)};
  bool onfly = std::is_same<T, float>::value && H->m32.p;
  auto half_sweep = [&](auto mode, int c) {
    constexpr int MODE = decltype(mode)::value;
    if constexpr (std::is_same<T, float>::value) {
      if (onfly) {
        k0_smooth_onfly<MODE><<<nb, kBlock, 0, s>>>(g, c, r, z, q);
        return;
      }
    }
    k0_smooth<T, MODE><<<nb, kBlock, 0, s>>>(g, c, r, z, chat, dinv);
  };
  if (H->prm.nu_pre >= 1) {
    {
      LL_PROFW(LL_KIND_L0_SMOOTH, 15.0 * H->l0_cells[0], (24 + 12 * (double)sizeof(T)) * H->l0_cells[0]);
      half_sweep(std::integral_constant<int, 0>(), 0);
      LL_LAUNCHED();
    }
    {
      LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[1], (24 + 24 * (double)sizeof(T)) * H->l0_cells[1]);
      half_sweep(std::integral_constant<int, 1>(), 1);
      LL_LAUNCHED();
    }
    for (int sweep = 1; sweep < H->prm.nu_pre; ++sweep) {
      {
        LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[0], (24 + 24 * (double)sizeof(T)) * H->l0_cells[0]);
        half_sweep(std::integral_constant<int, 1>(), 0);
        LL_LAUNCHED();
      }
      {
        LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[1], (24 + 24 * (double)sizeof(T)) * H->l0_cells[1]);
        half_sweep(std::integral_constant<int, 1>(), 1);
        LL_LAUNCHED();
      }
    }
    int init_end = H->nlev > 2 ? L1.cs[1] : 0;  // level 1's first colour, unless it is the coarsest
    if (H->prm.nu_pre == 1) {  // right after one forward sweep: the neighbours' part only
      LL_PROFW(LL_KIND_L0_RESTRICT, 33.0 * H->l0_cells[0], (8 + 27.0 * sizeof(T)) * H->l0_cells[0]);
      if constexpr (std::is_same<T, float>::value) {  // C formed from m~ in the kernel
        k0_restrict_onfly<<<cdiv(L1.n, kBlock), kBlock, 0, s>>>(g, z, q, L1.n, L1.mptr0, L1.mem0, L1.b<T>(),
                                                                init_end, L1.dinv<T>(), L1.x<T>(), L1.o2n);
      } else {
        // the colour-0 residual in one pass by slot, then its restriction:
        // measured 1.5 % faster per float64 step than one kernel per
        // aggregate that gathers its members' coefficients
        k0_residual_c0<T><<<cdiv(g.nh, kBlock), kBlock, 0, s>>>(g, z, chat, H->r0tmp64.p);
        LL_LAUNCHED();
        k0_restrict_c0<T><<<cdiv(L1.n, kBlock), kBlock, 0, s>>>(g, H->r0tmp64.p, L1.n, L1.mptr0, L1.mem0,
                                                                 L1.b<T>(), init_end, L1.dinv<T>(), L1.x<T>(),
                                                                 L1.o2n);
      }
    } else {
      LL_PROFW(LL_KIND_L0_RESTRICT, 48.0 * H->l0_cells[0], (24 + 15.0 * sizeof(T)) * H->l0_cells[0]);
      k0_restrict<T><<<cdiv(L1.n, kBlock), kBlock, 0, s>>>(g, r, z, chat, inv_dt, L1.n, L1.mptr0, L1.mem0,
                                                                   L1.b<T>(), init_end, L1.dinv<T>(), L1.x<T>(),
                                                                   L1.o2n);
    }
    LL_LAUNCHED();
  } else {
    LL_PROF(LL_KIND_L0_RESTRICT);
    k_zero<T><<<cdiv(H->n3, kBlock), kBlock, 0, s>>>(H->n3, z);
    LL_LAUNCHED();
    k0_restrict_b<T><<<cdiv(L1.n, kBlock), kBlock, 0, s>>>(g, r, L1.n, L1.mptr, L1.mem, L1.b<T>());
    LL_LAUNCHED();
  }
  coarse_problem<T, TM>(H, 1);
  if (H->prm.nu_post >= 1) {
    // the correction on the colour-0 slots only (the colour-1 half-sweep
    // reads them; colour 1's own x and then colour 0's are overwritten),
    // then a plain half-sweep: measured 1.2 % faster per float64 step than
    // the prolongation folded into the half-sweep's neighbour sums
    {
      LL_PROFW(LL_KIND_L0_SMOOTH, 3.0 * H->l0_cells[0], (4 + 9.0 * sizeof(T)) * H->l0_cells[0]);
      k0_prolong<T><<<cdiv(g.nh, kBlock), kBlock, 0, s>>>(g, H->agg0, L1.x<T>(), z, 0L, g.nh);
      LL_LAUNCHED();
    }
    {
      LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[1], (24 + 24 * (double)sizeof(T)) * H->l0_cells[1]);
      half_sweep(std::integral_constant<int, 1>(), 1);
      LL_LAUNCHED();
    }
    {
      LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[0], (24 + 24 * (double)sizeof(T)) * H->l0_cells[0]);
      half_sweep(std::integral_constant<int, 1>(), 0);
      LL_LAUNCHED();
    }
    for (int sweep = 1; sweep < H->prm.nu_post; ++sweep) {
      {
        LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[1], (24 + 24 * (double)sizeof(T)) * H->l0_cells[1]);
        half_sweep(std::integral_constant<int, 1>(), 1);
        LL_LAUNCHED();
      }
      {
        LL_PROFW(LL_KIND_L0_SMOOTH, 48.0 * H->l0_cells[0], (24 + 24 * (double)sizeof(T)) * H->l0_cells[0]);
        half_sweep(std::integral_constant<int, 1>(), 0);
        LL_LAUNCHED();
      }
    }
  } else {
    LL_PROF(LL_KIND_L0_RESTRICT);
    k0_prolong<T><<<cdiv(H->n2, kBlock), kBlock, 0, s>>>(g, H->agg0, L1.x<T>(), z, 0L, H->n2);
    LL_LAUNCHED();
  }
}

// ---------------------------------------------------------------------------
// GCR (Algorithm 1) with classical Gram-Schmidt applied twice
// ---------------------------------------------------------------------------
void read_head(ll_mg_hierarchy* H) {
  LL_CU(cudaMemcpyAsync(H->h_head, H->scal.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, H->s));
  LL_CU(cudaStreamSynchronize(H->s));
}

void finish(ll_mg_hierarchy* H, int nvals, double* out) {
  LL_PROF(LL_KIND_GCR_VECTOR);
  k_finish<<<nvals, kBlock, 0, H->s>>>(H->partial, out);
  LL_LAUNCHED();
}

void true_residual_launch(ll_mg_hierarchy* H) {
  {
    LL_PROFW(LL_KIND_OUTER_APPLY, 42.0 * H->g.n, 144.0 * H->g.n);
    kg_residual<<<kRedBlocks, kBlock, 0, H->s>>>(H->g, H->bw, H->xw, H->chat64, 1.0 / H->dt, H->r, H->partial);
    LL_LAUNCHED();
  }
  finish(H, 2, &H->scal.p->rn2);
}

void true_residual(ll_mg_hierarchy* H) {
  true_residual_launch(H);
  read_head(H);
}

// One GCR iteration j (Algorithm 1, steps 1-5) without host interaction:
// z_j = V-cycle(r), c_j = A z_j, two classical Gram-Schmidt passes against
// c_0..c_{j-1}, gamma_jj, alpha_j, r -= alpha_j c_j and |r|^2.
template <typename T, typename TM>
void iteration_body(ll_mg_hierarchy* H, int j) {
  cudaStream_t s = H->s;
  const GridGeom& g = H->g;
  long n3 = H->n3;
  int nbs = cdiv(H->n2, kBlock);
  GcrScal* S = H->scal.p;
  T* zj = H->Z<T>() + (size_t)j * n3;
  double* cj = H->C.p + (size_t)j * n3;
  vcycle<T, TM>(H, H->r, zj);                                                       // step 1
  if constexpr (!std::is_same<T, double>::value) {
    // mixed path: the product of the float32 z in float32-pair arithmetic
    // (see kg_apply_ff), C^ as the pair (chat32, chatlo)
    LL_PROFW(LL_KIND_OUTER_APPLY, 42.0 * g.n, 108.0 * g.n);
    double idt = 1.0 / H->dt;
    float idt_hi = (float)idt, idt_lo = (float)(idt - (double)idt_hi);
    kg_apply_ff<<<nbs, kBlock, 0, s>>>(g, zj, H->chat32, H->chatlo, idt_hi, idt_lo, cj);  // step 2
    LL_LAUNCHED();
  } else if (H->nlev > 1 && H->prm.nu_post >= 1) {
    // step 2, c = A z: the V-cycle's last half-sweep solved the colour-0 rows
    // of A z = r exactly (float64 path), so only colour 1 needs the product
    LL_PROFW(LL_KIND_OUTER_APPLY, 42.0 * H->l0_cells[1], 120.0 * H->l0_cells[1] + 48.0 * H->l0_cells[0]);
    kg_copy_colour0<<<cdiv(g.nh, kBlock), kBlock, 0, s>>>(g, H->r, cj);
    LL_LAUNCHED();
    kg_apply<T><<<cdiv(g.nh, kBlock), kBlock, 0, s>>>(g, zj, H->chat64, 1.0 / H->dt, cj, g.nh);
    LL_LAUNCHED();
  } else {
    LL_PROFW(LL_KIND_OUTER_APPLY, 42.0 * g.n, 120.0 * g.n);
    kg_apply<T><<<nbs, kBlock, 0, s>>>(g, zj, H->chat64, 1.0 / H->dt, cj);  // step 2
    LL_LAUNCHED();
  }
  // step 3: classical Gram-Schmidt, the same projection as the modified
  // Gram-Schmidt loop of Algorithm 1 in exact arithmetic.  A second pass
  // corrects the first pass's rounding; it runs only when the first removed
  // more than half of |c|^2 (k_gs_coef sets the device flag pass2 that gates
  // the second pass's kernels).  The dots of the pass that ends the
  // projection also give step 4's |c|^2 and c.r, and its update takes step 5
  // (r -= alpha_j c_j, |r|^2) in the same sweep over the vectors.
  if (j > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      const double* gate = pass == 0 ? nullptr : &S->pass2;
      // The timing scopes count no work for the second pass: the host does not
      // know whether it ran, and it mostly returns at once (the kind's rate is
      // then a lower bound).
      double wk = pass == 0 ? 1.0 : 0.0;
      for (int i0 = 0; i0 < j; i0 += kDotChunk) {
        int cnt = std::min(kDotChunk, j - i0);
        bool self = i0 == 0;  // |c|^2 and c.r before the projection, with the first dots
        {
          LL_PROFW(LL_KIND_GCR_VECTOR, wk * 2.0 * (cnt + (self ? 2 : 0)) * n3, wk * 8.0 * (cnt + (self ? 2 : 1)) * n3);
          if (self)
            launch_multidot<kDotChunk, true>(cnt, s, n3, H->C, i0, cj, H->partial, gate, H->r);
          else
            launch_multidot<kDotChunk, false>(cnt, s, n3, H->C, i0, cj, H->partial, gate);
          LL_LAUNCHED();
        }
        {
          LL_PROF(LL_KIND_GCR_VECTOR);
          k_finish<<<cnt, kBlock, 0, s>>>(H->partial, S->d + i0, gate);
          LL_LAUNCHED();
          if (self) {
            k_finish<<<2, kBlock, 0, s>>>(H->partial + (size_t)cnt * kRedBlocks, S->cq, gate);
            LL_LAUNCHED();
          }
        }
      }
      {
        LL_PROF(LL_KIND_GCR_VECTOR);
        k_gs_coef<<<1, 1, 0, s>>>(S, j, pass == 0, gate);
        LL_LAUNCHED();
      }
      {
        LL_PROFW(LL_KIND_GCR_VECTOR, wk * 2.0 * (j + 2) * n3, wk * 8.0 * (j + 4) * n3);
        kg_multiaxpy_r<<<kRedBlocks, kBlock, 0, s>>>(n3, cj, H->C, j, S->coef, H->r, &S->rnow, &S->rcoef,
                                                     H->partial, gate);
        LL_LAUNCHED();
      }
    }
  } else {
    {
      LL_PROFW(LL_KIND_GCR_VECTOR, 4.0 * n3, 16.0 * n3);
      kg_dot2<<<kRedBlocks, kBlock, 0, s>>>(n3, cj, H->r, H->partial);             // step 4
      LL_LAUNCHED();
    }
    finish(H, 2, &S->cc);
    {
      LL_PROF(LL_KIND_GCR_VECTOR);
      k_norm_coef<<<1, 1, 0, s>>>(S, j);
      LL_LAUNCHED();
    }
    {
      LL_PROFW(LL_KIND_GCR_VECTOR, 4.0 * n3, 24.0 * n3);
      kg_rupdate<<<kRedBlocks, kBlock, 0, s>>>(n3, H->r, cj, &S->rcoef, H->partial); // step 5
      LL_LAUNCHED();
    }
  }
  finish(H, 1, &S->rn2);
}

// the graphs hold 1/dt as a kernel argument: a new dt drops them
void graphs_for_dt(ll_mg_hierarchy* H) {
  if (H->graph_dt != H->dt) {
    for (int q = 0; q < kMaxRestart; ++q) H->drop_graph(q);
    H->graph_dt = H->dt;
  }
}

// run iteration j, from a CUDA graph captured on first use (one launch
// instead of a few hundred), then fold any graph-timed kernels into the totals
template <typename T, typename TM>
void run_iteration(ll_mg_hierarchy* H, int j) {
  if (!H->use_graphs) {
    iteration_body<T, TM>(H, j);
    return;
  }
  graphs_for_dt(H);
  if (H->graphs[j] && H->graph_mask[j] != H->prof_mask) H->drop_graph(j);
  if (!H->graphs[j]) {
    cudaGraph_t graph;
    long long before = t_launches;
    LL_CU(cudaStreamBeginCapture(H->s, cudaStreamCaptureModeThreadLocal));
    H->capturing = j;
    try {
      iteration_body<T, TM>(H, j);
    } catch (Status) {
      H->capturing = -1;
      cudaStreamEndCapture(H->s, &graph);
      throw;
    }
    H->capturing = -1;
    LL_CU(cudaStreamEndCapture(H->s, &graph));
    cudaError_t e = cudaGraphInstantiate(&H->graphs[j], graph, 0);
    cudaGraphDestroy(graph);
    LL_CU(e);
    H->graph_mask[j] = H->prof_mask;
    H->graph_kernels[j] = t_launches - before;  // counted per launch below
    g_launches.fetch_sub(H->graph_kernels[j]);
  }
  LL_CU(cudaGraphLaunch(H->graphs[j], H->s));
  g_launches.fetch_add(H->graph_kernels[j]);
  if (!H->gpairs[j].empty()) {
    LL_CU(cudaStreamSynchronize(H->s));
    for (auto& q : H->gpairs[j]) {
      float ms = 0;
      LL_CU(cudaEventElapsedTime(&ms, q.b, q.e));
      H->prof_ms[q.kind] += ms;
      H->prof_n[q.kind] += q.nl;
      H->prof_flops[q.kind] += q.flops;
      H->prof_bytes[q.kind] += q.bytes;
    }
  }
}

// The true residual norms at the restarts of one solve, for the stagnation
// stop of ll_mg_params (stall_window, stall_ratio).
struct StallHist {
  std::vector<std::pair<int, double>> at;  // (iterations so far, norm)
  // true: stop (the norm rn at `total` iterations exceeds stall_ratio times
  // the norm at the latest restart at least stall_window iterations
  // earlier); otherwise the restart is recorded
  bool stalled(const ll_mg_params& p, int total, double rn) {
    if (p.stall_window > 0)
      for (int k = (int)at.size() - 1; k >= 0; --k)
        if (at[k].first <= total - p.stall_window) {
          if (rn > p.stall_ratio * at[k].second) return true;
          break;
        }
    at.push_back({total, rn});
    return false;
  }
};

template <typename T, typename TM>
int gcr(ll_mg_hierarchy* H, const double* b_nat, double* x_nat, double rtol, int* iters, double* relres) {
  cudaStream_t s = H->s;
  const GridGeom& g = H->g;
  long n3 = H->n3;
  int nbs = cdiv(H->n2, kBlock), nbv = cdiv(n3, kBlock);
  k_to_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, b_nat, H->bw);
  LL_LAUNCHED();
  k_to_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, x_nat, H->xw);
  LL_LAUNCHED();
  GcrScal* S = H->scal.p;
  int total = 0, status = LL_NOT_CONVERGED;
  double bnorm = 0;
  bool current = false;  // the loop ended on the true residual of the final x
  StallHist stall;
  for (;;) {
    true_residual(H);
    double rn2 = H->h_head[0];
    bnorm = sqrt(H->h_head[1]);
    if (bnorm == 0.0) {
      k_zero<double><<<nbv, kBlock, 0, s>>>(n3, H->xw);
      LL_LAUNCHED();
      status = LL_OK;
      break;
    }
    if (!isfinite(rn2)) {
      status = LL_BREAKDOWN;
      break;
    }
    if (sqrt(rn2) < rtol * bnorm) {
      status = LL_OK;
      current = true;
      break;
    }
    if (total >= H->prm.maxit || stall.stalled(H->prm, total, sqrt(rn2))) {
      current = true;
      break;
    }
    int m = std::min(H->prm.restart, H->prm.maxit - total);
    int jdone = 0;
    bool broke = false;
    for (int j = 0; j < m; ++j) {
      run_iteration<T, TM>(H, j);
      ++total;
      read_head(H);
      double gjj = H->h_head[4];
      if (!(gjj > 0.0) || !isfinite(gjj)) {
        broke = true;
        break;
      }
      jdone = j + 1;
      double rj = sqrt(H->h_head[0]);
      if (!isfinite(rj)) {
        broke = true;
        break;
      }
      if (rj < rtol * bnorm) break;                                                  // step 6
    }
    if (jdone > 0) {
      {
        LL_PROF(LL_KIND_GCR_VECTOR);
        k_backsub<<<1, 1, 0, s>>>(S, jdone);
        LL_LAUNCHED();
      }
      {
        LL_PROFW(LL_KIND_GCR_VECTOR, 2.0 * jdone * n3, (16.0 + sizeof(T) * jdone) * n3);
        kg_xupdate<T><<<nbv, kBlock, 0, s>>>(n3, H->xw, H->Z<T>(), jdone, S->y);
        LL_LAUNCHED();
      }
    }
    if (broke) {
      status = LL_BREAKDOWN;
      break;
    }
  }
  if (!current) true_residual(H);
  if (iters) *iters = total;
  if (relres) *relres = bnorm > 0 ? sqrt(H->h_head[0]) / bnorm : 0.0;
  k_from_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, H->xw, x_nat);
  LL_LAUNCHED();
  LL_CU(cudaStreamSynchronize(s));
  return status;
}

int solve(ll_mg_hierarchy* H, const double* b, double* x, double rtol, int* it, double* rr) {
  if (rtol <= 0) rtol = H->prm.rtol;
  if (H->prm.precision == LL_MIXED_BF16) return gcr<float, __nv_bfloat16>(H, b, x, rtol, it, rr);
  if (H->prm.precision == LL_MIXED_FP32) return gcr<float, float>(H, b, x, rtol, it, rr);
  return gcr<double, double>(H, b, x, rtol, it, rr);
}

bool valid_params(const ll_mg_params& p) {
  return p.rtol >= 0 && p.maxit >= 0 && p.restart >= 1 && p.restart <= kMaxRestart && p.nu_pre >= 0 &&
         p.nu_pre <= 16 && p.nu_post >= 0 && p.nu_post <= 16 && p.coarsest_cells >= 1 && p.max_levels >= 1 &&
         p.max_levels <= kMaxLevels && p.rounds >= 1 &&
         (p.precision == LL_FP64 || p.precision == LL_MIXED_FP32 || p.precision == LL_MIXED_BF16) &&
         p.kcycle >= 0 && p.kcycle <= kMaxLevels &&
         (p.coarse_lanes == 0 || p.coarse_lanes == kRowLanes || p.coarse_lanes == 8) &&
         (p.coarse_block == 0 || p.coarse_block == 32 || p.coarse_block == 64 || p.coarse_block == 128 ||
          p.coarse_block == 256) &&
         p.stall_window >= 0 && (p.stall_window == 0 || (p.stall_ratio > 0 && isfinite(p.stall_ratio)));
}

// standalone = false: an instance of a batch, solved only through the batch's
// union hierarchy (no SELL-32 copies)
int create(const double* m, double alpha, double dt, double h, ll_grid grid, const ll_mg_params* p, void* stream,
           ll_mg_hierarchy** out, bool standalone = true) {
  ll_mg_hierarchy* H = nullptr;
  try {
    H = new ll_mg_hierarchy();
    ll_mg_default_params(&H->prm);
    if (p) H->prm = *p;
    H->user = (cudaStream_t)stream;
    LL_CU(cudaStreamCreateWithFlags(&H->s, cudaStreamNonBlocking));
    LL_CU(cudaEventCreateWithFlags(&H->entry_ev, cudaEventDisableTiming));
    const char* ng = getenv("LLMG_NO_GRAPHS");
    H->use_graphs = !(ng && ng[0] == '1');
    enter(H);
    H->alpha = alpha;
    H->dt = dt;
    H->h = h;
    GridGeom& g = H->g;
    g.nx = grid.nx;
    g.ny = grid.ny;
    g.nz = grid.nz;
    g.nxh = (grid.nx + 1) / 2;
    g.nh = (long)g.nxh * grid.ny * grid.nz;
    g.n = (long)grid.nx * grid.ny * grid.nz;
    H->n2 = 2 * g.nh;
    H->n3 = 3 * H->n2;
    H->sell_ok = standalone && H->prm.precision == LL_FP64 && H->prm.coarse_lanes == 0 && H->prm.coarse_block == 0;
    symbolic(H);
    allocate(H);
    setup_counts(H);
    setup_tail(H);
    numeric(H, m);
    *out = H;
    return LL_OK;
  } catch (Status st) {
    delete H;
    return st.code;
  } catch (std::bad_alloc&) {
    delete H;
    return LL_ENOMEM;
  }
}

}  // namespace

#include "ll_batch.cuh"
#include "ll_autotune.cuh"

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void ll_mg_default_params(ll_mg_params* p) {
  if (!p) return;
  p->rtol = 1e-8;
  p->maxit = 1000;
  p->restart = 10;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->coarsest_cells = 64;
  p->max_levels = 20;
  p->rounds = 32;
  p->seed = 0;
  p->precision = LL_FP64;
  p->kcycle = 0;
  p->coarse_lanes = 0;
  p->coarse_block = 0;
  p->stall_window = 0;
  p->stall_ratio = 0.99;
}

static bool valid_problem(double alpha, double dt, double h, ll_grid grid) {
  if (!(dt > 0) || !(h > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(h) || !isfinite(alpha)) return false;
  if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1) return false;
  long n = (long)grid.nx * grid.ny * grid.nz;
  return n >= 2 && n < (1L << 29);
}

int ll_mg_setup(const double* m_tilde, double alpha, double dt, double h, ll_grid grid, const ll_mg_params* p,
                void* cuda_stream, ll_mg_hierarchy** out) {
  if (!m_tilde || !out || !valid_problem(alpha, dt, h, grid)) return LL_EINVAL;
  if (p && !valid_params(*p)) return LL_EINVAL;
  return create(m_tilde, alpha, dt, h, grid, p, cuda_stream, out);
}

int ll_mg_update(ll_mg_hierarchy* H, const double* m_tilde, double alpha, double dt) {
  if (!H || !m_tilde || !(dt > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(alpha)) return LL_EINVAL;
  try {
    enter(H);
    if (alpha != H->alpha || dt != H->dt) H->step_hist = false;  // the kept states belong to the old step
    H->alpha = alpha;
    H->dt = dt;
    numeric(H, m_tilde);
    return LL_OK;
  } catch (Status st) {
    return st.code;
  }
}

int ll_mg_solve(ll_mg_hierarchy* H, const double* rhs, double* x, double rtol, int* iterations,
                double* rel_residual) {
  if (!H || !rhs || !x) return LL_EINVAL;
  try {
    enter(H);
    return solve(H, rhs, x, rtol, iterations, rel_residual);
  } catch (Status st) {
    return st.code;
  }
}

// time steps on an existing hierarchy; fresh = numeric setup already done for
// m; src = explicit source terms (q, he0, he1, he2) or NULL
// Time steps of m in place.  The initial approximation of each solve: m and
// the (up to kStepHist) states before it that are known -- within a call
// from its second step, and from the first step when m is bit for bit the
// last output of the previous call on this hierarchy (a continued
// integration) -- extrapolated with the backward-difference terms that keep
// shrinking (the oracle's step_guess; not for x_save, the adjoint's forward
// map, whose solves start from m).
static int steps(ll_mg_hierarchy* H, double* m, int n_steps, int* iters_per_step, double* relres_per_step,
                 bool fresh, const double* src = nullptr, double* x_save = nullptr) {
  int worst = LL_OK;
  double dt = H->dt;
  try {
    long n3 = 3 * H->g.n;
    bool guess = x_save == nullptr;
    int depth = 0;  // earlier states known for the next step's guess
    if (guess) {
      if (!H->step_last.p) {
        for (auto& b : H->step_h) b.alloc(n3);
        H->step_last.alloc(n3);
        H->step_norms.alloc(kStepHist);
        H->step_differ.alloc(1);
      }
      if (H->step_hist && n_steps > 0) {
        H->step_differ.zero(H->s);
        k_differ<<<cdiv(n3, kBlock), kBlock, 0, H->s>>>(n3, m, H->step_last, H->step_differ);
        LL_LAUNCHED();
        int differ = 1;
        LL_CU(cudaMemcpyAsync(&differ, H->step_differ.p, sizeof(int), cudaMemcpyDeviceToHost, H->s));
        LL_CU(cudaStreamSynchronize(H->s));
        if (differ == 0) depth = H->step_depth;
      }
      H->step_hist = false;  // set again when every step of this call has completed
    }
    auto hist = [&](int j) { return H->step_h[(H->step_i + j) % kStepHist].p; };
    for (int k = 0; k < n_steps; ++k) {
      if (k > 0 || !fresh) numeric(H, m);
      if (src)
        k_rhs_llg<<<cdiv(H->g.n, kBlock), kBlock, 0, H->s>>>(H->g.n, m, H->alpha, 1.0 / dt, src[0], src[1], src[2],
                                                             src[3], H->stepb);
      else
        k_scale<<<cdiv(n3, kBlock), kBlock, 0, H->s>>>(n3, m, 1.0 / dt, H->stepb);
      LL_LAUNCHED();
      if (depth > 0) {
        StepStates S = {};
        S.s[0] = m;
        for (int l = 1; l <= depth; ++l) S.s[l] = hist(l - 1);
        k_step_diff_norms<<<kRedBlocks, kBlock, 0, H->s>>>(n3, depth, S, H->partial);
        LL_LAUNCHED();
        k_finish<<<kStepHist, kBlock, 0, H->s>>>(H->partial, H->step_norms);
        LL_LAUNCHED();
        double nrm[kStepHist];
        LL_CU(cudaMemcpyAsync(nrm, H->step_norms.p, kStepHist * sizeof(double), cudaMemcpyDeviceToHost, H->s));
        LL_CU(cudaStreamSynchronize(H->s));
        int order = 1;  // the terms D^j m while their norms shrink (nrm[j-1] = |D^j m|^2)
        for (int j = 2; j <= depth && nrm[j - 1] < nrm[j - 2]; ++j) order = j;
        StepCoef C = {};
        for (int l = 0; l <= order; ++l) {  // (-1)^l C(order+1, l+1)
          double b = 1.0;
          for (int q = 0; q <= l; ++q) b = b * (double)(order + 1 - q) / (double)(q + 1);
          C.c[l] = (l % 2 ? -1.0 : 1.0) * b;
        }
        k_step_guess<<<cdiv(n3, kBlock), kBlock, 0, H->s>>>(n3, order, S, C, H->stepx);
        LL_LAUNCHED();
      } else {
        LL_CU(cudaMemcpyAsync(H->stepx.p, m, n3 * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
      }
      if (guess) {  // m^n becomes the newest earlier state (the oldest slot is reused)
        H->step_i = (H->step_i + kStepHist - 1) % kStepHist;
        LL_CU(cudaMemcpyAsync(hist(0), m, n3 * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
        depth = std::min(depth + 1, kStepHist);
        H->step_depth = depth;
      }
      int it = 0;
      double rr = 0;
      int s2 = solve(H, H->stepb, H->stepx, H->prm.rtol, &it, &rr);
      if (iters_per_step) iters_per_step[k] = it;
      if (relres_per_step) relres_per_step[k] = rr;
      worst = std::max(worst, s2);
      if (x_save)  // the solution before the projection, step k
        LL_CU(cudaMemcpyAsync(x_save + (size_t)k * n3, H->stepx.p, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                              H->s));
      H->flag.zero(H->s);
      k_renormalise<<<cdiv(H->g.n, kBlock), kBlock, 0, H->s>>>(H->g.n, H->stepx, m, H->flag);
      LL_LAUNCHED();
      check_flag(H, LL_BREAKDOWN);
    }
    if (guess && n_steps > 0 && worst == LL_OK) {
      LL_CU(cudaMemcpyAsync(H->step_last.p, m, n3 * sizeof(double), cudaMemcpyDeviceToDevice, H->s));
      H->step_hist = true;
    }
  } catch (Status e) {
    worst = e.code;
    H->step_hist = false;
  }
  return worst;
}

int ll_step(double* m, int n_steps, double alpha, double dt, double h, ll_grid grid, const ll_mg_params* p,
            void* cuda_stream, int* iters_per_step, double* relres_per_step) {
  if (!m || n_steps < 0 || !valid_problem(alpha, dt, h, grid)) return LL_EINVAL;
  if (p && !valid_params(*p)) return LL_EINVAL;
  if (n_steps == 0) return LL_OK;
  ll_mg_hierarchy* H = nullptr;
  int st = create(m, alpha, dt, h, grid, p, cuda_stream, &H);
  if (st != LL_OK) return st;
  int worst = steps(H, m, n_steps, iters_per_step, relres_per_step, true);
  delete H;
  return worst;
}

int ll_mg_step(ll_mg_hierarchy* H, double* m, int n_steps, int* iters_per_step, double* relres_per_step) {
  if (!H || !m || n_steps < 0) return LL_EINVAL;
  try {
    enter(H);
  } catch (Status st) {
    return st.code;
  }
  return steps(H, m, n_steps, iters_per_step, relres_per_step, false);
}

int ll_mg_step_llg(ll_mg_hierarchy* H, double* m, int n_steps, double q, const double* he, int* iters_per_step,
                   double* relres_per_step) {
  if (!H || !m || n_steps < 0 || !isfinite(q)) return LL_EINVAL;
  double src[4] = {q, he ? he[0] : 0.0, he ? he[1] : 0.0, he ? he[2] : 0.0};
  if (!isfinite(src[1]) || !isfinite(src[2]) || !isfinite(src[3])) return LL_EINVAL;
  try {
    enter(H);
  } catch (Status st) {
    return st.code;
  }
  return steps(H, m, n_steps, iters_per_step, relres_per_step, false, src);
}

int ll_mg_step_save(ll_mg_hierarchy* H, double* m, int n_steps, double* x_save, int* iters_per_step,
                    double* relres_per_step) {
  if (!H || !m || !x_save || n_steps < 0) return LL_EINVAL;
  try {
    enter(H);
  } catch (Status st) {
    return st.code;
  }
  int st = steps(H, m, n_steps, iters_per_step, relres_per_step, false, nullptr, x_save);
  cudaStreamSynchronize(H->s);
  return st;
}

int ll_mg_step_host(ll_mg_hierarchy* H, double* m_host, int n_steps, int* iters_per_step,
                    double* relres_per_step) {
  if (!H || !m_host || n_steps < 0) return LL_EINVAL;
  size_t bytes = 3 * (size_t)H->g.n * sizeof(double);
  try {
    enter(H);
    if (!H->hostm.p) H->hostm.alloc(3 * H->g.n);
    LL_CU(cudaMemcpyAsync(H->hostm.p, m_host, bytes, cudaMemcpyHostToDevice, H->s));
  } catch (Status st) {
    return st.code;
  }
  int worst = steps(H, H->hostm.p, n_steps, iters_per_step, relres_per_step, false);
  if (worst < 0) return worst;
  if (cudaMemcpyAsync(m_host, H->hostm.p, bytes, cudaMemcpyDeviceToHost, H->s) != cudaSuccess ||
      cudaStreamSynchronize(H->s) != cudaSuccess)
    return LL_ECUDA;
  return worst;
}

long long ll_launch_count(void) { return g_launches.load(); }

int ll_fp64_fma_probe(double* sink, long long iters, int blocks, void* cuda_stream, double* flops) {
  if (!sink || iters < 1 || blocks < 1) return LL_EINVAL;
  k_fp64_fma_probe<<<blocks, kProbeThreads, 0, (cudaStream_t)cuda_stream>>>(sink, iters);
  if (cudaGetLastError() != cudaSuccess) return LL_ECUDA;
  count_launch();
  if (flops) *flops = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
  return LL_OK;
}

void ll_mg_destroy(ll_mg_hierarchy* H) {
  if (H) {
    cudaStreamSynchronize(H->s);
    delete H;
  }
}

const char* ll_status_string(int status) {
  switch (status) {
    case LL_OK: return "converged";
    case LL_NOT_CONVERGED: return "not converged (maxit reached, or stagnated under the stall test)";
    case LL_BREAKDOWN: return "breakdown (non-finite residual or zero GCR norm)";
    case LL_EINVAL: return "invalid argument";
    case LL_ECUDA: return "CUDA runtime error";
    case LL_ENOMEM: return "out of device memory";
    case LL_SINGULAR_COARSE: return "singular block or coarsest matrix";
    case LL_ELIMIT: return "structural limit exceeded";
    default: return "unknown status";
  }
}

const char* ll_last_cuda_error(void) { return t_cuda_error; }

int ll_mg_levels(const ll_mg_hierarchy* H) { return H ? H->nlev : -1; }

int ll_mg_level_cells(const ll_mg_hierarchy* H, int l) {
  if (!H || l < 0 || l >= H->nlev) return -1;
  return l == 0 ? (int)H->g.n : H->lev[l].n;
}

int ll_mg_level_aggregates(const ll_mg_hierarchy* H, int l, int* agg) {
  if (!H || !agg || l < 0 || l >= H->nlev - 1) return LL_EINVAL;
  const int* src = l == 0 ? H->agg_nat0.p : H->lev[l].agg_orig.p;
  int n = ll_mg_level_cells(H, l);
  if (cudaMemcpy(agg, src, n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LL_ECUDA;
  return LL_OK;
}

int ll_mg_level_colours(const ll_mg_hierarchy* H, int l, int* colour) {
  if (!H || !colour || l < 0 || l >= H->nlev) return LL_EINVAL;
  if (l == 0) {
    const GridGeom& g = H->g;
    for (long k = 0; k < g.n; ++k) {
      long x = k % g.nx, t = k / g.nx, y = t % g.ny, z = t / g.ny;
      colour[k] = (int)((x + y + z) & 1);
    }
    return LL_OK;
  }
  if (cudaMemcpy(colour, H->lev[l].colour.p, H->lev[l].n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LL_ECUDA;
  return LL_OK;
}

int ll_mg_level_blocks(const ll_mg_hierarchy* H, int l) {
  if (!H || l < 1 || l >= H->nlev) return -1;
  return H->lev[l].nnzb;
}

int ll_mg_level_operator(const ll_mg_hierarchy* H, int l, int* rowptr, int* col, double* val) {
  if (!H || l < 1 || l >= H->nlev || !rowptr || !col || !val) return LL_EINVAL;
  const CLevel& C = H->lev[l];
  // the operator is stored in the colour-class numbering; return it in the
  // aggregation's numbering, columns ascending
  std::vector<int> rp(C.n + 1), cl(C.nnzb), n2o(C.n), o2n(C.n);
  std::vector<double> va(9L * C.nnzb);
  std::vector<float> va32;
  bool f32 = C.val64.p == nullptr;  // mixed hierarchy: the float32 Galerkin values
  if (f32) va32.resize(9L * C.nnzb);
  if (cudaMemcpy(rp.data(), C.rowptr.p, (C.n + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(cl.data(), C.col.p, C.nnzb * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      (f32 ? cudaMemcpy(va32.data(), C.val32.p, 9L * C.nnzb * sizeof(float), cudaMemcpyDeviceToHost)
           : cudaMemcpy(va.data(), C.val64.p, 9L * C.nnzb * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      cudaMemcpy(n2o.data(), C.n2o.p, C.n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LL_ECUDA;
  if (f32)
    for (size_t i = 0; i < va.size(); ++i) va[i] = va32[i];
  for (int r = 0; r < C.n; ++r) o2n[n2o[r]] = r;
  int q = 0;
  rowptr[0] = 0;
  for (int o = 0; o < C.n; ++o) {
    int r = o2n[o];
    std::vector<std::pair<int, int>> blocks;
    for (int p = rp[r]; p < rp[r + 1]; ++p) blocks.push_back({n2o[cl[p]], p});
    std::sort(blocks.begin(), blocks.end());
    for (auto& bp : blocks) {
      col[q] = bp.first;
      for (int e = 0; e < 9; ++e) val[9L * q + e] = va[9L * bp.second + e];
      ++q;
    }
    rowptr[o + 1] = q;
  }
  return LL_OK;
}

int ll_mg_profile(ll_mg_hierarchy* H, unsigned int kinds) {
  if (!H) return LL_EINVAL;
  if (cudaStreamSynchronize(H->s) != cudaSuccess) return LL_ECUDA;
  H->prof_mask = kinds;
  H->ev_used = 0;
  for (auto& v : H->prof_pairs) v.clear();
  for (int k = 0; k < LL_NUM_KINDS; ++k) {
    H->prof_ms[k] = 0;
    H->prof_n[k] = 0;
    H->prof_flops[k] = 0;
    H->prof_bytes[k] = 0;
  }
  return LL_OK;
}

int ll_mg_profile_read(ll_mg_hierarchy* H, int kind, double* total_ms, long long* launches, double* flops,
                       double* bytes) {
  if (!H || kind < 0 || kind >= LL_NUM_KINDS) return LL_EINVAL;
  if (cudaStreamSynchronize(H->s) != cudaSuccess) return LL_ECUDA;
  double tot = H->prof_ms[kind];
  for (auto& pr : H->prof_pairs[kind]) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess) return LL_ECUDA;
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = H->prof_n[kind];
  if (flops) *flops = H->prof_flops[kind];
  if (bytes) *bytes = H->prof_bytes[kind];
  return LL_OK;
}

int ll_mg_apply(ll_mg_hierarchy* H, const double* x, double* y) {
  if (!H || !x || !y) return LL_EINVAL;
  try {
    enter(H);
    const GridGeom& g = H->g;
    int nbs = cdiv(H->n2, kBlock);
    k_to_rb<double, double><<<nbs, kBlock, 0, H->s>>>(g, H->nat_of_slot, x, H->xw);
    LL_LAUNCHED();
    kg_apply<double><<<nbs, kBlock, 0, H->s>>>(g, H->xw, H->chat64, 1.0 / H->dt, H->r);
    LL_LAUNCHED();
    k_from_rb<double, double><<<nbs, kBlock, 0, H->s>>>(g, H->nat_of_slot, H->r, y);
    LL_LAUNCHED();
    LL_CU(cudaStreamSynchronize(H->s));
    return LL_OK;
  } catch (Status st) {
    return st.code;
  }
}

int ll_mg_vcycle(ll_mg_hierarchy* H, const double* r, double* z) {
  if (!H || !r || !z) return LL_EINVAL;
  try {
    enter(H);
    const GridGeom& g = H->g;
    int nbs = cdiv(H->n2, kBlock);
    k_to_rb<double, double><<<nbs, kBlock, 0, H->s>>>(g, H->nat_of_slot, r, H->bw);
    LL_LAUNCHED();
    if (H->prm.precision != LL_FP64) {
      if (H->prm.precision == LL_MIXED_BF16) vcycle<float, __nv_bfloat16>(H, H->bw, H->Z32.p);
      else vcycle<float, float>(H, H->bw, H->Z32.p);
      k_from_rb<float, double><<<nbs, kBlock, 0, H->s>>>(g, H->nat_of_slot, H->Z32.p, z);
    } else {
      vcycle<double, double>(H, H->bw, H->Z64.p);
      k_from_rb<double, double><<<nbs, kBlock, 0, H->s>>>(g, H->nat_of_slot, H->Z64.p, z);
    }
    LL_LAUNCHED();
    LL_CU(cudaStreamSynchronize(H->s));
    return LL_OK;
  } catch (Status st) {
    return st.code;
  }
}

int ll_mg_smooth(ll_mg_hierarchy* H, int l, const double* b, double* x, int forward) {
  if (!H || !b || !x || l < 0 || l >= H->nlev || H->prm.precision != LL_FP64) return LL_EINVAL;
  if (l == H->nlev - 1 && l > 0) return LL_EINVAL;  // the coarsest level is solved, not smoothed
  try {
    enter(H);
    const GridGeom& g = H->g;
    cudaStream_t s = H->s;
    if (l == 0) {
      if (H->nlev == 1) return LL_EINVAL;
      int nbs = cdiv(H->n2, kBlock), nb = cdiv(g.nh, kBlock);
      k_to_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, b, H->bw);
      LL_LAUNCHED();
      k_to_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, x, H->xw);
      LL_LAUNCHED();
      for (int t = 0; t < 2; ++t) {
        int c = forward ? t : 1 - t;
        k0_smooth<double, 1><<<nb, kBlock, 0, s>>>(g, c, H->bw, H->xw.p, H->chat64, H->dinv64);
        LL_LAUNCHED();
      }
      k_from_rb<double, double><<<nbs, kBlock, 0, s>>>(g, H->nat_of_slot, H->xw, x);
      LL_LAUNCHED();
    } else {  // vectors given in the aggregation's numbering
      CLevel& L = H->lev[l];
      int nb = cdiv(L.n, kBlock);
      kb_gather3<double><<<nb, kBlock, 0, s>>>(L.n, L.n2o, b, L.b64.p);
      LL_LAUNCHED();
      kb_gather3<double><<<nb, kBlock, 0, s>>>(L.n, L.n2o, x, L.x64.p);
      LL_LAUNCHED();
      smooth_level<double, double>(H, l, forward != 0);
      kb_scatter3<double><<<nb, kBlock, 0, s>>>(L.n, L.n2o, L.x64.p, x);
      LL_LAUNCHED();
    }
    LL_CU(cudaStreamSynchronize(s));
    return LL_OK;
  } catch (Status st) {
    return st.code;
  }
}

// ---------------------------------------------------------------------------
// batches of independent instances
// ---------------------------------------------------------------------------
int ll_mg_batch_setup(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                      const double* h, const ll_grid* grids, const ll_mg_params* p, void* cuda_stream,
                      ll_mg_batch** out) {
  if (count < 1 || !m_tilde || !alpha || !dt || !h || !grids || !out) return LL_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!m_tilde[i] || !valid_problem(alpha[i], dt[i], h[i], grids[i])) return LL_EINVAL;
  if (p && !valid_params(*p)) return LL_EINVAL;
  if (p && p->precision == LL_MIXED_BF16) return LL_EINVAL;
  return batch_create(count, m_tilde, alpha, dt, h, grids, p, cuda_stream, out);
}

int ll_mg_batch_update(ll_mg_batch* B, const double* const* m_tilde, const double* alpha, const double* dt) {
  if (!B || !m_tilde || !alpha || !dt) return LL_EINVAL;
  for (int i = 0; i < B->ninst; ++i)
    if (!m_tilde[i] || !(dt[i] > 0) || !(alpha[i] >= 0) || !isfinite(dt[i]) || !isfinite(alpha[i])) return LL_EINVAL;
  if (!B->groups.empty())
    return for_groups(B, [&](ll_mg_batch* G, const std::vector<int>& idx) {
      std::vector<const double*> mg;
      std::vector<double> ag, dg;
      for (int i : idx) {
        mg.push_back(m_tilde[i]);
        ag.push_back(alpha[i]);
        dg.push_back(dt[i]);
      }
      return ll_mg_batch_update(G, mg.data(), ag.data(), dg.data());
    });
  try {
    batch_enter(B);
    LL_CU(cudaStreamSynchronize(B->U->s));
    for (int i = 0; i < B->ninst; ++i) {  // queue every instance (own streams), then check
      ll_mg_hierarchy* H = B->inst[i];
      H->alpha = alpha[i];
      H->dt = dt[i];
      numeric_launch(H, m_tilde[i]);
    }
    for (auto* H : B->inst) numeric_check(H);
    batch_refresh(B);
    for (auto& c : B->children) batch_refresh(c.second);  // sub-batches share the instances
    return LL_OK;
  } catch (Status st) {
    return st.code;
  }
}

int ll_mg_batch_solve(ll_mg_batch* B, const double* const* rhs, double* const* x, double rtol, int* iterations,
                      double* rel_residual, int* status) {
  if (!B || !rhs || !x) return LL_EINVAL;
  for (int i = 0; i < B->ninst; ++i)
    if (!rhs[i] || !x[i]) return LL_EINVAL;
  if (!B->groups.empty()) {
    std::vector<int> its(B->ninst, 0), sts(B->ninst, LL_NOT_CONVERGED);
    std::vector<double> rrs(B->ninst, 0.0);
    int rc = for_groups(B, [&](ll_mg_batch* G, const std::vector<int>& idx) {
      std::vector<const double*> rg;
      std::vector<double*> xg;
      std::vector<int> ig(idx.size()), sg(idx.size());
      std::vector<double> qg(idx.size());
      for (int i : idx) {
        rg.push_back(rhs[i]);
        xg.push_back(x[i]);
      }
      int r = ll_mg_batch_solve(G, rg.data(), xg.data(), rtol, ig.data(), qg.data(), sg.data());
      for (size_t k = 0; k < idx.size(); ++k) {
        its[idx[k]] = ig[k];
        rrs[idx[k]] = qg[k];
        sts[idx[k]] = sg[k];
      }
      return r;
    });
    if (rc < 0) return rc;
    if (iterations) std::copy(its.begin(), its.end(), iterations);
    if (rel_residual) std::copy(rrs.begin(), rrs.end(), rel_residual);
    if (status) std::copy(sts.begin(), sts.end(), status);
    int worst = LL_OK;
    for (int st : sts) {
      if (st == LL_BREAKDOWN) worst = LL_BREAKDOWN;
      else if (st == LL_NOT_CONVERGED && worst == LL_OK) worst = LL_NOT_CONVERGED;
    }
    return worst;
  }
  try {
    batch_enter(B);
    return batch_solve(B, rhs, x, rtol, iterations, rel_residual, status);
  } catch (Status st) {
    return st.code;
  }
}

int ll_mg_batch_count(const ll_mg_batch* B) { return B ? B->ninst : 0; }
int ll_mg_batch_levels(const ll_mg_batch* B) { return B && B->U ? B->U->nlev : -1; }
long long ll_mg_batch_level_rows(const ll_mg_batch* B, int level) {
  if (!B || !B->U || level < 0 || level >= B->U->nlev) return -1;
  return B->U->lev[level].n;
}
int ll_mg_batch_level_colours(const ll_mg_batch* B, int level) {
  if (!B || !B->U || level < 0 || level >= B->U->nlev) return -1;
  return B->U->lev[level].ncol;
}
int ll_mg_batch_subbatches(const ll_mg_batch* B) {
  if (!B) return 0;
  int n = (int)B->children.size();
  for (auto* g : B->groups) n += ll_mg_batch_subbatches(g);
  return n;
}

int ll_mg_batch_instance_levels(const ll_mg_batch* B, int i) {
  if (!B || i < 0 || i >= B->ninst) return -1;
  for (size_t g = 0; g < B->groups.size(); ++g)
    for (size_t k = 0; k < B->gidx[g].size(); ++k)
      if (B->gidx[g][k] == i) return ll_mg_batch_instance_levels(B->groups[g], (int)k);
  return B->inst[i]->nlev;
}

int ll_mg_batch_groups(const ll_mg_batch* B) { return B ? std::max(1, (int)B->groups.size()) : 0; }

int ll_mg_batch_instance_group(const ll_mg_batch* B, int i) {
  if (!B || i < 0 || i >= B->ninst) return -1;
  for (size_t g = 0; g < B->groups.size(); ++g)
    for (int k : B->gidx[g])
      if (k == i) return (int)g;
  return 0;
}

int ll_mg_batch_autotune(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                         const double* h, const ll_grid* grids, const ll_mg_params* base, const char* cache_path,
                         void* cuda_stream, ll_mg_params* chosen, int* keys_tuned) {
  if (count < 1 || !m_tilde || !alpha || !dt || !h || !grids || !chosen) return LL_EINVAL;
  ll_mg_params b;
  ll_mg_default_params(&b);
  if (base) b = *base;
  if (!valid_params(b) || b.precision == LL_MIXED_BF16) return LL_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!m_tilde[i] || !valid_problem(alpha[i], dt[i], h[i], grids[i])) return LL_EINVAL;
  try {
    return autotune(count, m_tilde, alpha, dt, h, grids, b, cache_path, cuda_stream, chosen, keys_tuned);
  } catch (Status st) {
    return st.code;
  } catch (std::bad_alloc&) {
    return LL_ENOMEM;
  }
}

int ll_mg_tune_octave(double dt, double h) {
  if (!(dt > 0) || !(h > 0) || !isfinite(dt) || !isfinite(h)) return INT_MIN;
  return tune_octave(dt, h);
}

int ll_mg_tune_lookup(const char* cache_path, ll_grid grid, double dt, double h, ll_mg_params* p) {
  if (!cache_path || !p || !(dt > 0) || !(h > 0)) return LL_EINVAL;
  auto c = tune_read(cache_path);
  auto it = c.find(tune_key(p->precision, grid, dt, h));
  if (it == c.end()) return 0;
  *p = tune_apply(*p, it->second);
  return 1;
}

int ll_mg_batch_setup_groups(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                             const double* h, const ll_grid* grids, const ll_mg_params* p, void* cuda_stream,
                             ll_mg_batch** out) {
  if (count < 1 || !m_tilde || !alpha || !dt || !h || !grids || !p || !out) return LL_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!m_tilde[i] || !valid_problem(alpha[i], dt[i], h[i], grids[i])) return LL_EINVAL;
    if (!valid_params(p[i]) || p[i].precision == LL_MIXED_BF16) return LL_EINVAL;
  }
  try {
    return batch_create_groups(count, m_tilde, alpha, dt, h, grids, p, cuda_stream, out);
  } catch (Status st) {
    return st.code;
  } catch (std::bad_alloc&) {
    return LL_ENOMEM;
  }
}

void ll_mg_batch_destroy(ll_mg_batch* B) { delete B; }

// ---------------------------------------------------------------------------
// adjoint: A^T solves and the vector-Jacobian product of one step
// ---------------------------------------------------------------------------
int ll_mg_adjoint_setup(const double* m_tilde, double alpha, double dt, double h, ll_grid grid,
                        const ll_mg_params* p, void* cuda_stream, ll_mg_batch** out) {
  if (!m_tilde || !out || !valid_problem(alpha, dt, h, grid)) return LL_EINVAL;
  if (p && !valid_params(*p)) return LL_EINVAL;
  if (p && (p->kcycle != 0 || p->precision == LL_MIXED_BF16)) return LL_EINVAL;
  const double* ms[1] = {m_tilde};
  return batch_create(1, ms, &alpha, &dt, &h, &grid, p, cuda_stream, out, true);
}

int ll_mg_step_vjp(ll_mg_batch* T, const double* m, double alpha, double dt, const double* x, const double* g,
                   double* m_bar, double* alpha_bar, double rtol, int* iterations, double* rel_residual) {
  if (!T || !T->transposed || T->ninst != 1 || !m || !x || !g || !m_bar) return LL_EINVAL;
  if (!(dt > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(alpha)) return LL_EINVAL;
  try {
    batch_enter(T);
    LL_CU(cudaStreamSynchronize(T->U->s));
    ll_mg_hierarchy* H = T->inst[0];
    cudaStream_t s = T->U->s;
    H->alpha = alpha;
    H->dt = dt;
    numeric(H, m);
    batch_refresh(T);
    long n = H->g.n;
    k_vjp_xbar<<<cdiv(n, kBlock), kBlock, 0, s>>>(n, x, g, H->stepb);
    LL_LAUNCHED();
    LL_CU(cudaMemsetAsync(H->stepx.p, 0, 3 * n * sizeof(double), s));
    const double* rhs[1] = {H->stepb.p};
    double* lam[1] = {H->stepx.p};
    int st1 = LL_OK;
    int rc = batch_solve(T, rhs, lam, rtol, iterations, rel_residual, &st1);
    k_vjp_param<<<kRedBlocks, kBlock, 0, s>>>(H->g.nx, H->g.ny, H->g.nz, m, x, H->stepx, alpha, 1.0 / dt,
                                              1.0 / (H->h * H->h), m_bar, H->partial);
    LL_LAUNCHED();
    k_finish<<<1, kBlock, 0, s>>>(H->partial, H->partial.p + kRedBlocks);
    LL_LAUNCHED();
    double a = 0;
    LL_CU(cudaMemcpyAsync(&a, H->partial.p + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    LL_CU(cudaStreamSynchronize(s));
    if (alpha_bar) *alpha_bar = -a;
    return rc;
  } catch (Status st) {
    return st.code;
  }
}

}  // extern "C"
