// Symbolic-setup routines (integer graph work on the GPU), see ll_setup.cu.
#pragma once

#include "ll_internal.cuh"

namespace llmg {

int exclusive_scan(const int* in, int* out, int n, cudaStream_t s);
void build_grid_graph(int nx, int ny, int nz, DevGraph& g, cudaStream_t s);
int matching_pass(const DevGraph& g, int rounds, uint32_t seed, int attach, int* group, cudaStream_t s);
void build_members(int n, const int* map, int nc, DBuf<int>& mptr, DBuf<int>& mem, cudaStream_t s);
void contract_graph(const DevGraph& g, const int* map, int nc, const int* mptr, const int* mem, DevGraph& out,
                    cudaStream_t s);
int aggregate_level(const DevGraph& g, int rounds, uint32_t seed, int* agg, cudaStream_t s);
int colour_graph(const DevGraph& g, uint32_t seed, int* colour, cudaStream_t s);
constexpr int kRowKeys = 256;        // distinct bucketed row-work keys (see row_work_keys)
constexpr int kRowKeysExact = 1024;  // distinct exact row-work keys
void row_work_keys(const DevGraph& g, const int* colour, bool exact, DBuf<int>& key, cudaStream_t s);
void colour_classes(int n, const int* colour, int ncol, const int* key, int nkeys, DBuf<int>& cptr, DBuf<int>& crow,
                    std::vector<int>& h_cptr, cudaStream_t s);
void order_by_length(int n, const int* sptr, DBuf<int>& perm, cudaStream_t s);
void bsr_pattern(const DevGraph& g, DBuf<int>& rowptr, DBuf<int>& col, DBuf<int>& diag, int& nnzb, cudaStream_t s);
void slot_map_level1(const GridGeom& g, const int* agg_nat, const DevGraph& g1, const int* rowptr, const int* col,
                     int nnzb, DBuf<int>& sptr, DBuf<int>& sidx, DBuf<int>& sw, cudaStream_t s);
void slot_map_bsr(int nf, const int* frp, const int* fcol, const int* agg, const int* crp, const int* ccol, int cnnzb,
                  DBuf<int>& sptr, DBuf<int>& sidx, cudaStream_t s);
void rb_maps(const GridGeom& g, const int* agg_nat, int* agg_rb, int* nat_of_slot, cudaStream_t s);
void members_colour0(int nc, const int* mptr, const int* mem, long nh, DBuf<int>& optr, DBuf<int>& out,
                     cudaStream_t s);
void permute_graph(const DevGraph& g, const int* n2o, const int* o2n, DevGraph& out, cudaStream_t s);
void invert_perm(int n, const int* n2o, int* o2n, cudaStream_t s);
void map_through(int n, const int* idx, const int* m1, const int* m2, int* out, cudaStream_t s);

}  // namespace llmg
