// tree.h -- Barnes-Hut octree build and traversal (Sec. 2.2): host interface.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "gs.h"

namespace gs {

// Workspace of the octree steps (owned by a context).
// Shared scratch (sort buffers, source records, partial sums) plus `nslots`
// slots, each holding one step's tree and interaction lists so that the
// backward stage can reuse the forward stage's decisions for the same state.
struct TreeWork {
  void* mem = nullptr;   // shared scratch
  size_t bytes = 0;
  void* smem = nullptr;  // slots
  size_t slot_bytes = 0;
  int nslots = 0;
  int64_t cap_n = 0;     // points it was sized for
  int64_t cap_groups = 0; // walk groups it was sized for
  int64_t* d_counts = nullptr;  // interaction counters {point, node}
  int64_t lcap = 0;      // chunks in each slot's interaction-list pool
  int lcap_req = 0;      // requested entries per list (0 = budget-based pool)
  int lcap_from_req = 0; // the request the current allocation was made for
  int wsplit_req = 0;    // walk lists per slice: 0 = by tree size, else 1 or 2
  int* d_status = nullptr;  // device status word of the owning context
};

// Many independent point sets ("subjects") in one forest.  Subject s owns
// points [off[s], off[s+1]) in the input order and, after the sort (by
// subject, then Morton code), the same range of sorted positions; its own
// octree (quantised in its own bounding box) is a contiguous preorder range,
// and no node spans two subjects.  Walk groups hold up to 32 sorted points of
// one subject: {first sorted position, count, off[s], off[s+1]}.
struct BHForest {
  int S = 0;                        // 0: one point set (no forest)
  const int64_t* off = nullptr;     // S + 1 offsets (device)
  const int4* groups = nullptr;     // G walk groups (device)
  int G = 0;
  float* sbox = nullptr;            // 6 S floats: per-subject bounding boxes
  const double* centers = nullptr;  // S x 3 recentring points of the packs
};

// Inputs of one tree step: pack = scaled recentred FP32 positions and
// momenta (pair layout, entry = input index), raw = FP32 positions
// {x, y, z, 0}.
struct BHStep {
  int slot;       // tree slot of this step
  int64_t N, Npad;
  double s;       // coordinate scale of the pack
  float thr;      // far threshold r*r (FP32)
  const float4* pack;
  const float4* raw;
  BHForest f;
  int leaf = 1;   // leaf-size variant (1 = the paper's rule)
  bool trunc = false;  // pure truncation variant (far nodes dropped, pairs cut)
  int crit = 0;        // far test: 0 the paper's distance rule, 1 opening angle
};

cudaError_t tree_setup();
// groups: walk groups to provide for (0: ceil(N / 32), one point set)
gs_status tree_reserve(TreeWork& w, int64_t N, int slots, cudaStream_t st, int64_t groups = 0);
void tree_release(TreeWork& w);
// Builds the tree of one state (abpack = NULL in the forward stage).
gs_status bh_build(TreeWork& w, const BHStep& b, const float4* abpack, bool zero_counts,
                   cudaStream_t st);
// Recomputes the sums and source records of the tree stored in b.slot for
// new (p, alpha, beta) -- the backward stage of the same state reuses the
// forward stage's tree and lists.
gs_status bh_aggregate(TreeWork& w, const BHStep& b, const float4* abpack, bool zero_counts,
                       cudaStream_t st);
// Walks the tree in b.slot and records the interaction lists there.
gs_status bh_walk(TreeWork& w, const BHStep& b, bool counts, cudaStream_t st);
// Evaluates the recorded lists (forward or backward stage) and applies the
// epilogue.
gs_status bh_eval_fwd(TreeWork& w, const BHStep& b, const FwdEpi& e, bool counts,
                      cudaStream_t st);
gs_status bh_eval_adj(TreeWork& w, const BHStep& b, const AdjEpi& e, bool counts,
                      cudaStream_t st);
void bh_counts(TreeWork& w, int64_t* cnt);
// Per-target decision record of the tree in b.slot (one point set, not the
// truncation variant): tally = 5 N device int64, stats = NULL or 2 device
// int64 (see gs_bh_tally in gs.h).
gs_status bh_tally(TreeWork& w, const BHStep& b, int64_t* tally, int64_t* stats,
                   cudaStream_t st);

// Outside points (tracers, forward only) walking the tree of b.slot as
// targets: positions xraw (FP32, by index), records xrec (scaled, by index);
// tracer_order sorts them by Morton code in the tree's root box (scratch of
// tracer_scratch_bytes(M)) and picks each 32-tracer group's slice cut.  The
// tree's lists are overwritten.  The workspace must hold ceil(M/32) groups.
struct BHTargets {
  const float4* xraw = nullptr;
  const float4* xrec = nullptr;
  const uint32_t* xperm = nullptr;
  const int* xmid = nullptr;
  int64_t M = 0;
  int G = 0;
};
size_t tracer_scratch_bytes(int64_t M);
gs_status tracer_order(TreeWork& w, const BHStep& b, const float4* xraw, int64_t M,
                       void* scratch, BHTargets* out, cudaStream_t st);
gs_status bh_walk_targets(TreeWork& w, const BHStep& b, const BHTargets& x, cudaStream_t st);
// Evaluates the tracers' lists and applies the tracer epilogue.
gs_status bh_eval_targets(TreeWork& w, const BHStep& b, const BHTargets& x, const TracerEpi& e,
                          cudaStream_t st);
// Builds the tree on one state and exports it (see gs_tree in gs.h).
gs_status tree_export(TreeWork& w, const float4* raw, const float4* pack, int64_t N,
                      uint32_t* codes, int32_t* order, int32_t* nodes, float* range, int64_t cap,
                      int64_t* n_nodes, cudaStream_t st);
// Builds the tree on one state with its forward (abpack NULL) or adjoint
// sums and exports each node's sums in input units (see gs_tree_sums in
// gs.h); center, s, mu: the pack's recentring point (device), scale and
// beta scale.
gs_status tree_sums(TreeWork& w, const float4* raw, const float4* pack, const float4* abpack,
                    int64_t N, const double* center, double s, double mu, double* sums,
                    int64_t cap, int64_t* n_nodes, cudaStream_t st);
// Uniform-grid neighbour search of the truncation variant (GS_TRUNC with
// the "trunc_grid" option, one point set): cells of side 0.51 r (doubled
// until at most grid_cells(N) cells cover the FP32 bounding box), points
// sorted stably by cell in `scratch` (grid_scratch_bytes(N) bytes), then one
// right-hand side whose pairs are exactly those passing the truncation
// test.  counts: NULL or 2 device int64, set to {kept pairs, 0}.
size_t grid_scratch_bytes(int64_t N);
gs_status grid_rhs(void* scratch, int64_t N, const float4* raw, const float4* pack,
                   const float4* abpack, float r, float thr, bool adj, const FwdEpi& fe,
                   const AdjEpi& ae, int64_t* counts, cudaStream_t st);
const char* bh_last_error();

}  // namespace gs
