// tree.h -- Barnes-Hut octree build and traversal (Sec. 2.2): host interface.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "gs.h"

namespace gs {

// Workspace of the octree steps (owned by a context).
struct TreeWork {
  void* mem = nullptr;  // one allocation, carved into the arrays below
  size_t bytes = 0;
  int64_t cap_n = 0;    // points it was sized for
  bool adjoint = false;
  int64_t* d_counts = nullptr;  // interaction counters {point, node}
  void* lmem = nullptr;         // interaction lists (tree_impl.h BHLists)
  size_t lbytes = 0;
  int lcap = 0;                 // entries per list
  int lcap_req = 0;             // requested entries per list (0 = default)
};

// Inputs of one tree step: pack = scaled recentred FP32 positions and
// momenta (pair layout), raw = FP32 positions {x, y, z, 0}.
struct BHStep {
  int64_t N, Npad;
  double s;       // coordinate scale of the pack
  float thr;      // far threshold r*r (FP32)
  const float4* pack;
  const float4* raw;
};

cudaError_t tree_setup();
gs_status tree_reserve(TreeWork& w, int64_t N, bool adjoint, cudaStream_t st);
void tree_release(TreeWork& w);
// Builds the tree of one state (abpack = NULL in the forward stage).
gs_status bh_build(TreeWork& w, const BHStep& b, const float4* abpack, bool zero_counts,
                   cudaStream_t st);
// Walks the tree built last and records the interaction lists.
gs_status bh_walk(TreeWork& w, const BHStep& b, bool counts, cudaStream_t st);
// Evaluates the recorded lists (forward or backward stage) and applies the
// epilogue.
gs_status bh_eval_fwd(TreeWork& w, const BHStep& b, const FwdEpi& e, bool counts,
                      cudaStream_t st);
gs_status bh_eval_adj(TreeWork& w, const BHStep& b, const AdjEpi& e, bool counts,
                      cudaStream_t st);
void bh_counts(TreeWork& w, int64_t* cnt);
// Builds the tree on one state and exports it (see gs_tree in gs.h).
gs_status tree_export(TreeWork& w, const float4* raw, const float4* pack, int64_t N,
                      uint32_t* codes, int32_t* order, int32_t* nodes, float* range, int64_t cap,
                      int64_t* n_nodes, cudaStream_t st);
const char* bh_last_error();

}  // namespace gs
