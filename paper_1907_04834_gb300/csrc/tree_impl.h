// tree_impl.h -- device-side layout of the Barnes-Hut octree shared by the
// build (tree.cu) and the traversal (traverse.cu) kernels.
//
// Points are sorted by 30-bit Morton code (10 levels; bit 3b+2 = x bit b).
// Nodes are stored in depth-first preorder, children in Morton order:
//   * an internal node is a cell that holds >= 2 points and has >= 2
//     non-empty child cells (a chain of single-child cells has the same
//     members and the same actual range as its lowest cell, so it takes the
//     same decision and the same summary: it is stored once), or a depth-10
//     cell holding >= 2 points (its children are its points);
//   * a leaf is one point.
// Node x's subtree occupies preorder indices [x, skip(x)); a leaf has
// skip = x + 1, so traversal is a forward scan that either steps into a node
// (x + 1) or jumps over it (skip(x)).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gs {

struct TreeArrays {
  // per point (capacity N)
  uint32_t* key;    // sorted Morton codes (after the sort)
  uint32_t* perm;   // sorted position -> original index
  uint32_t* key_alt;
  uint32_t* perm_alt;
  uint32_t* codes;  // Morton code per original index (before the sort)
  uint32_t* ssub;   // forest: subject of each sorted position
  uint32_t* mask;   // bit D set: an internal node of depth D starts here
  uint32_t* offs;   // N + 1: exclusive prefix count of internal nodes
  int32_t* own_a;   // per boundary i (between sorted i, i+1): node start or -1
  int32_t* own_b;   // node end (inclusive)
  // scratch
  uint32_t* hist;   // radix histograms / scan input
  uint32_t* hscan;  // scanned histograms
  uint32_t* bsum;   // scan block sums
  float* bbox_part; // per-block bounding boxes
  float* bbox;      // 6 floats: lo, hi
  // per node (capacity 2N), preorder index
  float4* nbox;     // 2 per node: {lo.xyz, skip (int bits)}, {hi.xyz, count (int bits)}
  float4* nrec;     // 4 per node: source record {xs}, {P}, {A}, {B / n}
  int2* nsc;        // {skip, count} written at build time
  int2* ninfo;      // {depth (-1 = leaf), first sorted position} (kept per step: the
                    // leaf-size variant's walk reads it, also when re-walking a kept tree)
  int32_t* nparent; // preorder id of the parent, -1 for the root
  int32_t* inode;   // internal nodes in preorder (kept per step): k-th -> its preorder id
  double* isum;     // 12 per node: sums of xs, p, a, b over members (FP32 pairs)
  // node sums over member ranges (scratch of each aggregation): per sorted
  // point its values (4 float4: xs, p, a, b) and FP32 position; per chunk of
  // 32 and of 1024 sorted points, the sums (12 FP32 pairs) and the range
  float4* spt;
  float4* sraw;
  float2* c1sum;
  float4* c1box;
  float2* c2sum;
  float4* c2box;
  int32_t* bigq;    // internal nodes of many range pieces, summed a warp each
  int32_t* bigc;    // their count
  int64_t* counts;  // {point interactions, node interactions}
  // single-pass sort and scan of one point set (zeroed together, os_bytes):
  uint32_t* os_hist;            // 3 x 1024 digit counts of the 30-bit codes
  int* os_ctr;                  // tile counters: 3 sort passes, the node-offset scan
  unsigned long long* os_stat;  // 3 passes x sort tiles x 1024 look-back words
  unsigned long long* sc_stat;  // scan tiles look-back words
  size_t os_bytes;
  int* status;      // the context's device status word (bounded waits record here)
};

// Interaction lists of one traversal.  A group of 32 points has BH_SLICES
// slices (node ranges) whose sums are kept apart and combined in a fixed
// order; the walk may split each slice into `wsplit` walk lists (walk slices
// per group wk = BH_SLICES * wsplit) to spread a small tree's walk over more
// warps.  The evaluation reads a slice's walk lists as one entry sequence in
// fixed batches, so the sums do not depend on the split.  Entries live
// in a pool of chunks of BH_CHUNK entries; a walk list is the chain of chunks
// starting at head[l] (next[c] links them in order).
constexpr int BH_SLICES = 4;
constexpr int BH_MAX_WK = 16;  // walk lists per group at most
// (256-entry chunks: measured 43.3 -> 42.4 ms per blobs100k gradient for the
// walk and the two evaluations together against 64-entry chunks)
constexpr int BH_CHUNK = 256;
struct BHLists {
  int2* ent;      // pool: n_chunks x BH_CHUNK entries {node, lane mask}
  int* next;      // per chunk: next chunk of the same list
  int* head;      // per walk list: first chunk
  int* len;       // per walk list: entries recorded
  int* ovf_x;     // per walk list: >= 0 if the pool ran out (its slice is re-walked)
  int* used;      // chunks taken from the pool (reset before each walk)
  int n_chunks;   // pool size
  float2* part;   // per slice x 9 x 32: partial sums of the slice (at most 9 components)
  float2* fb;     // per slice x 9 x 32: partial sums of a re-walked slice
  // Scheduling (never the results): order[k] is the slice the k-th warp of an
  // evaluation takes, longest first; worder is the longest-first order of the
  // last walk's lists, which the next walk of as many lists (*worder_n) takes
  // as its estimate of their cost.
  int* order;     // per slice (this step)
  int* worder;    // per walk list (shared by the steps)
  int* worder_n;  // list count of worder; -1 when it holds none
  int* gticket;   // per group: slices summed so far (the last one combines; back to 0)
  int* ohist;     // the orders' counts per class and block (2 x 256 x 256)
};

__device__ __forceinline__ int total_nodes(const TreeArrays& t, int N) {
  return N + (int)t.offs[N];
}

// A walk group: up to 32 consecutive sorted points of one point set, and the
// preorder node range [nb, ne) of that set's tree.  groups == NULL: one point
// set, group g = sorted points [32 g, 32 g + 32).
struct GroupInfo {
  int first, count, nb, ne;
  int mid;  // node at which the group's slices are cut (the leaf of its middle point)
};
__device__ __forceinline__ GroupInfo group_info(const TreeArrays& t, int N, const int4* groups,
                                                int g) {
  GroupInfo gi;
  if (!groups) {
    gi.first = g * 32;
    gi.count = min(32, N - gi.first);
    gi.nb = 0;
    gi.ne = total_nodes(t, N);
  } else {
    const int4 v = groups[g];
    gi.first = v.x;
    gi.count = v.y;
    gi.nb = v.z + (int)t.offs[v.z];
    gi.ne = v.w + (int)t.offs[v.w];
  }
  const int i = gi.first + min(16, gi.count - 1);
  gi.mid = i + (int)t.offs[i + 1];
  return gi;
}

// Three-input maximum (sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// FP32 distance-squared from a point to an axis-aligned box: per axis
// max(lo - x, 0, x - hi), then (dx*dx + dy*dy) + dz*dz, every operation
// rounded to nearest and none contracted; the x and y axes take packed f32x2
// subtractions and one packed product (same roundings).
__device__ __forceinline__ float box_dist2(float x, float y, float z, const float4& lo,
                                           const float4& hi) {
  const f2 p = f2_make(x, y);
  float ax, ay, bx, by;
  f2_split(f2_sub(f2_make(lo.x, lo.y), p), ax, ay);
  f2_split(f2_sub(p, f2_make(hi.x, hi.y)), bx, by);
  const float dx = fmax3(ax, 0.f, bx), dy = fmax3(ay, 0.f, by);
  const float dz = fmax3(__fsub_rn(lo.z, z), 0.f, __fsub_rn(z, hi.z));
  const f2 d = f2_make(dx, dy);
  float sx, sy;
  f2_split(f2_mul(d, d), sx, sy);
  return __fadd_rn(__fadd_rn(sx, sy), __fmul_rn(dz, dz));
}

// Unevaluated FP32 pair sums (hi + lo, hi the rounded sum): each addition is
// Knuth's TwoSum, which returns the rounding error of hi exactly, so a pair
// holds a sum with about twice FP32's precision at FP32 speed.
struct Pair {
  float hi, lo;
};
__device__ __forceinline__ void pair_add(Pair& s, float x) {
  const float t = __fadd_rn(s.hi, x);
  const float bp = __fsub_rn(t, s.hi);
  const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, e);
}
// adds a value given as (x, y) = x + y with |y| small (a pair, or a Kahan
// sum and its compensation)
__device__ __forceinline__ void pair_add(Pair& s, float2 v) {
  pair_add(s, v.x);
  s.lo = __fadd_rn(s.lo, v.y);
}
// hi + lo renormalised (|lo| <= ulp(hi) / 2), stored as (hi, lo)
__device__ __forceinline__ float2 pair_store(const Pair& s) {
  const float t = __fadd_rn(s.hi, s.lo);
  return make_float2(t, __fsub_rn(s.lo, __fsub_rn(t, s.hi)));
}
// the pair's value rounded to FP32
__device__ __forceinline__ float pair_value(const Pair& s) { return __fadd_rn(s.hi, s.lo); }

// Walk groups and, for a forest, the per-subject recentring points used by
// the forward epilogue.
struct WalkGroups {
  const int4* groups;      // NULL: one point set
  int G;                   // number of groups
  const int64_t* off;      // forest: S + 1 offsets
  int S;
  const double* centers;   // forest: S x 3
  int leaf;                // leaf-size variant: near nodes of <= leaf points taken exactly
  bool trunc;              // pure truncation: far nodes dropped, pairs cut at the threshold
  int crit;                // far test: 0 the paper's distance rule, 1 opening angle
  int wsplit;              // walk lists per slice: 1, 2 or 4
  // Outside targets (tracer points walking this tree, forward only); xperm
  // NULL: the targets are the tree's own points.  Tracer groups are 32
  // consecutive tracers in tracer-code order over the whole tree.
  const float4* xraw;      // FP32 positions {x, y, z, 0} by tracer index
  const float4* xrec;      // scaled records {xs, ys, zs, 0} by tracer index
  const uint32_t* xperm;   // sorted tracer position -> tracer index
  const int* xmid;         // per group: the node at which its slices are cut
  int xM;                  // number of tracers
};

// Group g of the targets described by wg (tree points or outside tracers).
__device__ __forceinline__ GroupInfo target_group(const TreeArrays& t, int N, const WalkGroups& wg,
                                                  int g) {
  if (!wg.xperm) return group_info(t, N, wg.groups, g);
  GroupInfo gi;
  gi.first = g * 32;
  gi.count = min(32, wg.xM - gi.first);
  gi.nb = 0;
  gi.ne = total_nodes(t, N);
  gi.mid = wg.xmid[g];
  return gi;
}

// counts: NULL or 2 int64 accumulating {point, node} interactions.
// scheduled: take the lists in the previous walk's longest-first order (when
// it has as many lists), then sort this walk's lists by length into L.order
// and L.worder.  Only the order in which warps take lists changes, never a
// result.
cudaError_t launch_bh_walk(const TreeArrays& t, int N, const float4* raw, float thr,
                           const BHLists& L, const WalkGroups& wg, int64_t* counts,
                           bool scheduled, cudaStream_t st);
// Decision record of every target of one point set (no truncation): tally
// (5 N int64, zeroed by the caller) accumulates per original index {point
// interactions, node interactions, fingerprint sums of each, nodes reached}
// -- the walk's own decisions, recorded instead of listed; stats (NULL or 2
// int64, zeroed by the caller) accumulates the walk's warp iterations and
// list entries.
cudaError_t launch_bh_tally(const TreeArrays& t, int N, const float4* raw, float thr,
                            const WalkGroups& wg, int64_t* tally, int64_t* stats,
                            cudaStream_t st);
// fallback for overflowed lists, evaluation, fixed-order combine + epilogue;
// scheduled: evaluate in L.order (written by a scheduled walk of these lists)
cudaError_t launch_bh_eval(const TreeArrays& t, int N, const float4* raw, float thr,
                           const BHLists& L, const WalkGroups& wg, bool adj, const FwdEpi& fe,
                           const AdjEpi& ae, const TracerEpi& te, int64_t* counts,
                           bool scheduled, cudaStream_t st);

// Uniform cell grid of the truncation variant (device views; see grid_build
// in tree.h).  Points sorted stably by cell id (z * ny + y) * nx + x; cell c
// holds sorted positions [cstart[c], cstart[c + 1]).  Cells have side
// h >= 0.51 r, so two points within r of each other lie at most
// GRID_REACH cells apart per axis.
constexpr int GRID_REACH = 2;
struct GridView {
  const uint32_t* perm = nullptr;  // N: sorted position -> input index
  const uint32_t* key = nullptr;   // N: cell id per sorted position
  const int* cstart = nullptr;     // C + 1 (C = dims[3])
  const int* dims = nullptr;       // {nx, ny, nz, C}
};
// One warp per 32 consecutive sorted points: sources are the points of the
// cells within GRID_REACH cells of any of them (row by row), cut by the
// truncation test; fixed-order sums, then the epilogue.  counts: NULL or 2
// int64 accumulating {kept pairs, 0}.
cudaError_t launch_grid_eval(const GridView& g, int N, const float4* pack, const float4* abpack,
                             const float4* raw, float thr, bool adj, const FwdEpi& fe,
                             const AdjEpi& ae, int64_t* counts, cudaStream_t st);

}  // namespace gs
