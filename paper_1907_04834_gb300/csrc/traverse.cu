// traverse.cu -- Barnes-Hut traversal of Sec. 2.2 (Fig. 1), forward (Eq. 4
// and the momentum-dot replacement) and backward (alpha, beta replaced by
// their node averages), for groups of 32 Morton-consecutive points.
//
// Every lane applies its own point's rule at each node it reaches (three
// cases of Sec. 2.2):
//   leaf                          -> exact interaction with that point;
//   internal, range farther than the threshold -> one interaction with the
//                                    node summary; the lane then ignores the
//                                    node's subtree (resume = skip);
//   internal, otherwise           -> open the node.
// Nodes are in depth-first preorder, so a group walks the node array forward,
// stepping into a node when any lane opens it and jumping to skip otherwise.
// A lane's interactions are exactly those of its own recursive traversal.
//
// Pure truncation (a variant, not the paper's approximation): far boxes are
// dropped instead of summarised, and the evaluation keeps only the pairs
// whose FP32 raw positions pass the same test as the far rule applied to
// the two points (d2 <= r*r); a point's distance to its leaf's box is never
// below the box distance in FP32, so dropping far boxes loses no such pair.
//
// Leaf-size variant (leaf > 1): a node holding at most `leaf` points that a
// lane does not find far is taken exactly, all of its points at once,
// instead of being opened; its points are emitted as point entries (~i for
// sorted point i) that the evaluation maps to their leaf records.  leaf = 1
// is the paper's rule.
//
// Two phases:
//   walk     -- decisions only, few registers.  A group's node range is cut
//               into BH_SLICES slices around the group's own leaves, and each
//               slice is walked by one or two warps (walk lists); a walk that
//               starts inside the range first tests the ancestors of its
//               first node, which gives every lane the state it would have
//               there.  Each walk list is an ordered list of (node, lane mask)
//               entries; runs of consecutive leaves are appended in one step
//               (a lane changes activity only at its resume point, so a run is
//               cut there).
//   evaluate -- one warp per slice streams the entries of the slice's walk
//               lists in batches of TR_CAP, stages the source records in
//               shared memory and evaluates two sources per f32x2 instruction
//               (a far node acts as one source at its centroid with momentum
//               P, derivative A and momentum derivative B/n).
// A slice one of whose walk lists outgrew its capacity is walked again by a
// fused walk+evaluate kernel that batches entries exactly as the list
// evaluation does, so results do not depend on the capacity, nor on how
// many walk lists a slice was split into.  Partial sums are combined in a
// fixed order: results are deterministic.
#include <climits>

#include "kernels.h"
#include "tree_impl.h"

namespace gs {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// One warp per block: a block's slot frees as soon as its walk list or slice
// is done, and the next one (longest first) starts there.  Measured on
// blobs100k against four warps per block: walk 18.1 -> 16.0 ms and adjoint
// evaluation 18.1 -> 17.6 ms per gradient (forward evaluation unchanged);
// two warps per block, or warps taking walk lists from a common cursor,
// 18.2 ms.
constexpr int TR_WARPS = 1;
constexpr int WK_WARPS = 1;
constexpr int TR_CAP = 128;  // evaluation batch (entries staged at a time)

// Per-lane own data (record of the lane's point).
struct Own {
  int i, o;  // sorted position, original index
  bool valid;
  float4 m0, m1, m2, m3;  // record: xs, p, a, b
  float rx, ry, rz;       // FP32 raw position (truncation test)
};

__device__ __forceinline__ Own load_own(const TreeArrays& t, const WalkGroups& wg,
                                        const GroupInfo& gi, int lane, bool adj) {
  Own w;
  w.i = gi.first + lane;
  w.valid = lane < gi.count;
  const int ii = w.valid ? w.i : gi.first;
  if (wg.xperm) {  // an outside target: its record, no momentum
    w.o = (int)wg.xperm[ii];
    w.m0 = wg.xrec[w.o];
    w.m1 = make_float4(0.f, 0.f, 0.f, 0.f);
    w.m2 = w.m1;
    w.m3 = w.m1;
    const float4 r = wg.xraw[w.o];
    w.rx = r.x, w.ry = r.y, w.rz = r.z;
    return w;
  }
  w.o = (int)t.perm[ii];
  const int leaf = ii + (int)t.offs[ii + 1];
  w.m0 = t.nrec[4 * leaf];
  w.m1 = t.nrec[4 * leaf + 1];
  w.m2 = make_float4(0.f, 0.f, 0.f, 0.f);
  w.m3 = w.m2;
  if (adj) {
    w.m2 = t.nrec[4 * leaf + 2];
    w.m3 = t.nrec[4 * leaf + 3];
  }
  const float4 rb = t.nbox[2 * leaf];  // a leaf's box is its point
  w.rx = rb.x, w.ry = rb.y, w.rz = rb.z;
  return w;
}

// Far test of a node for point (x, y, z).  crit 0 (the paper's rule): the
// FP32 distance to the actual range exceeds r (thr = r*r).  crit 1
// (opening-angle variant): s*s < theta^2 * d2 with s the largest side of the
// range, d2 the squared FP32 distance to its centre (lo + hi) * 0.5 and
// thr = theta^2, each operation rounded.
__device__ __forceinline__ bool far_test(float x, float y, float z, const float4& lo,
                                         const float4& hi, float thr, int crit) {
  if (crit == 0) return box_dist2(x, y, z, lo, hi) > thr;
  const float s = fmaxf(fmaxf(__fsub_rn(hi.x, lo.x), __fsub_rn(hi.y, lo.y)),
                        __fsub_rn(hi.z, lo.z));
  const float dx = __fsub_rn(x, __fmul_rn(__fadd_rn(lo.x, hi.x), 0.5f));
  const float dy = __fsub_rn(y, __fmul_rn(__fadd_rn(lo.y, hi.y), 0.5f));
  const float dz = __fsub_rn(z, __fmul_rn(__fadd_rn(lo.z, hi.z), 0.5f));
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  return __fmul_rn(s, s) < __fmul_rn(thr, d2);
}

// Truncation test of a pair in FP32: (dx*dx + dy*dy) + dz*dz <= thr, each
// operation rounded, no contraction.
__device__ __forceinline__ bool within(float ax, float ay, float az, float bx, float by, float bz,
                                       float thr) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) <= thr;
}

// Cut k (0 <= k <= 8) of the group's node range [nb, ne) into eight walk
// slices: nb, then L - D 2^(3-k) for k = 1, 2, 3, L, and L + D 2^(k-5) for
// k = 5, 6, 7 (clamped to the range), then ne, with L the leaf of the
// group's middle point and D = clamp((ne - nb) / 32, 256, 4096): narrow
// slices near the group, where the walk opens most nodes.
__device__ __forceinline__ int walk_cut8(const GroupInfo& gi, int k) {
  if (k <= 0) return gi.nb;
  if (k >= 8) return gi.ne;
  const int mid = gi.mid;
  const int D = min(max((gi.ne - gi.nb) >> 5, 256), 4096);
  if (k < 4) return max(gi.nb, mid - (D << (3 - k)));
  if (k == 4) return mid;
  return min(gi.ne, mid + (D << (k - 5)));
}

// Cut k (0 <= k <= wk) of the group's node range into wk = 4, 8 or 16 walk
// slices: for 4 the even cuts of the eight, for 16 the eight and the
// midpoints between them.  The evaluation's four slices [cut 0, cut wk/4),
// ... are the same node ranges whatever wk is.  Any cut points give the
// same interactions; finer walk slices only spread a group's walk over more
// warps, so that no single long walk holds the GPU at the end of a launch.
// The cuts depend only on the current tree, so results are reproducible.
__device__ __forceinline__ int walk_cut(const GroupInfo& gi, int k, int wk) {
  if (wk == 16) {
    const int a = walk_cut8(gi, k >> 1);
    return (k & 1) ? (a + walk_cut8(gi, (k >> 1) + 1)) >> 1 : a;
  }
  return walk_cut8(gi, k * (8 / wk));
}

// Slice evaluated by warp `wl` of a launch over all G * BH_SLICES slices
// when no longest-first order is given: the warps of one block take the same
// slice of consecutive groups (lists of similar length), the last slices --
// on average the longest -- first.
__device__ __forceinline__ int list_of_warp(int wl, int G) {
  return (wl % G) * BH_SLICES + (BH_SLICES - 1 - wl / G);
}

// True if a walk list of slice e (walk lists e*wsplit .. +wsplit-1, walk
// lists numbered g*wk + k) ran out of pool: the fallback evaluates it.
__device__ __forceinline__ bool slice_overflowed(const BHLists& L, int e, int wsplit) {
  bool o = false;
  for (int j = 0; j < wsplit; j++) o = o || L.ovf_x[e * wsplit + j] >= 0;
  return o;
}

// Resume point of this lane at node s: test the ancestors of s from the root
// down; the first one this lane finds far, or (leaf-size variant) near but
// of at most `leaf` points -- taken whole by the slice that visits it --
// makes it skip past s.
template <bool VAR>
__device__ int resume_at(const TreeArrays& t, int s, float rx, float ry, float rz, float thr,
                         int leaf, int crit, int resume) {
  // Tested bottom-up; ancestors' subtrees nest, so the highest qualifying
  // ancestor -- the first one found from the root down -- has the largest
  // skip.
  int r = resume;
  for (int a = t.nparent[s]; a >= 0; a = t.nparent[a]) {
    const float4 lo = t.nbox[2 * a], hi = t.nbox[2 * a + 1];
    const bool far = VAR ? far_test(rx, ry, rz, lo, hi, thr, crit)
                         : box_dist2(rx, ry, rz, lo, hi) > thr;
    if (far | (VAR && __float_as_int(hi.w) <= leaf)) r = max(r, __float_as_int(lo.w));
  }
  return r;
}

// ------------------------------------------------------------------ evaluation
// Staged source records: per source the record's components (6 forward,
// 12 adjoint), then for truncation the FP32 raw position (3); NS of them,
// rounded up to even.  Paired layout: sources e, e + 1 (e even) of components
// c, c + 1 (c even) form one 16-byte word {c:e, c:e+1, c+1:e, c+1:e+1}, so
// one shared load gives two components of two sources, each an f32x2
// operand (the exact kernels' pack layout).  Otherwise component-major
// (stride TR_CAP), one 8-byte load per component of two sources.  Measured
// on blobs100k: paired forward 9.26 -> 9.00 ms per gradient, paired adjoint
// 17.34 -> 17.96 ms (128 registers against 123), so only the forward pairs.
template <bool ADJ, bool TRUNC>
struct Soa {
  static constexpr bool kPaired = !ADJ;
  static constexpr int NS = ((ADJ ? 12 : 6) + (TRUNC ? 3 : 0) + 1) & ~1;
  static __device__ __forceinline__ int at(int c, int e) {
    return kPaired ? ((e >> 1) * (NS >> 1) + (c >> 1)) * 4 + (c & 1) * 2 + (e & 1)
                   : c * TR_CAP + e;
  }
  // components 2g, 2g + 1 of sources e, e + 1 (e even)
  static __device__ __forceinline__ ulonglong2 ld(const float* soa, int g, int e) {
    if constexpr (kPaired) {
      return reinterpret_cast<const ulonglong2*>(soa)[(e >> 1) * (NS >> 1) + g];
    } else {
      const f2* a = reinterpret_cast<const f2*>(soa + 2 * g * TR_CAP + e);
      return make_ulonglong2(a[0], a[TR_CAP / 2]);
    }
  }
};

template <bool ADJ>
struct Acc {
  static constexpr int NC = ADJ ? 9 : 6;
  Kahan K[NC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < NC; c++) K[c].zero();
  }
};

// Evaluates sources e in [0, n) (n even) whose records are staged in soa
// (Soa layout) and whose lane masks are in mask[] (8-byte aligned).
// TRUNC: the raw positions follow the record components in soa; a pair is
// also dropped unless it passes the truncation test, and npair counts the
// pairs kept.
template <bool ADJ, bool TRUNC>
__device__ __forceinline__ void eval_batch(Acc<ADJ>& A, const float* soa, const unsigned* mask,
                                           int n, int lane, const Own& me, float thr,
                                           int& npair) {
  using S = Soa<ADJ, TRUNC>;
  constexpr int NR = ADJ ? 12 : 6;
  const uint2* mp = reinterpret_cast<const uint2*>(mask);
  // whether this lane takes sources e and e + 1
  auto keep = [&](int e, bool& b0, bool& b1) {
    const uint2 m = mp[e >> 1];
    b0 = (m.x >> lane) & 1u;
    b1 = (m.y >> lane) & 1u;
    if constexpr (TRUNC) {
      b0 = b0 && within(me.rx, me.ry, me.rz, soa[S::at(NR, e)], soa[S::at(NR + 1, e)],
                        soa[S::at(NR + 2, e)], thr);
      b1 = b1 && within(me.rx, me.ry, me.rz, soa[S::at(NR, e + 1)], soa[S::at(NR + 1, e + 1)],
                        soa[S::at(NR + 2, e + 1)], thr);
      npair += (b0 ? 1 : 0) + (b1 ? 1 : 0);
    }
  };
  const f2 X = f2_dup(me.m0.x), Y = f2_dup(me.m0.y), Z = f2_dup(me.m0.z);
  const f2 U = f2_dup(me.m1.x), V = f2_dup(me.m1.y), W = f2_dup(me.m1.z);
  if constexpr (!ADJ) {
    f2 fx = 0, fy = 0, fz = 0, hx = 0, hy = 0, hz = 0;
#pragma unroll 2
    for (int e = 0; e < n; e += 2) {
      bool b0, b1;
      keep(e, b0, b1);
      const ulonglong2 q0 = S::ld(soa, 0, e), q1 = S::ld(soa, 1, e), q2 = S::ld(soa, 2, e);
      const f2 dx = f2_sub(X, q0.x), dy = f2_sub(Y, q0.y), dz = f2_sub(Z, q1.x);
      f2 r = f2_mul(dx, dx);
      r = f2_fma(dy, dy, r);
      r = f2_fma(dz, dz, r);
      float r0, r1;
      f2_split(r, r0, r1);
      const f2 g = f2_make(b0 ? ex2_neg(r0) : 0.f, b1 ? ex2_neg(r1) : 0.f);
      const f2 PX = q1.y, PY = q2.x, PZ = q2.y;
      fx = f2_fma(g, PX, fx);
      fy = f2_fma(g, PY, fy);
      fz = f2_fma(g, PZ, fz);
      f2 c = f2_mul(U, PX);
      c = f2_fma(V, PY, c);
      c = f2_fma(W, PZ, c);
      const f2 cg = f2_mul(c, g);
      hx = f2_fma(cg, dx, hx);
      hy = f2_fma(cg, dy, hy);
      hz = f2_fma(cg, dz, hz);
    }
    A.K[0].add(f2_sum(fx));
    A.K[1].add(f2_sum(fy));
    A.K[2].add(f2_sum(fz));
    A.K[3].add(f2_sum(hx));
    A.K[4].add(f2_sum(hy));
    A.K[5].add(f2_sum(hz));
  } else {
    // the three adjoint sums A13', A2', B' (beta scaled in the records)
    const f2 AX = f2_dup(me.m2.x), AY = f2_dup(me.m2.y), AZ = f2_dup(me.m2.z);
    const f2 BX = f2_dup(me.m3.x), BY = f2_dup(me.m3.y), BZ = f2_dup(me.m3.z);
    f2 ax = 0, ay = 0, az = 0, a2x = 0, a2y = 0, a2z = 0, bx = 0, by = 0, bz = 0;
    for (int e = 0; e < n; e += 2) {
      bool b0, b1;
      keep(e, b0, b1);
      const ulonglong2 q0 = S::ld(soa, 0, e), q1 = S::ld(soa, 1, e), q2 = S::ld(soa, 2, e);
      const ulonglong2 q3 = S::ld(soa, 3, e), q4 = S::ld(soa, 4, e), q5 = S::ld(soa, 5, e);
      const f2 dx = f2_sub(X, q0.x), dy = f2_sub(Y, q0.y), dz = f2_sub(Z, q1.x);
      f2 r = f2_mul(dx, dx);
      r = f2_fma(dy, dy, r);
      r = f2_fma(dz, dz, r);
      float r0, r1;
      f2_split(r, r0, r1);
      const f2 g = f2_make(b0 ? ex2_neg(r0) : 0.f, b1 ? ex2_neg(r1) : 0.f);
      const f2 PX = q1.y, PY = q2.x, PZ = q2.y;
      const f2 QX = q3.x, QY = q3.y, QZ = q4.x;  // a_j (or A)
      f2 c = f2_mul(U, PX);
      c = f2_fma(V, PY, c);
      c = f2_fma(W, PZ, c);
      f2 sa = f2_mul(AX, PX);  // a_i . p_j
      sa = f2_fma(AY, PY, sa);
      sa = f2_fma(AZ, PZ, sa);
      sa = f2_fma(QX, U, sa);  // + a_j . p_i
      sa = f2_fma(QY, V, sa);
      sa = f2_fma(QZ, W, sa);
      const f2 wx = f2_sub(BX, q4.y), wy = f2_sub(BY, q5.x), wz = f2_sub(BZ, q5.y);
      f2 wd = f2_mul(wx, dx);
      wd = f2_fma(wy, dy, wd);
      wd = f2_fma(wz, dz, wd);
      const f2 cg = f2_mul(c, g);
      a2x = f2_fma(cg, wx, a2x);
      a2y = f2_fma(cg, wy, a2y);
      a2z = f2_fma(cg, wz, a2z);
      const f2 kap = f2_fma(cg, wd, f2_mul(g, sa));
      ax = f2_fma(kap, dx, ax);
      ay = f2_fma(kap, dy, ay);
      az = f2_fma(kap, dz, az);
      bx = f2_fma(g, f2_fma(wd, PX, QX), bx);
      by = f2_fma(g, f2_fma(wd, PY, QY), by);
      bz = f2_fma(g, f2_fma(wd, PZ, QZ), bz);
    }
    A.K[0].add(f2_sum(ax));
    A.K[1].add(f2_sum(ay));
    A.K[2].add(f2_sum(az));
    A.K[3].add(f2_sum(a2x));
    A.K[4].add(f2_sum(a2y));
    A.K[5].add(f2_sum(a2z));
    A.K[6].add(f2_sum(bx));
    A.K[7].add(f2_sum(by));
    A.K[8].add(f2_sum(bz));
  }
}

// Stages the records of queued nodes[0, n) into soa (padding n to even);
// TRUNC: also their FP32 raw positions (entries are leaves then).
template <bool ADJ, bool TRUNC>
__device__ __forceinline__ int stage_records(const TreeArrays& t, const int* nodes,
                                             unsigned* mask, float* soa, int n, int lane) {
  using S = Soa<ADJ, TRUNC>;
  constexpr int NR = ADJ ? 12 : 6;
  for (int e = lane; e < n; e += 32) {
    int nd = nodes[e];
    if (nd < 0) nd = ~nd + (int)t.offs[~nd + 1];  // point entry -> its leaf
    const float4 r0 = t.nrec[4 * nd], r1 = t.nrec[4 * nd + 1];
    soa[S::at(0, e)] = r0.x, soa[S::at(1, e)] = r0.y, soa[S::at(2, e)] = r0.z;
    soa[S::at(3, e)] = r1.x, soa[S::at(4, e)] = r1.y, soa[S::at(5, e)] = r1.z;
    if constexpr (ADJ) {
      const float4 r2 = t.nrec[4 * nd + 2], r3 = t.nrec[4 * nd + 3];
      soa[S::at(6, e)] = r2.x, soa[S::at(7, e)] = r2.y, soa[S::at(8, e)] = r2.z;
      soa[S::at(9, e)] = r3.x, soa[S::at(10, e)] = r3.y;
      soa[S::at(11, e)] = r3.z;
    }
    if constexpr (TRUNC) {
      const float4 rb = t.nbox[2 * nd];
      soa[S::at(NR, e)] = rb.x, soa[S::at(NR + 1, e)] = rb.y;
      soa[S::at(NR + 2, e)] = rb.z;
    }
  }
  if (n & 1) {
    if (lane == 0) mask[n] = 0u;
    if (lane < S::NS) soa[S::at(lane, n)] = 0.f;
    n++;
  }
  return n;
}

// ------------------------------------------------------------------ walk
// Walks nodes [x, end) for one group.  At each node the lanes still active
// (no summarised ancestor) take their decision; `sink` receives runs of
// entries (first node, count, lane mask): a summarised node, a run of
// consecutive leaves, or -- when an opened node's children are all leaves --
// those children at once.  sink.full() true (checked once per node) stops
// the walk; returns false if stopped.
// VAR = false compiles the paper's rule only (leaf and trunc ignored).
template <bool COUNT, bool VAR, class Sink>
__device__ __forceinline__ bool walk_nodes(const TreeArrays& t, float4 (*sbox)[2], int& x,
                                           int end, const float4& rr, float thr, int leaf,
                                           bool trunc, int crit, int& resume, Sink& sink,
                                           int lane, long long& np, long long& nn) {
  int base = INT_MIN / 2;
  // window bit masks (bit j = node base + j): leaf, "all children leaves"
  unsigned leafmask = 0u, botmask = 0u;
  while (x < end) {
    if (sink.full()) return false;
    sink.step();
    int off = x - base;
    if ((unsigned)off >= 32u) {  // stage the next 32 node boxes
      __syncwarp();
      base = x;
      off = 0;
      const int j = base + lane;
      bool lf = false, bt = false;
      if (j < end) {
        const float4 lo = t.nbox[2 * j], hi = t.nbox[2 * j + 1];
        sbox[lane][0] = lo;
        sbox[lane][1] = hi;
        const int sk = __float_as_int(lo.w), cn = __float_as_int(hi.w);
        lf = sk == j + 1;
        // children all leaves, at most 32 of them, subtree inside the range
        bt = !lf && sk - j == cn + 1 && cn <= 32 && sk <= end;
      }
      leafmask = __ballot_sync(FULL, lf);
      botmask = __ballot_sync(FULL, bt);
      __syncwarp();
    }
    if ((leafmask >> off) & 1u) {
      // a run of consecutive leaves; lanes change activity only at their
      // resume points, so the run is cut at the first one inside it
      const unsigned rest = ~(leafmask >> off);
      int r = rest ? __ffs(rest) - 1 : 32 - off;
      const int rmin = __reduce_min_sync(FULL, resume > x ? resume : INT_MAX);
      r = min(r, rmin - x);
      const unsigned mk = __ballot_sync(FULL, resume <= x);
      if (mk) {
        if (r == 1) sink.add1(x, mk);
        else sink.add(x, r, mk, false);
        if (COUNT && !(VAR && trunc)) np += (long long)__popc(mk) * r;
      }
      x += r;
      continue;
    }
    const float4 bl = sbox[off][0], bh = sbox[off][1];
    const int skip = __float_as_int(bl.w);
    const bool active = x >= resume;
    sink.reach(active);
    // (bitwise &: the test is computed on every lane, no branch; measured
    // 5% faster than the short-circuit form)
    const bool far = active & (VAR ? far_test(rr.x, rr.y, rr.z, bl, bh, thr, crit)
                                   : box_dist2(rr.x, rr.y, rr.z, bl, bh) > thr);
    const unsigned mt = __ballot_sync(FULL, far), mo = __ballot_sync(FULL, active && !far);
    // an opened node whose children are all leaves: take them at once; a
    // node of at most `leaf` points (leaf-size variant): take its points
    const int ncount = __float_as_int(bh.w);
    const bool bottom = mo && ((botmask >> off) & 1u);
    const bool bucket = VAR && mo && !bottom && ncount <= leaf;
    // (truncation: a far node is dropped, not summarised)
    const unsigned ms = (VAR && trunc) ? 0u : mt;
    if (ms | ((bottom || bucket) ? 1u : 0u)) {
      const int cn = (bottom || bucket) ? ncount : 0;
      if (ms) sink.add1(x, ms);
      if (bottom) sink.add(x + 1, cn, mo, false);
      if (bucket) sink.add(t.ninfo[x].y, cn, mo, true);
      if (COUNT && !(VAR && trunc)) nn += __popc(mt), np += (long long)__popc(mo) * cn;
    }
    if (far) resume = skip;
    x = (mo && !bottom && !bucket) ? x + 1 : skip;
  }
  return true;
}

// Sink of the list walk: entries buffered in shared memory and written to
// the list BH_CHUNK at a time in chunks taken from the pool.  When the pool
// is exhausted the list is abandoned (the slice is re-walked later).
constexpr int kReserve = 2;  // chunks reserved from the pool at a time
struct ListSink {
  const BHLists* L;
  int2* buf;     // 2 * BH_CHUNK entries in shared memory
  int head, tail, written, cnt, lane;
  bool ovf;
  int res_next, res_end;  // chunks reserved by this warp, not yet used
  __device__ __forceinline__ bool full() const { return ovf; }
  __device__ __forceinline__ void step() {}
  __device__ __forceinline__ void reach(bool) {}
  __device__ __forceinline__ void put_chunk(int n) {
    if (ovf) return;
    if (res_next == res_end) {
      int c = 0;
      if (lane == 0) c = atomicAdd(L->used, kReserve);
      c = __shfl_sync(FULL, c, 0);
      res_next = c;
      res_end = c + kReserve;
    }
    const int c = res_next++;
    if (c >= L->n_chunks) {
      ovf = true;
      return;
    }
    int2* dst = L->ent + (size_t)c * BH_CHUNK;
    for (int e = lane; e < n; e += 32) dst[e] = buf[e];
    if (lane == 0) {
      if (tail < 0) head = c;
      else L->next[tail] = c;
    }
    tail = c;
    written += n;
  }
  // n <= 32 entries (a leaf run, a node's children or points, or one node),
  // so at most one chunk fills per call; points: entries ~(node0 + k)
  __device__ __forceinline__ void add(int node0, int n, unsigned mask, bool points) {
    const int c2 = cnt + n;
    auto enc = [&](int k) { return points ? ~(node0 + k) : node0 + k; };
    if (lane < n && cnt + lane < BH_CHUNK) buf[cnt + lane] = make_int2(enc(lane), (int)mask);
    if (c2 < BH_CHUNK) {
      cnt = c2;
      return;
    }
    __syncwarp();
    put_chunk(BH_CHUNK);
    __syncwarp();
    const int rest = c2 - BH_CHUNK;
    if (lane < rest) buf[lane] = make_int2(enc((n - rest) + lane), (int)mask);
    cnt = rest;
  }
  // one entry (a far node: the most frequent case), written by lane 0
  __device__ __forceinline__ void add1(int node, unsigned mask) {
    if (lane == 0) buf[cnt] = make_int2(node, (int)mask);
    if (++cnt < BH_CHUNK) return;
    __syncwarp();
    put_chunk(BH_CHUNK);
    __syncwarp();
    cnt = 0;
  }
  // hands the first BH_CHUNK buffered entries over and moves the others
  // (at most BH_CHUNK) to the front
  __device__ __forceinline__ void flush_front() {
    __syncwarp();
    put_chunk(BH_CHUNK);
    const int rest = cnt - BH_CHUNK;
    int2 v0 = make_int2(0, 0), v1 = make_int2(0, 0);
    if (lane < rest) v0 = buf[BH_CHUNK + lane];
    if (lane + 32 < rest) v1 = buf[BH_CHUNK + 32 + lane];
    __syncwarp();
    if (lane < rest) buf[lane] = v0;
    if (lane + 32 < rest) buf[32 + lane] = v1;
    __syncwarp();
    cnt = rest;
  }
  __device__ __forceinline__ void finish() {
    __syncwarp();
    while (cnt >= BH_CHUNK && !ovf) flush_front();
    if (cnt && !ovf) put_chunk(cnt);
    cnt = 0;
  }
};

// The list walk of the paper's rule (leaf size 1, distance criterion, no
// truncation): the decisions and entries of walk_nodes<false, false>, in
// the same order, appended by predicated stores to the sink's two-chunk
// buffer (a node adds at most 33 entries) and handed over a chunk at a
// time.  Returns false if the list pool ran out.
__device__ __forceinline__ bool walk_paper(const TreeArrays& t, float4 (*sbox)[2], int& x,
                                           int end, const float4& rr, float thr, int& resume,
                                           ListSink& sink, int lane) {
  int base = INT_MIN / 2;
  unsigned leafmask = 0u, botmask = 0u;
  int2* buf = sink.buf;
  while (x < end) {
    if (sink.cnt >= BH_CHUNK) {
      sink.flush_front();
      if (sink.ovf) return false;
    }
    int off = x - base;
    if ((unsigned)off >= 32u) {  // stage the next 32 node boxes
      __syncwarp();
      base = x;
      off = 0;
      const int j = base + lane;
      bool lf = false, bt = false;
      if (j < end) {
        const float4 lo = t.nbox[2 * j], hi = t.nbox[2 * j + 1];
        sbox[lane][0] = lo;
        sbox[lane][1] = hi;
        const int sk = __float_as_int(lo.w), cn = __float_as_int(hi.w);
        lf = sk == j + 1;
        bt = !lf && sk - j == cn + 1 && cn <= 32 && sk <= end;
      }
      leafmask = __ballot_sync(FULL, lf);
      botmask = __ballot_sync(FULL, bt);
      __syncwarp();
    }
    const int cnt = sink.cnt;
    if ((leafmask >> off) & 1u) {
      // a run of consecutive leaves, cut at the first resume point in it
      const unsigned rest = ~(leafmask >> off);
      int r = rest ? __ffs(rest) - 1 : 32 - off;
      const int rmin = __reduce_min_sync(FULL, resume > x ? resume : INT_MAX);
      r = min(r, rmin - x);
      const unsigned mk = __ballot_sync(FULL, resume <= x);
      if (mk && lane < r) buf[cnt + lane] = make_int2(x + lane, (int)mk);
      sink.cnt = cnt + (mk ? r : 0);
      x += r;
      continue;
    }
    const float4 bl = sbox[off][0], bh = sbox[off][1];
    const int skip = __float_as_int(bl.w);
    const bool active = x >= resume;
    const bool far = active & (box_dist2(rr.x, rr.y, rr.z, bl, bh) > thr);
    const unsigned mt = __ballot_sync(FULL, far), mo = __ballot_sync(FULL, active && !far);
    const bool bottom = mo && ((botmask >> off) & 1u);
    // the summary entry, then (an opened node whose children are all
    // leaves) those children at once
    if (mt && lane == 0) buf[cnt] = make_int2(x, (int)mt);
    const int c1 = cnt + (mt ? 1 : 0);
    const int cn = bottom ? __float_as_int(bh.w) : 0;
    if (lane < cn) buf[c1 + lane] = make_int2(x + 1 + lane, (int)mo);
    sink.cnt = c1 + cn;
    if (far) resume = skip;
    x = (mo && !bottom) ? x + 1 : skip;
  }
  return true;
}

// Walk list l of one group slice: emits its ordered interaction list.
template <bool COUNT, bool VAR>
__device__ __forceinline__ void walk_list(const TreeArrays& t, int N, const float4* raw,
                                          float thr, const BHLists& L, const WalkGroups& wg,
                                          int64_t* counts, int l, int wk, float4 (*sbox)[2],
                                          int2* ent, int lane) {
  const int g = l / wk, k = l % wk;
  const GroupInfo gi = target_group(t, N, wg, g);
  const bool valid = lane < gi.count;
  const int ti = gi.first + (valid ? lane : 0);
  const float4 rr = wg.xperm ? wg.xraw[wg.xperm[ti]] : raw[(int)t.perm[ti]];
  int x = walk_cut(gi, k, wk);
  const int end = walk_cut(gi, k + 1, wk);
  int resume = valid ? 0 : INT_MAX;
  // (an empty slice may start at the node count: no node to test there)
  if (k > 0 && valid && x < end)
    resume = resume_at<VAR>(t, x, rr.x, rr.y, rr.z, thr, wg.leaf, wg.crit, resume);
  ListSink sink{&L, ent, -1, -1, 0, 0, lane, false, 0, 0};
  long long np = 0, nn = 0;
  bool done;
  if (!COUNT && !VAR)
    done = walk_paper(t, sbox, x, end, rr, thr, resume, sink, lane);
  else
    done = walk_nodes<COUNT, VAR>(t, sbox, x, end, rr, thr, wg.leaf, wg.trunc, wg.crit, resume,
                                  sink, lane, np, nn);
  sink.finish();
  done = done && !sink.ovf;
  if (lane == 0) {
    L.head[l] = sink.head;
    L.len[l] = sink.written;
    L.ovf_x[l] = done ? -1 : x;
  }
  if (COUNT && done && lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)np);
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[1]), (unsigned long long)nn);
  }
}

// The list walk, one warp per walk list: the wl-th in the order `word` (when
// it holds as many lists as this walk has; else in index order).
template <bool COUNT, bool VAR>
__global__ void __launch_bounds__(WK_WARPS * 32)
    k_bh_walk(TreeArrays t, int N, const float4* __restrict__ raw, float thr, BHLists L,
              WalkGroups wg, int64_t* counts, const int* __restrict__ word) {
  __shared__ float4 s_box[WK_WARPS][32][2];
  __shared__ int2 s_ent[WK_WARPS][2 * BH_CHUNK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wk = BH_SLICES * wg.wsplit;
  const int nl = wg.G * wk;
  const bool ordered = word && *L.worder_n == nl;
  const int wl = blockIdx.x * WK_WARPS + w;
  if (wl >= nl) return;
  walk_list<COUNT, VAR>(t, N, raw, thr, L, wg, counts, ordered ? word[wl] : wl, wk, s_box[w],
                        s_ent[w], lane);
}

// ------------------------------------------------------------------ tally
// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the generator's output for state `key`.
__device__ __forceinline__ unsigned long long mix64(unsigned long long key) {
  unsigned long long z = key + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Sink of the decision record: per lane, the number of points and nodes the
// lane takes and the sums (mod 2^64) of mix64(key) over them, key = (first
// sorted position << 32) | member count -- the same sources give the same
// record whatever the order.  Entries are those the list walk emits: one
// entry (a far node or a single leaf), or n point entries (a leaf run, an
// all-leaf node's children, or a leaf-size bucket's points).
struct TallySink {
  const TreeArrays* t;
  int lane;
  long long np, nn, nr;       // this lane's points, nodes, nodes reached
  unsigned long long hp, hn;
  long long iters, entries;   // the warp's walk iterations and list entries
  __device__ __forceinline__ bool full() const { return false; }
  __device__ __forceinline__ void step() { iters++; }
  __device__ __forceinline__ void reach(bool active) { nr += active ? 1 : 0; }
  __device__ __forceinline__ void add1(int node, unsigned mask) {
    entries++;
    if (!((mask >> lane) & 1u)) return;
    const int skip = __float_as_int(t->nbox[2 * node].w);
    const int cnt = __float_as_int(t->nbox[2 * node + 1].w);
    const unsigned long long key =
        ((unsigned long long)(unsigned)t->ninfo[node].y << 32) | (unsigned)cnt;
    if (skip == node + 1) np++, hp += mix64(key);  // a leaf: one point
    else nn++, hn += mix64(key);
  }
  __device__ __forceinline__ void add(int node0, int n, unsigned mask, bool points) {
    entries += n;
    if (!((mask >> lane) & 1u)) return;
    for (int k = 0; k < n; k++) {
      const int pos = points ? node0 + k : t->ninfo[node0 + k].y;
      np++;
      hp += mix64(((unsigned long long)(unsigned)pos << 32) | 1u);
    }
  }
};

// Decision record of every target (tests): one warp per walk list, exactly
// the walk of k_bh_walk (slice cuts, ancestor test at the slice start, the
// same walk_nodes), with the tally sink in place of the list; per target
// tally[4 o + {0, 1, 2, 3}] += {points, nodes, point sum, node sum}.
template <bool VAR>
__global__ void __launch_bounds__(TR_WARPS * 32)
    k_bh_tally(TreeArrays t, int N, const float4* __restrict__ raw, float thr, WalkGroups wg,
               unsigned long long* tally, unsigned long long* stats) {
  __shared__ float4 s_box[TR_WARPS][32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wk = BH_SLICES * wg.wsplit;
  const int l = blockIdx.x * TR_WARPS + w;
  if (l >= wg.G * wk) return;
  const int g = l / wk, k = l % wk;
  const GroupInfo gi = target_group(t, N, wg, g);
  const bool valid = lane < gi.count;
  const int ti = gi.first + (valid ? lane : 0);
  const int o = (int)t.perm[ti];
  const float4 rr = raw[o];
  int x = walk_cut(gi, k, wk);
  const int end = walk_cut(gi, k + 1, wk);
  int resume = valid ? 0 : INT_MAX;
  if (k > 0 && valid && x < end)
    resume = resume_at<VAR>(t, x, rr.x, rr.y, rr.z, thr, wg.leaf, wg.crit, resume);
  TallySink sink{&t, lane, 0, 0, 0, 0ull, 0ull, 0, 0};
  long long np = 0, nn = 0;
  walk_nodes<false, VAR>(t, s_box[w], x, end, rr, thr, wg.leaf, false, wg.crit, resume, sink,
                         lane, np, nn);
  if (stats && lane == 0) {
    atomicAdd(&stats[0], (unsigned long long)sink.iters);
    atomicAdd(&stats[1], (unsigned long long)sink.entries);
  }
  if (!valid) return;
  atomicAdd(&tally[5 * (size_t)o + 0], (unsigned long long)sink.np);
  atomicAdd(&tally[5 * (size_t)o + 1], (unsigned long long)sink.nn);
  atomicAdd(&tally[5 * (size_t)o + 2], sink.hp);
  atomicAdd(&tally[5 * (size_t)o + 3], sink.hn);
  atomicAdd(&tally[5 * (size_t)o + 4], (unsigned long long)sink.nr);
}

// ------------------------------------------------------------------ combine
// Group g once all its slices are summed: per point (one lane each) the
// slices' partial sums in slice order as FP32 pairs, then the FP64 epilogue.
template <bool ADJ>
__device__ __forceinline__ void combine_group(const TreeArrays& t, int N, const BHLists& L,
                                              const WalkGroups& wg, int g, int lane,
                                              const FwdEpi& fe, const AdjEpi& ae,
                                              const TracerEpi& te) {
  constexpr int NC = Acc<ADJ>::NC;
  const GroupInfo gi = target_group(t, N, wg, g);
  if (lane >= gi.count) return;
  const int i = gi.first + lane;
  Pair S[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) S[c] = Pair{0.f, 0.f};
  for (int k = 0; k < BH_SLICES; k++) {
    const int l = g * BH_SLICES + k;
    const float2* src = slice_overflowed(L, l, wg.wsplit) ? L.fb : L.part;
#pragma unroll
    for (int c = 0; c < NC; c++) pair_add(S[c], __ldcg(&src[((size_t)l * NC + c) * 32 + lane]));
  }
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) acc[c] = (double)S[c].hi + (double)S[c].lo;
  if (wg.xperm) {  // tracer targets: the velocity of Eq. 3 is the F part
    if constexpr (!ADJ) tracer_epilogue(wg.xperm[i], acc, te);
    return;
  }
  const int o = (int)t.perm[i];
  if constexpr (!ADJ) {
    // a forest's subjects have their own recentring points
    const double* c = wg.centers ? wg.centers + 3 * subject_of(wg.off, wg.S, o) : fe.center;
    fwd_epilogue_at(o, o, c, acc, acc + 3, fe);
  } else {
    adj_epilogue(o, acc, acc + 3, acc + 6, ae);
  }
}

// Called by a warp that has written the partial sums of one slice of group
// g (list evaluation or fallback): the group's ticket counts its finished
// slices, and the warp that finishes the last one combines the group (each
// writer fences its sums before counting, the combiner after).
template <bool ADJ>
__device__ __forceinline__ void finish_slice(const TreeArrays& t, int N, const BHLists& L,
                                             const WalkGroups& wg, int g, int lane,
                                             const FwdEpi& fe, const AdjEpi& ae,
                                             const TracerEpi& te) {
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) {
    last = atomicAdd(&L.gticket[g], 1) == BH_SLICES - 1;
    if (last) L.gticket[g] = 0;
  }
  if (!__shfl_sync(FULL, last, 0)) return;
  __threadfence();
  combine_group<ADJ>(t, N, L, wg, g, lane, fe, ae, te);
}

// ------------------------------------------------------------------ evaluate
// One warp per slice: partial sums of its entries, part[(e*NC + c)*32 + lane].
// The entries of the slice's walk lists are read as one sequence, TR_CAP
// at a time (256 against 128 entries: forward faster, adjoint slower, the
// two together about the same), so the batches (and the sums) are those of
// an unsplit walk.  The adjoint variant is held
// to 128 registers (16 warps per SM): measured faster than 12 at 168.
template <bool ADJ, bool TRUNC>
__global__ void __launch_bounds__(TR_WARPS * 32, ADJ ? 16 / TR_WARPS : 1)
    k_bh_eval(TreeArrays t, int N, BHLists L, WalkGroups wg, float thr, int64_t* counts,
              const int* __restrict__ order, FwdEpi fe, AdjEpi ae, TracerEpi te) {
  constexpr int NS = Soa<ADJ, TRUNC>::NS;
  constexpr int NC = Acc<ADJ>::NC;
  __shared__ __align__(16) float s_soa[TR_WARPS][NS * TR_CAP];
  __shared__ int s_node[TR_WARPS][TR_CAP];
  __shared__ __align__(16) unsigned s_mask[TR_WARPS][TR_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wl = blockIdx.x * TR_WARPS + w;
  if (wl >= wg.G * BH_SLICES) return;
  const int e = order ? order[wl] : list_of_warp(wl, wg.G);
  const int ws = wg.wsplit, l0 = e * ws;
  if (slice_overflowed(L, e, ws)) return;  // evaluated whole by the fallback
  const Own me = load_own(t, wg, target_group(t, N, wg, e / BH_SLICES), lane, ADJ);
  Acc<ADJ> A;
  A.zero();
  int npair = 0;
  int n = 0;
  for (int j = 0; j < ws; j++) n += L.len[l0 + j];
  // reader state: walk list j, its current chunk, offset there, entries left
  int j = 0, chunk = L.head[l0], off = 0, left = L.len[l0];
  for (int c0 = 0; c0 < n; c0 += TR_CAP) {
    const int cn = min(TR_CAP, n - c0);
    __syncwarp();
    for (int got = 0; got < cn;) {
      while (left == 0) {  // next walk list of the slice (entries remain)
        j++;
        chunk = L.head[l0 + j];
        off = 0;
        left = L.len[l0 + j];
      }
      const int take = min(min(BH_CHUNK - off, left), cn - got);
      const int2* src = L.ent + (size_t)chunk * BH_CHUNK + off;
      for (int q = lane; q < take; q += 32) {
        const int2 v = src[q];
        s_node[w][got + q] = v.x;
        s_mask[w][got + q] = (unsigned)v.y;
      }
      got += take;
      off += take;
      left -= take;
      if (off == BH_CHUNK && left > 0) {
        chunk = L.next[chunk];
        off = 0;
      }
    }
    __syncwarp();
    const int ce = stage_records<ADJ, TRUNC>(t, s_node[w], s_mask[w], s_soa[w], cn, lane);
    __syncwarp();
    eval_batch<ADJ, TRUNC>(A, s_soa[w], s_mask[w], ce, lane, me, thr, npair);
  }
#pragma unroll
  for (int c = 0; c < NC; c++) L.part[((size_t)e * NC + c) * 32 + lane] = A.K[c].out();
  if (TRUNC && counts) {
    const int tot = __reduce_add_sync(FULL, (unsigned)npair);
    if (lane == 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)tot);
  }
  finish_slice<ADJ>(t, N, L, wg, e / BH_SLICES, lane, fe, ae, te);
}

// ------------------------------------------------------------------ fallback
// Sink that evaluates queued entries in place, in batches of TR_CAP entries
// aligned exactly like the list evaluation's batches, so a slice gives the
// same sums whichever path evaluates it.
template <bool ADJ, bool TRUNC>
struct EvalSink {
  const TreeArrays* t;
  int* node;
  unsigned* mask;
  float* soa;
  Acc<ADJ>* A;
  const Own* me;
  int cnt, lane;
  float thr;
  int npair;
  __device__ __forceinline__ bool full() const { return false; }
  __device__ __forceinline__ void step() {}
  __device__ __forceinline__ void reach(bool) {}
  __device__ __forceinline__ void flush() {
    __syncwarp();
    const int ce = stage_records<ADJ, TRUNC>(*t, node, mask, soa, cnt, lane);
    __syncwarp();
    eval_batch<ADJ, TRUNC>(*A, soa, mask, ce, lane, *me, thr, npair);
    __syncwarp();
    cnt = 0;
  }
  __device__ __forceinline__ void add1(int node, unsigned mk) { add(node, 1, mk, false); }
  __device__ __forceinline__ void add(int node0, int n, unsigned mk, bool points) {
    while (n > 0) {
      const int take = min(n, TR_CAP - cnt);
      if (lane < take) {
        node[cnt + lane] = points ? ~(node0 + lane) : node0 + lane;
        mask[cnt + lane] = mk;
      }
      cnt += take;
      node0 += take;
      n -= take;
      if (cnt == TR_CAP) flush();
    }
  }
};

// Evaluates a slice one of whose walk lists overflowed: walks the slice
// again, its walk slices one after the other with the lanes' state carried
// over (the same entries as one walk over the slice), and evaluates in
// place; partial sums go to L.fb[(e*NC + c)*32 + lane].  COUNT: a walk
// list's interactions are counted here only if that list overflowed (the
// walk counted the others).
template <bool ADJ, bool COUNT, bool TRUNC>
__global__ void __launch_bounds__(TR_WARPS * 32)
    k_bh_fallback(TreeArrays t, int N, const float4* __restrict__ raw, float thr, BHLists L,
                  WalkGroups wg, int64_t* counts, FwdEpi fe, AdjEpi ae, TracerEpi te) {
  constexpr int NS = Soa<ADJ, TRUNC>::NS;
  constexpr int NC = Acc<ADJ>::NC;
  __shared__ float4 s_box[TR_WARPS][32][2];
  __shared__ __align__(16) float s_soa[TR_WARPS][NS * TR_CAP];
  __shared__ int s_node[TR_WARPS][TR_CAP];
  __shared__ __align__(16) unsigned s_mask[TR_WARPS][TR_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (blockIdx.x * TR_WARPS + w >= wg.G * BH_SLICES) return;
  const int e = list_of_warp(blockIdx.x * TR_WARPS + w, wg.G);
  const int ws = wg.wsplit, wk = BH_SLICES * ws;
  if (!slice_overflowed(L, e, ws)) return;
  const int g = e / BH_SLICES, k0 = (e % BH_SLICES) * ws;
  const GroupInfo gi = target_group(t, N, wg, g);
  const Own me = load_own(t, wg, gi, lane, ADJ);
  const float4 rr = wg.xperm ? make_float4(me.rx, me.ry, me.rz, 0.f) : raw[me.o];
  int x = walk_cut(gi, k0, wk);
  int resume = me.valid ? 0 : INT_MAX;
  if (k0 > 0 && me.valid && x < walk_cut(gi, k0 + ws, wk))
    resume = resume_at<true>(t, x, rr.x, rr.y, rr.z, thr, wg.leaf, wg.crit, resume);
  Acc<ADJ> A;
  A.zero();
  EvalSink<ADJ, TRUNC> sink{&t, s_node[w], s_mask[w], s_soa[w], &A, &me, 0, lane, thr, 0};
  long long np = 0, nn = 0;
  for (int j = 0; j < ws; j++) {
    long long pj = 0, qj = 0;
    walk_nodes<COUNT, true>(t, s_box[w], x, walk_cut(gi, k0 + j + 1, wk), rr, thr, wg.leaf,
                            TRUNC, wg.crit, resume, sink, lane, pj, qj);
    if (L.ovf_x[e * ws + j] >= 0) np += pj, nn += qj;
  }
  if (sink.cnt) sink.flush();
#pragma unroll
  for (int c = 0; c < NC; c++) L.fb[((size_t)e * NC + c) * 32 + lane] = A.K[c].out();
  if (COUNT && TRUNC) {  // pairs kept by the truncation test
    const int tot = __reduce_add_sync(FULL, (unsigned)sink.npair);
    if (lane == 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)tot);
  } else if (COUNT && lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)np);
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[1]), (unsigned long long)nn);
  }
  finish_slice<ADJ>(t, N, L, wg, g, lane, fe, ae, te);
}

// Longest-first orders of the walk lists (worder, and *worder_n = nw) and of
// the nw / ws slices (order; a slice's length is that of its ws walk lists
// together): a counting sort on length classes of about 12% width (the
// leading bit and the three below it: 8 classes per octave, monotone in the
// length), over up to kOrderMaxBlocks blocks per order, each a contiguous
// range of items: per block and class the counts (k_order_count), their
// exclusive scan in class-then-block order (k_order_scan), then each block
// places its items from its offsets (k_order_place).  Items of one class
// land in any order; every item appears once.  (One block per order took
// 21 us per walk at N = 10^5 and 133 us at N = 10^6.)
constexpr int kOrderThreads = 256, kOrderClasses = 256, kOrderMaxBlocks = 256;
constexpr int kOrderPer = 2048;  // items per block at least (up to kOrderMaxBlocks blocks)
__device__ __forceinline__ int len_class(int v) {
  if (v < 16) return max(v, 0);
  const int e = 31 - __clz(v);  // >= 4
  return min(kOrderClasses - 1, 16 + 8 * (e - 4) + ((v >> (e - 3)) & 7));
}
__host__ __device__ __forceinline__ int order_blocks(int n) {
  return max(1, min(kOrderMaxBlocks, (n + kOrderPer - 1) / kOrderPer));
}
// order `kind` (0: walk lists, 1: slices): its item count, lists per item,
// blocks, and block b's item range
struct OrderPart {
  int n, per, B, i0, i1;
  __device__ OrderPart(int kind, int nw, int ws, int b) {
    n = kind ? nw / ws : nw;
    per = kind ? ws : 1;
    B = order_blocks(n);
    const int chunk = (n + B - 1) / B;
    i0 = min(n, b * chunk);
    i1 = min(n, i0 + chunk);
  }
  // class index kOrderClasses - 1 - class: longest first
  __device__ int cls(const int* len, int e) const {
    int v = 0;
    for (int j = 0; j < per; j++) v += len[e * per + j];
    return kOrderClasses - 1 - len_class(v);
  }
};

// grid (order blocks of the walk lists, 2): per block and class, the count
// of its items;
// hist[kind][c * B + b]
__global__ void __launch_bounds__(kOrderThreads)
    k_order_count(const int* __restrict__ len, int nw, int ws, int* hist) {
  __shared__ int s_c[kOrderClasses];
  const int kind = blockIdx.y, tid = threadIdx.x;
  const OrderPart P(kind, nw, ws, blockIdx.x);
  if ((int)blockIdx.x >= P.B) return;
  for (int c = tid; c < kOrderClasses; c += kOrderThreads) s_c[c] = 0;
  __syncthreads();
  for (int e = P.i0 + tid; e < P.i1; e += kOrderThreads) atomicAdd(&s_c[P.cls(len, e)], 1);
  __syncthreads();
  int* h = hist + (size_t)kind * kOrderClasses * kOrderMaxBlocks;
  for (int c = tid; c < kOrderClasses; c += kOrderThreads) h[c * P.B + blockIdx.x] = s_c[c];
}

// one block per order: exclusive scan of its kOrderClasses x B counts (each
// thread a contiguous run of them)
__global__ void __launch_bounds__(kOrderThreads) k_order_scan(int nw, int ws, int* hist) {
  __shared__ int s_w[kOrderThreads / 32];
  const int kind = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const OrderPart P(kind, nw, ws, 0);
  int* h = hist + (size_t)kind * kOrderClasses * kOrderMaxBlocks;
  const int m = kOrderClasses * P.B, run = (m + kOrderThreads - 1) / kOrderThreads;
  const int a = min(m, tid * run), b = min(m, a + run);
  int loc = 0;
  for (int k = a; k < b; k++) loc += h[k];
  int inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < wid; k++) before += s_w[k];
  int s = before + inc - loc;
  for (int k = a; k < b; k++) {
    const int c = h[k];
    h[k] = s;
    s += c;
  }
}

// grid as k_order_count: each block places its items from its offsets
__global__ void __launch_bounds__(kOrderThreads)
    k_order_place(const int* __restrict__ len, int nw, int ws, const int* __restrict__ hist,
                  int* order, int* worder, int* worder_n) {
  __shared__ int s_c[kOrderClasses];
  const int kind = blockIdx.y, tid = threadIdx.x;
  const OrderPart P(kind, nw, ws, blockIdx.x);
  if ((int)blockIdx.x >= P.B) return;
  const int* h = hist + (size_t)kind * kOrderClasses * kOrderMaxBlocks;
  for (int c = tid; c < kOrderClasses; c += kOrderThreads) s_c[c] = h[c * P.B + blockIdx.x];
  __syncthreads();
  int* out = kind ? order : worder;
  for (int e = P.i0 + tid; e < P.i1; e += kOrderThreads) out[atomicAdd(&s_c[P.cls(len, e)], 1)] = e;
  if (kind == 0 && blockIdx.x == 0 && tid == 0) *worder_n = nw;
}

inline unsigned warp_blocks(int64_t warps) { return (unsigned)((warps + TR_WARPS - 1) / TR_WARPS); }

// ------------------------------------------------------------------ grid
// Truncation over the uniform cell grid.  Warp g takes the sorted points
// [32 g, 32 g + 32) as targets (consecutive in cell order: nearly always one
// or two cells) and sweeps the cells within GRID_REACH of the warp's cell
// range one (z, y) row at a time -- a row of cells is one contiguous range of
// sorted positions -- staging TR_CAP sources at a time from the packs.  Every
// staged source carries a full lane mask: the list evaluation's truncation
// test decides each pair, and counts the kept ones.  Sums in row order, then
// the epilogue.
template <bool ADJ>
__global__ void __launch_bounds__(TR_WARPS * 32)
    k_grid_eval(GridView gv, int N, const float4* __restrict__ pack,
                const float4* __restrict__ abpack, const float4* __restrict__ raw, float thr,
                int64_t* counts, FwdEpi fe, AdjEpi ae) {
  using S = Soa<ADJ, true>;
  constexpr int NR = ADJ ? 12 : 6, NS = S::NS;
  constexpr int NC = Acc<ADJ>::NC;
  __shared__ __align__(16) float s_soa[TR_WARPS][NS * TR_CAP];
  __shared__ __align__(16) unsigned s_mask[TR_WARPS][TR_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int first = (blockIdx.x * TR_WARPS + w) * 32;
  if (first >= N) return;  // the whole warp
  const int cnt = min(32, N - first);
  const bool valid = lane < cnt;
  const int sp = first + (valid ? lane : cnt - 1);
  const int o = (int)gv.perm[sp];
  Own me;
  me.i = sp;
  me.o = o;
  me.valid = valid;
  {
    float a[3], b[3];
    pack_read(pack, o, a, b);
    me.m0 = make_float4(a[0], a[1], a[2], 0.f);
    me.m1 = make_float4(b[0], b[1], b[2], 0.f);
    me.m2 = make_float4(0.f, 0.f, 0.f, 0.f);
    me.m3 = me.m2;
    if (ADJ) {
      pack_read(abpack, o, a, b);
      me.m2 = make_float4(a[0], a[1], a[2], 0.f);
      me.m3 = make_float4(b[0], b[1], b[2], 0.f);
    }
    const float4 r = raw[o];
    me.rx = r.x, me.ry = r.y, me.rz = r.z;
  }
  const int nx = gv.dims[0], ny = gv.dims[1], nz = gv.dims[2];
  const uint32_t key = gv.key[sp];
  const unsigned cx = key % (uint32_t)nx, cy = (key / (uint32_t)nx) % (uint32_t)ny,
                 cz = key / ((uint32_t)nx * (uint32_t)ny);
  const int x0 = max((int)__reduce_min_sync(FULL, cx) - GRID_REACH, 0);
  const int x1 = min((int)__reduce_max_sync(FULL, cx) + GRID_REACH, nx - 1);
  const int y0 = max((int)__reduce_min_sync(FULL, cy) - GRID_REACH, 0);
  const int y1 = min((int)__reduce_max_sync(FULL, cy) + GRID_REACH, ny - 1);
  const int z0 = max((int)__reduce_min_sync(FULL, cz) - GRID_REACH, 0);
  const int z1 = min((int)__reduce_max_sync(FULL, cz) + GRID_REACH, nz - 1);
  Acc<ADJ> A;
  A.zero();
  int npair = 0;
  float* soa = s_soa[w];
  unsigned* mask = s_mask[w];
  for (int z = z0; z <= z1; z++)
    for (int y = y0; y <= y1; y++) {
      const int row = (z * ny + y) * nx;  // < C <= 2^30
      const int s0 = gv.cstart[row + x0], s1 = gv.cstart[row + x1 + 1];
      for (int b0 = s0; b0 < s1; b0 += TR_CAP) {
        const int n = min(TR_CAP, s1 - b0);
        __syncwarp();
        for (int e = lane; e < n; e += 32) {
          const int so = (int)gv.perm[b0 + e];
          float a[3], b[3];
          pack_read(pack, so, a, b);
          for (int c = 0; c < 3; c++) soa[S::at(c, e)] = a[c], soa[S::at(3 + c, e)] = b[c];
          if (ADJ) {
            pack_read(abpack, so, a, b);
            for (int c = 0; c < 3; c++)
              soa[S::at(6 + c, e)] = a[c], soa[S::at(9 + c, e)] = b[c];
          }
          const float4 r = raw[so];
          soa[S::at(NR, e)] = r.x, soa[S::at(NR + 1, e)] = r.y;
          soa[S::at(NR + 2, e)] = r.z;
          mask[e] = FULL;
        }
        int ne = n;
        if (n & 1) {  // pad to an even count with an entry no lane takes
          if (lane == 0) mask[n] = 0u;
          if (lane < NS) soa[S::at(lane, n)] = 0.f;
          ne++;
        }
        __syncwarp();
        eval_batch<ADJ, true>(A, soa, mask, ne, lane, me, thr, npair);
      }
    }
  if (counts) {
    long long tot = valid ? npair : 0;
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_down_sync(FULL, tot, d);
    if (lane == 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)tot);
  }
  if (!valid) return;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    const float2 v = A.K[c].out();
    acc[c] = (double)v.x + (double)v.y;
  }
  if constexpr (!ADJ) fwd_epilogue_at(o, o, fe.center, acc, acc + 3, fe);
  else adj_epilogue(o, acc, acc + 3, acc + 6, ae);
}

}  // namespace

cudaError_t launch_bh_walk(const TreeArrays& t, int N, const float4* raw, float thr,
                           const BHLists& L, const WalkGroups& wg, int64_t* counts,
                           bool scheduled, cudaStream_t st) {
  const int nl = wg.G * BH_SLICES * wg.wsplit;
  const unsigned nb = (unsigned)((nl + WK_WARPS - 1) / WK_WARPS);
  const bool var = wg.leaf > 1 || wg.trunc || wg.crit != 0;  // the paper's rule: lean walk
  // the previous walk's order (taken if it covers as many lists)
  const int* word = scheduled ? L.worder : nullptr;
  if (counts && var)
    k_bh_walk<true, true><<<nb, WK_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, word);
  else if (counts)
    k_bh_walk<true, false><<<nb, WK_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, word);
  else if (var)
    k_bh_walk<false, true><<<nb, WK_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, word);
  else
    k_bh_walk<false, false><<<nb, WK_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, word);
  if (scheduled) {
    const dim3 grid(order_blocks(nl), 2);
    k_order_count<<<grid, kOrderThreads, 0, st>>>(L.len, nl, wg.wsplit, L.ohist);
    k_order_scan<<<2, kOrderThreads, 0, st>>>(nl, wg.wsplit, L.ohist);
    k_order_place<<<grid, kOrderThreads, 0, st>>>(L.len, nl, wg.wsplit, L.ohist, L.order,
                                                   L.worder, L.worder_n);
  }
  note_launches(scheduled ? 4 : 1);
  return cudaGetLastError();
}

cudaError_t launch_bh_tally(const TreeArrays& t, int N, const float4* raw, float thr,
                            const WalkGroups& wg, int64_t* tally, int64_t* stats,
                            cudaStream_t st) {
  const unsigned nb = warp_blocks((int64_t)wg.G * BH_SLICES * wg.wsplit);
  auto* out = reinterpret_cast<unsigned long long*>(tally);
  auto* sts = reinterpret_cast<unsigned long long*>(stats);
  if (wg.leaf > 1 || wg.crit != 0)
    k_bh_tally<true><<<nb, TR_WARPS * 32, 0, st>>>(t, N, raw, thr, wg, out, sts);
  else
    k_bh_tally<false><<<nb, TR_WARPS * 32, 0, st>>>(t, N, raw, thr, wg, out, sts);
  note_launches(1);
  return cudaGetLastError();
}

template <bool ADJ, bool TRUNC>
static void eval_launch(const TreeArrays& t, int N, const float4* raw, float thr,
                        const BHLists& L, const WalkGroups& wg, const FwdEpi& fe,
                        const AdjEpi& ae, const TracerEpi& te, int64_t* counts,
                        const int* order, cudaStream_t st) {
  const unsigned nb = warp_blocks((int64_t)wg.G * BH_SLICES);
  // list evaluation, then the fallback for overflowed slices; the warp that
  // finishes a group's last slice (in either kernel) combines the group
  k_bh_eval<ADJ, TRUNC><<<nb, TR_WARPS * 32, 0, st>>>(t, N, L, wg, thr, counts, order, fe, ae,
                                                      te);
  if (counts)
    k_bh_fallback<ADJ, true, TRUNC>
        <<<nb, TR_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, fe, ae, te);
  else
    k_bh_fallback<ADJ, false, TRUNC>
        <<<nb, TR_WARPS * 32, 0, st>>>(t, N, raw, thr, L, wg, counts, fe, ae, te);
}

cudaError_t launch_bh_eval(const TreeArrays& t, int N, const float4* raw, float thr,
                           const BHLists& L, const WalkGroups& wg, bool adj, const FwdEpi& fe,
                           const AdjEpi& ae, const TracerEpi& te, int64_t* counts,
                           bool scheduled, cudaStream_t st) {
  const int* ord = scheduled ? L.order : nullptr;
  if (wg.trunc) {
    if (!adj) eval_launch<false, true>(t, N, raw, thr, L, wg, fe, ae, te, counts, ord, st);
    else eval_launch<true, true>(t, N, raw, thr, L, wg, fe, ae, te, counts, ord, st);
  } else {
    if (!adj) eval_launch<false, false>(t, N, raw, thr, L, wg, fe, ae, te, counts, ord, st);
    else eval_launch<true, false>(t, N, raw, thr, L, wg, fe, ae, te, counts, ord, st);
  }
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_grid_eval(const GridView& g, int N, const float4* pack, const float4* abpack,
                             const float4* raw, float thr, bool adj, const FwdEpi& fe,
                             const AdjEpi& ae, int64_t* counts, cudaStream_t st) {
  const int groups = (N + 31) / 32;
  const unsigned nb = (unsigned)((groups + TR_WARPS - 1) / TR_WARPS);
  if (!adj)
    k_grid_eval<false><<<nb, TR_WARPS * 32, 0, st>>>(g, N, pack, abpack, raw, thr, counts, fe, ae);
  else
    k_grid_eval<true><<<nb, TR_WARPS * 32, 0, st>>>(g, N, pack, abpack, raw, thr, counts, fe, ae);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gs
