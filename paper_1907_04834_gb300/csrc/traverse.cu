// traverse.cu -- Barnes-Hut traversal of Sec. 2.2 (Fig. 1), forward (Eq. 4
// and the momentum-dot replacement) and backward (alpha, beta replaced by
// their node averages), one warp per 32 Morton-consecutive points.
//
// The warp walks the preorder node array once, front to back.  At node x
// every lane applies its own point's rule (three cases of Sec. 2.2):
//   leaf                     -> exact interaction with that point;
//   internal, range farther than the threshold -> one interaction with the
//                               node summary; the lane then ignores x's
//                               subtree (resume = skip(x));
//   internal, otherwise      -> open x.
// The warp steps into x when any lane opens it, else jumps to skip(x).  A
// lane's interactions are exactly those of its own recursive traversal;
// lanes that have already summarised an ancestor stay idle inside it.
// Node boxes are staged 32 at a time in shared memory (the walk only moves
// forward) with a bit mask of which are leaves; a run of consecutive leaves
// is queued in one step (lanes change activity only at their resume points,
// so the run is cut at the first one).  Interactions are queued as (node,
// lane mask) and evaluated in batches of >= 32, two sources per f32x2
// instruction, with the records staged in shared memory.  A far node acts as
// one source at its centroid with momentum P, position derivative A and
// momentum derivative B/n, so the pair arithmetic is the exact kernel's.
#include <climits>

#include "kernels.h"
#include "tree_impl.h"

namespace gs {

namespace {

constexpr int TR_WARPS = 4;
constexpr int TR_BUF = 32;  // flush when this many interactions are queued
constexpr int TR_CAP = 64;  // queue capacity (a leaf run adds at most 32)

template <bool ADJ>
__global__ void __launch_bounds__(TR_WARPS * 32)
    k_bh_traverse(TreeArrays t, int N, const float4* __restrict__ raw, float thr, FwdEpi fe,
                  AdjEpi ae, int64_t* counts) {
  constexpr int NR = ADJ ? 12 : 6;   // record components used
  constexpr int NC = ADJ ? 15 : 6;   // accumulated components
  __shared__ float4 s_box[TR_WARPS][32][2];
  __shared__ __align__(16) float s_soa[TR_WARPS][NR][TR_CAP];
  __shared__ int s_node[TR_WARPS][TR_CAP];
  __shared__ unsigned s_mask[TR_WARPS][TR_CAP];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wg = blockIdx.x * TR_WARPS + w;
  if (wg * 32 >= N) return;  // the whole warp leaves together
  const int i = wg * 32 + lane;
  const bool valid = i < N;
  const int M = total_nodes(t, N);
  const int ii = valid ? i : N - 1;
  const int o = (int)t.perm[ii];
  const int leaf = ii + (int)t.offs[ii + 1];
  const float4 rr = raw[o];
  float4 m0 = t.nrec[4 * leaf], m1 = t.nrec[4 * leaf + 1];
  float4 m2 = make_float4(0.f, 0.f, 0.f, 0.f), m3 = m2;
  if constexpr (ADJ) {
    m2 = t.nrec[4 * leaf + 2];
    m3 = t.nrec[4 * leaf + 3];
  }
  // own position/momentum (and alpha, beta) duplicated into f32x2 pairs
  const f2 X = f2_dup(m0.x), Y = f2_dup(m0.y), Z = f2_dup(m0.z);
  const f2 U = f2_dup(m1.x), V = f2_dup(m1.y), W = f2_dup(m1.z);
  const f2 AX = f2_dup(m2.x), AY = f2_dup(m2.y), AZ = f2_dup(m2.z);
  const f2 BX = f2_dup(m3.x), BY = f2_dup(m3.y), BZ = f2_dup(m3.z);
  int resume = valid ? 0 : INT_MAX;
  Kahan K[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) K[c].zero();
  long long np = 0, nn = 0;
  int cnt = 0, base = INT_MIN / 2, x = 0;
  unsigned leafmask = 0u;

  // Evaluates the queued interactions, two sources per f32x2 instruction;
  // a lane whose bit is clear gets weight 0.
  auto flush = [&]() {
    __syncwarp();
    for (int e = lane; e < cnt; e += 32) {
      const int nd = s_node[w][e];
      const float4 r0 = t.nrec[4 * nd], r1 = t.nrec[4 * nd + 1];
      s_soa[w][0][e] = r0.x, s_soa[w][1][e] = r0.y, s_soa[w][2][e] = r0.z;
      s_soa[w][3][e] = r1.x, s_soa[w][4][e] = r1.y, s_soa[w][5][e] = r1.z;
      if constexpr (ADJ) {
        const float4 r2 = t.nrec[4 * nd + 2], r3 = t.nrec[4 * nd + 3];
        s_soa[w][6][e] = r2.x, s_soa[w][7][e] = r2.y, s_soa[w][8][e] = r2.z;
        s_soa[w][9][e] = r3.x, s_soa[w][10][e] = r3.y, s_soa[w][11][e] = r3.z;
      }
    }
    if (cnt & 1) {  // pad to an even count with an empty entry
      if (lane == 0) s_mask[w][cnt] = 0u;
      if (lane < NR) s_soa[w][lane][cnt] = 0.f;
    }
    __syncwarp();
    auto ld = [&](int c, int e) { return *reinterpret_cast<const f2*>(&s_soa[w][c][e]); };
    if constexpr (!ADJ) {
      f2 fx = 0, fy = 0, fz = 0, hx = 0, hy = 0, hz = 0;
      for (int e = 0; e < cnt; e += 2) {
        const bool b0 = (s_mask[w][e] >> lane) & 1u, b1 = (s_mask[w][e + 1] >> lane) & 1u;
        const f2 dx = f2_sub(X, ld(0, e)), dy = f2_sub(Y, ld(1, e)), dz = f2_sub(Z, ld(2, e));
        f2 r = f2_mul(dx, dx);
        r = f2_fma(dy, dy, r);
        r = f2_fma(dz, dz, r);
        float r0, r1;
        f2_split(r, r0, r1);
        const f2 g = f2_make(b0 ? ex2_neg(r0) : 0.f, b1 ? ex2_neg(r1) : 0.f);
        const f2 PX = ld(3, e), PY = ld(4, e), PZ = ld(5, e);
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
      K[0].add(f2_sum(fx));
      K[1].add(f2_sum(fy));
      K[2].add(f2_sum(fz));
      K[3].add(f2_sum(hx));
      K[4].add(f2_sum(hy));
      K[5].add(f2_sum(hz));
    } else {
      f2 a1x = 0, a1y = 0, a1z = 0, a2x = 0, a2y = 0, a2z = 0, a3x = 0, a3y = 0, a3z = 0;
      f2 b1x = 0, b1y = 0, b1z = 0, b2x = 0, b2y = 0, b2z = 0;
      for (int e = 0; e < cnt; e += 2) {
        const bool b0 = (s_mask[w][e] >> lane) & 1u, b1 = (s_mask[w][e + 1] >> lane) & 1u;
        const f2 dx = f2_sub(X, ld(0, e)), dy = f2_sub(Y, ld(1, e)), dz = f2_sub(Z, ld(2, e));
        f2 r = f2_mul(dx, dx);
        r = f2_fma(dy, dy, r);
        r = f2_fma(dz, dz, r);
        float r0, r1;
        f2_split(r, r0, r1);
        const f2 g = f2_make(b0 ? ex2_neg(r0) : 0.f, b1 ? ex2_neg(r1) : 0.f);
        const f2 PX = ld(3, e), PY = ld(4, e), PZ = ld(5, e);
        const f2 QX = ld(6, e), QY = ld(7, e), QZ = ld(8, e);  // a_j (or A)
        f2 c = f2_mul(U, PX);
        c = f2_fma(V, PY, c);
        c = f2_fma(W, PZ, c);
        f2 sa = f2_mul(AX, PX);  // a_i . p_j
        sa = f2_fma(AY, PY, sa);
        sa = f2_fma(AZ, PZ, sa);
        sa = f2_fma(QX, U, sa);  // + a_j . p_i
        sa = f2_fma(QY, V, sa);
        sa = f2_fma(QZ, W, sa);
        const f2 gs = f2_mul(g, sa);
        a1x = f2_fma(gs, dx, a1x);
        a1y = f2_fma(gs, dy, a1y);
        a1z = f2_fma(gs, dz, a1z);
        const f2 wx = f2_sub(BX, ld(9, e)), wy = f2_sub(BY, ld(10, e)),
                 wz = f2_sub(BZ, ld(11, e));
        f2 wd = f2_mul(wx, dx);
        wd = f2_fma(wy, dy, wd);
        wd = f2_fma(wz, dz, wd);
        const f2 cg = f2_mul(c, g);
        a2x = f2_fma(cg, wx, a2x);
        a2y = f2_fma(cg, wy, a2y);
        a2z = f2_fma(cg, wz, a2z);
        const f2 cw = f2_mul(cg, wd);
        a3x = f2_fma(cw, dx, a3x);
        a3y = f2_fma(cw, dy, a3y);
        a3z = f2_fma(cw, dz, a3z);
        b1x = f2_fma(g, QX, b1x);
        b1y = f2_fma(g, QY, b1y);
        b1z = f2_fma(g, QZ, b1z);
        const f2 gw = f2_mul(g, wd);
        b2x = f2_fma(gw, PX, b2x);
        b2y = f2_fma(gw, PY, b2y);
        b2z = f2_fma(gw, PZ, b2z);
      }
      K[0].add(f2_sum(a1x));
      K[1].add(f2_sum(a1y));
      K[2].add(f2_sum(a1z));
      K[3].add(f2_sum(a2x));
      K[4].add(f2_sum(a2y));
      K[5].add(f2_sum(a2z));
      K[6].add(f2_sum(a3x));
      K[7].add(f2_sum(a3y));
      K[8].add(f2_sum(a3z));
      K[9].add(f2_sum(b1x));
      K[10].add(f2_sum(b1y));
      K[11].add(f2_sum(b1z));
      K[12].add(f2_sum(b2x));
      K[13].add(f2_sum(b2y));
      K[14].add(f2_sum(b2z));
    }
    __syncwarp();
    cnt = 0;
  };

  while (x < M) {
    if (x >= base + 32) {  // stage the next 32 node boxes
      __syncwarp();
      base = x;
      const int j = base + lane;
      bool lf = false;
      if (j < M) {
        const float4 lo = t.nbox[2 * j], hi = t.nbox[2 * j + 1];
        s_box[w][lane][0] = lo;
        s_box[w][lane][1] = hi;
        lf = __float_as_int(lo.w) == j + 1;
      }
      leafmask = __ballot_sync(FULL, lf);
      __syncwarp();
    }
    const int off = x - base;
    if ((leafmask >> off) & 1u) {
      // a run of consecutive leaves: every lane active at x stays active
      // until the first resume point inside the run
      const unsigned rest = ~(leafmask >> off);
      int r = rest ? __ffs(rest) - 1 : 32 - off;
      const int lim = resume > x ? resume : INT_MAX;
      const int rmin = __reduce_min_sync(FULL, lim);
      if (rmin - x < r) r = rmin - x;
      const unsigned mk = __ballot_sync(FULL, resume <= x);
      if (mk) {
        if (lane < r) {
          s_node[w][cnt + lane] = x + lane;
          s_mask[w][cnt + lane] = mk;
        }
        np += (long long)__popc(mk) * r;
        cnt += r;
        if (cnt >= TR_BUF) flush();
      }
      x += r;
      continue;
    }
    // internal node: each active lane decides far (summarise) or open
    const float4 bl = s_box[w][off][0], bh = s_box[w][off][1];
    const int skip = __float_as_int(bl.w);
    const bool active = x >= resume;
    const bool far = active && box_dist2(rr.x, rr.y, rr.z, bl, bh) > thr;
    if (far) resume = skip;
    const unsigned mt = __ballot_sync(FULL, far), mo = __ballot_sync(FULL, active && !far);
    if (mt) {
      if (lane == 0) {
        s_node[w][cnt] = x;
        s_mask[w][cnt] = mt;
      }
      nn += __popc(mt);
      if (++cnt >= TR_BUF) flush();
    }
    x = mo ? x + 1 : skip;
  }
  if (cnt) flush();

  if (counts && lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[0]), (unsigned long long)np);
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[1]), (unsigned long long)nn);
  }
  if (!valid) return;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    const float2 v = K[c].out();
    acc[c] = (double)v.x + (double)v.y;
  }
  if constexpr (!ADJ) fwd_epilogue(o, acc, acc + 3, fe);
  else adj_epilogue(o, acc, acc + 3, acc + 6, acc + 9, acc + 12, ae);
}

inline unsigned tr_blocks(int N) {
  const int warps = (N + 31) / 32;
  return (unsigned)((warps + TR_WARPS - 1) / TR_WARPS);
}

}  // namespace

cudaError_t launch_bh_traverse_fwd(const TreeArrays& t, int N, const float4* raw, float thr,
                                   const FwdEpi& e, int64_t* counts, cudaStream_t st) {
  k_bh_traverse<false><<<tr_blocks(N), TR_WARPS * 32, 0, st>>>(t, N, raw, thr, e, AdjEpi{},
                                                               counts);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bh_traverse_adj(const TreeArrays& t, int N, const float4* raw, float thr,
                                   const AdjEpi& e, int64_t* counts, cudaStream_t st) {
  k_bh_traverse<true><<<tr_blocks(N), TR_WARPS * 32, 0, st>>>(t, N, raw, thr, FwdEpi{}, e,
                                                              counts);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gs
