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
// forward); interactions are queued as (node, lane mask) and evaluated in
// batches of 32 with the records staged in shared memory.  A far node acts as
// one source at its centroid with momentum P, position derivative A and
// momentum derivative B/n, so the pair arithmetic is the exact kernel's.
#include <climits>

#include "tree_impl.h"

namespace gs {

namespace {

constexpr int TR_WARPS = 4;
constexpr int TR_BUF = 32;

template <bool ADJ>
__global__ void __launch_bounds__(TR_WARPS * 32)
    k_bh_traverse(TreeArrays t, int N, const float4* __restrict__ raw, float thr, FwdEpi fe,
                  AdjEpi ae, int64_t* counts) {
  constexpr int R = ADJ ? 4 : 2;
  constexpr int NC = ADJ ? 15 : 6;
  __shared__ float4 s_box[TR_WARPS][32][2];
  __shared__ float4 s_rec[TR_WARPS][TR_BUF][R];
  __shared__ int s_node[TR_WARPS][TR_BUF];
  __shared__ unsigned s_mask[TR_WARPS][TR_BUF];
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
  const float4 m0 = t.nrec[4 * leaf], m1 = t.nrec[4 * leaf + 1];
  float4 m2 = make_float4(0.f, 0.f, 0.f, 0.f), m3 = m2;
  if constexpr (ADJ) {
    m2 = t.nrec[4 * leaf + 2];
    m3 = t.nrec[4 * leaf + 3];
  }
  int resume = valid ? 0 : INT_MAX;
  Kahan K[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) K[c].zero();
  long long np = 0, nn = 0;
  int cnt = 0, base = INT_MIN / 2, x = 0;

  auto flush = [&]() {
    __syncwarp();
    if (lane < cnt) {
      const int nd = s_node[w][lane];
#pragma unroll
      for (int r = 0; r < R; r++) s_rec[w][lane][r] = t.nrec[4 * nd + r];
    }
    __syncwarp();
    if constexpr (!ADJ) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, h0 = 0.f, h1 = 0.f, h2 = 0.f;
      for (int e = 0; e < cnt; e++) {
        const bool bit = (s_mask[w][e] >> lane) & 1u;
        const float4 A = s_rec[w][e][0], P = s_rec[w][e][1];
        const float dx = m0.x - A.x, dy = m0.y - A.y, dz = m0.z - A.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float g = bit ? ex2_neg(r2) : 0.f;
        f0 += g * P.x;
        f1 += g * P.y;
        f2 += g * P.z;
        const float cg = (m1.x * P.x + m1.y * P.y + m1.z * P.z) * g;
        h0 += cg * dx;
        h1 += cg * dy;
        h2 += cg * dz;
      }
      K[0].add(f0);
      K[1].add(f1);
      K[2].add(f2);
      K[3].add(h0);
      K[4].add(h1);
      K[5].add(h2);
    } else {
      float a1[3] = {0, 0, 0}, a2[3] = {0, 0, 0}, a3[3] = {0, 0, 0}, b1[3] = {0, 0, 0},
            b2[3] = {0, 0, 0};
      for (int e = 0; e < cnt; e++) {
        const bool bit = (s_mask[w][e] >> lane) & 1u;
        const float4 A = s_rec[w][e][0], P = s_rec[w][e][1], Aa = s_rec[w][e][2],
                     Bb = s_rec[w][e][3];
        const float d[3] = {m0.x - A.x, m0.y - A.y, m0.z - A.z};
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const float g = bit ? ex2_neg(r2) : 0.f;
        const float c = m1.x * P.x + m1.y * P.y + m1.z * P.z;
        const float s1 = (m2.x * P.x + m2.y * P.y + m2.z * P.z) +
                         (Aa.x * m1.x + Aa.y * m1.y + Aa.z * m1.z);
        const float wv[3] = {m3.x - Bb.x, m3.y - Bb.y, m3.z - Bb.z};
        const float wd = wv[0] * d[0] + wv[1] * d[1] + wv[2] * d[2];
        const float gs = g * s1, cg = c * g, cw = cg * wd, gw = g * wd;
        const float pa[3] = {P.x, P.y, P.z}, aa[3] = {Aa.x, Aa.y, Aa.z};
#pragma unroll
        for (int k = 0; k < 3; k++) {
          a1[k] += gs * d[k];
          a2[k] += cg * wv[k];
          a3[k] += cw * d[k];
          b1[k] += g * aa[k];
          b2[k] += gw * pa[k];
        }
      }
#pragma unroll
      for (int k = 0; k < 3; k++) {
        K[k].add(a1[k]);
        K[3 + k].add(a2[k]);
        K[6 + k].add(a3[k]);
        K[9 + k].add(b1[k]);
        K[12 + k].add(b2[k]);
      }
    }
    __syncwarp();
  };

  while (x < M) {
    if (x >= base + 32) {
      __syncwarp();
      base = x;
      const int j = base + lane;
      if (j < M) {
        s_box[w][lane][0] = t.nbox[2 * j];
        s_box[w][lane][1] = t.nbox[2 * j + 1];
      }
      __syncwarp();
    }
    const float4 bl = s_box[w][x - base][0];
    const int skip = __float_as_int(bl.w);
    const bool active = x >= resume;
    const bool is_leaf = (skip == x + 1);
    bool take, open;
    if (is_leaf) {
      take = active;
      open = false;
    } else {
      const float4 bh = s_box[w][x - base][1];
      const bool far = active && box_dist2(rr.x, rr.y, rr.z, bl, bh) > thr;
      take = far;
      open = active && !far;
      if (far) resume = skip;
    }
    const unsigned mt = __ballot_sync(FULL, take), mo = __ballot_sync(FULL, open);
    if (mt) {
      if (lane == 0) {
        s_node[w][cnt] = x;
        s_mask[w][cnt] = mt;
      }
      if (is_leaf) np += __popc(mt);
      else nn += __popc(mt);
      if (++cnt == TR_BUF) {
        flush();
        cnt = 0;
      }
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
  return cudaGetLastError();
}

cudaError_t launch_bh_traverse_adj(const TreeArrays& t, int N, const float4* raw, float thr,
                                   const AdjEpi& e, int64_t* counts, cudaStream_t st) {
  k_bh_traverse<true><<<tr_blocks(N), TR_WARPS * 32, 0, st>>>(t, N, raw, thr, FwdEpi{}, e,
                                                              counts);
  return cudaGetLastError();
}

}  // namespace gs
