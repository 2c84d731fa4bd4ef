// exact.cu -- exact all-pairs right-hand sides of the Hamiltonian flow
// (Sec. 2.1 Eq. 1) and of its discrete adjoint, O(N^2) per step.
//
// Work decomposition: a block owns EX_NT target points (one per thread) and a
// contiguous range of source tiles (split J ways so that the grid fills the
// GPU).  Source tiles of EX_TILE points are staged into shared memory by 1-D
// bulk copies (cp.async.bulk, no multicast) through an EX_STAGES-deep mbarrier
// pipeline; each thread streams the tile with f32x2 arithmetic, two sources
// per instruction, exp on MUFU ex2.  Per-tile FP32 partial sums are folded
// into Kahan accumulators; each block writes its compensated partial, and the
// last block to finish a target tile (ticket counter) sums the J partials in
// FP64 in a fixed order and applies the epilogue (Euler update + next pack),
// so results are deterministic.
#include "common.cuh"
#include "kernels.h"

namespace gs {

namespace {

constexpr int kFwdComps = 6;
constexpr int kAdjComps = 15;

struct TileRange {
  int t0, nt;
};
__device__ __forceinline__ TileRange tile_range(int bj, int J, int n_jtiles) {
  int a = (int)(((long long)bj * n_jtiles) / J);
  int b = (int)(((long long)(bj + 1) * n_jtiles) / J);
  return {a, b - a};
}

// Issue the bulk copies of source tile `t` into stage buffer `dst`.
template <int NPACK>
__device__ __forceinline__ void issue_tile(float4* dst, const float4* const* src, int t,
                                           uint64_t* bar) {
  constexpr unsigned kBytes = EX_TILE / 2 * 3 * sizeof(float4);
  mbar_expect_tx(bar, kBytes * NPACK);
#pragma unroll
  for (int k = 0; k < NPACK; k++)
    bulk_g2s(dst + k * (EX_TILE / 2 * 3), src[k] + (size_t)t * (EX_TILE / 2 * 3), kBytes, bar);
}

// Ticket: returns true in exactly one block per target tile -- the last one to
// publish its partials.  Resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned* tickets, int bi, int J) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(&tickets[bi], 1u);
    s_last = (prev == (unsigned)(J - 1));
    if (s_last) tickets[bi] = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// After a timed-out wait at tile `t`, wait (bounded again) for the copies
// still in flight: tiles t .. min(t + EX_STAGES, nt) - 1.
__device__ __noinline__ void drain_stages(uint64_t* bars, int t, int nt, int* status) {
  for (int u = t; u < nt && u < t + EX_STAGES; u++)
    (void)mbar_wait_bounded(&bars[u % EX_STAGES], (unsigned)((u / EX_STAGES) & 1), status,
                            400000000LL);
}

}  // namespace

// ---------------------------------------------------------------------------
// Forward: F_i = Sum_j g_ij p_j, S_i = Sum_j (p_i.p_j) g_ij d_s,ij.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EX_NT, 3)
    k_exact_fwd(const float4* __restrict__ pk, ExactGeom geo, float2* __restrict__ part,
                unsigned* __restrict__ tickets, FwdEpi epi, int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  const int tid = threadIdx.x, bi = blockIdx.x, bj = blockIdx.y;
  const int64_t i = (int64_t)bi * EX_NT + tid;
  const TileRange tr = tile_range(bj, geo.J, geo.n_jtiles);

  float qa[3], pa[3];
  pack_read(pk, i, qa, pa);
  const f2 xi = f2_dup(qa[0]), yi = f2_dup(qa[1]), zi = f2_dup(qa[2]);
  const f2 ui = f2_dup(pa[0]), vi = f2_dup(pa[1]), wi = f2_dup(pa[2]);

  const float4* srcs[1] = {pk};
  if (tid == 0) {
    for (int s = 0; s < EX_STAGES; s++) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < EX_STAGES && s < tr.nt; s++)
      issue_tile<1>(sbuf + s * (EX_TILE / 2 * 3), srcs, tr.t0 + s, &bars[s]);

  Kahan K[kFwdComps];
#pragma unroll
  for (int c = 0; c < kFwdComps; c++) K[c].zero();

  int aborted_at = -1;
  for (int t = 0; t < tr.nt; t++) {
    const int s = t % EX_STAGES;
    const unsigned par = (unsigned)((t / EX_STAGES) & 1);
    const bool ok = mbar_wait_bounded(&bars[s], par, status);
    if (__syncthreads_or(!ok)) {
      aborted_at = t;
      break;
    }
    const ulonglong2* tb = reinterpret_cast<const ulonglong2*>(sbuf + s * (EX_TILE / 2 * 3));
    f2 fx = 0, fy = 0, fz = 0, hx = 0, hy = 0, hz = 0;
#pragma unroll 4
    for (int m = 0; m < EX_TILE / 2; m++) {
      const ulonglong2 v0 = tb[3 * m + 0], v1 = tb[3 * m + 1], v2 = tb[3 * m + 2];
      const f2 dx = f2_sub(xi, v0.x), dy = f2_sub(yi, v0.y), dz = f2_sub(zi, v1.x);
      f2 r = f2_mul(dx, dx);
      r = f2_fma(dy, dy, r);
      r = f2_fma(dz, dz, r);
      const f2 g = gauss2(r);
      fx = f2_fma(g, v1.y, fx);
      fy = f2_fma(g, v2.x, fy);
      fz = f2_fma(g, v2.y, fz);
      f2 c = f2_mul(ui, v1.y);
      c = f2_fma(vi, v2.x, c);
      c = f2_fma(wi, v2.y, c);
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
    __syncthreads();
    if (tid == 0 && t + EX_STAGES < tr.nt)
      issue_tile<1>(sbuf + s * (EX_TILE / 2 * 3), srcs, tr.t0 + t + EX_STAGES, &bars[s]);
  }
  if (aborted_at >= 0 && tid == 0) drain_stages(bars, aborted_at, tr.nt, status);
#pragma unroll
  for (int c = 0; c < kFwdComps; c++)
    part[((size_t)bj * kFwdComps + c) * geo.Npad + i] = K[c].out();

  if (!last_block(tickets, bi, geo.J)) return;
  if (i >= geo.N) return;
  double acc[kFwdComps];
#pragma unroll
  for (int c = 0; c < kFwdComps; c++) acc[c] = 0.0;
  for (int b = 0; b < geo.J; b++)
#pragma unroll
    for (int c = 0; c < kFwdComps; c++) {
      const float2 v = __ldcg(&part[((size_t)b * kFwdComps + c) * geo.Npad + i]);
      acc[c] += (double)v.x + (double)v.y;
    }
  fwd_epilogue(i, acc, acc + 3, epi);
}

// ---------------------------------------------------------------------------
// Adjoint: with a = alpha^{k+1}, b = beta^{k+1}, w = b_i - b_j, d = d_s:
//   A1 = Sum g (a_i.p_j + a_j.p_i) d,  A2 = Sum c g w,  A3 = Sum c g (w.d) d,
//   B1 = Sum g a_j,                    B2 = Sum g (w.d) p_j.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EX_NT, 2)
    k_exact_adj(const float4* __restrict__ pk, const float4* __restrict__ ab, ExactGeom geo,
                float2* __restrict__ part, unsigned* __restrict__ tickets, AdjEpi epi,
                int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  const int tid = threadIdx.x, bi = blockIdx.x, bj = blockIdx.y;
  const int64_t i = (int64_t)bi * EX_NT + tid;
  const TileRange tr = tile_range(bj, geo.J, geo.n_jtiles);

  float qa[3], pa[3], aa[3], ba[3];
  pack_read(pk, i, qa, pa);
  pack_read(ab, i, aa, ba);
  const f2 xi = f2_dup(qa[0]), yi = f2_dup(qa[1]), zi = f2_dup(qa[2]);
  const f2 ui = f2_dup(pa[0]), vi = f2_dup(pa[1]), wi = f2_dup(pa[2]);
  const f2 axi = f2_dup(aa[0]), ayi = f2_dup(aa[1]), azi = f2_dup(aa[2]);
  const f2 bxi = f2_dup(ba[0]), byi = f2_dup(ba[1]), bzi = f2_dup(ba[2]);

  constexpr int kStage = 2 * (EX_TILE / 2 * 3);  // float4 per stage (two packs)
  const float4* srcs[2] = {pk, ab};
  if (tid == 0) {
    for (int s = 0; s < EX_STAGES; s++) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < EX_STAGES && s < tr.nt; s++)
      issue_tile<2>(sbuf + s * kStage, srcs, tr.t0 + s, &bars[s]);

  Kahan K[kAdjComps];
#pragma unroll
  for (int c = 0; c < kAdjComps; c++) K[c].zero();

  int aborted_at = -1;
  for (int t = 0; t < tr.nt; t++) {
    const int s = t % EX_STAGES;
    const unsigned par = (unsigned)((t / EX_STAGES) & 1);
    const bool ok = mbar_wait_bounded(&bars[s], par, status);
    if (__syncthreads_or(!ok)) {
      aborted_at = t;
      break;
    }
    const ulonglong2* tq = reinterpret_cast<const ulonglong2*>(sbuf + s * kStage);
    const ulonglong2* ta = tq + (EX_TILE / 2 * 3);
    f2 a1x = 0, a1y = 0, a1z = 0, a2x = 0, a2y = 0, a2z = 0, a3x = 0, a3y = 0, a3z = 0;
    f2 b1x = 0, b1y = 0, b1z = 0, b2x = 0, b2y = 0, b2z = 0;
#pragma unroll 2
    for (int m = 0; m < EX_TILE / 2; m++) {
      const ulonglong2 q0 = tq[3 * m + 0], q1 = tq[3 * m + 1], q2 = tq[3 * m + 2];
      const ulonglong2 s0 = ta[3 * m + 0], s1v = ta[3 * m + 1], s2 = ta[3 * m + 2];
      // q0 = {X, Y}, q1 = {Z, PX}, q2 = {PY, PZ}; s0 = {AX, AY}, s1v = {AZ, BX}, s2 = {BY, BZ}
      const f2 dx = f2_sub(xi, q0.x), dy = f2_sub(yi, q0.y), dz = f2_sub(zi, q1.x);
      f2 r = f2_mul(dx, dx);
      r = f2_fma(dy, dy, r);
      r = f2_fma(dz, dz, r);
      const f2 g = gauss2(r);
      f2 c = f2_mul(ui, q1.y);
      c = f2_fma(vi, q2.x, c);
      c = f2_fma(wi, q2.y, c);
      f2 sa = f2_mul(axi, q1.y);  // a_i . p_j
      sa = f2_fma(ayi, q2.x, sa);
      sa = f2_fma(azi, q2.y, sa);
      sa = f2_fma(s0.x, ui, sa);  // + a_j . p_i
      sa = f2_fma(s0.y, vi, sa);
      sa = f2_fma(s1v.x, wi, sa);
      const f2 gs = f2_mul(g, sa);
      a1x = f2_fma(gs, dx, a1x);
      a1y = f2_fma(gs, dy, a1y);
      a1z = f2_fma(gs, dz, a1z);
      const f2 wx = f2_sub(bxi, s1v.y), wy = f2_sub(byi, s2.x), wz = f2_sub(bzi, s2.y);
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
      b1x = f2_fma(g, s0.x, b1x);
      b1y = f2_fma(g, s0.y, b1y);
      b1z = f2_fma(g, s1v.x, b1z);
      const f2 gw = f2_mul(g, wd);
      b2x = f2_fma(gw, q1.y, b2x);
      b2y = f2_fma(gw, q2.x, b2y);
      b2z = f2_fma(gw, q2.y, b2z);
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
    __syncthreads();
    if (tid == 0 && t + EX_STAGES < tr.nt)
      issue_tile<2>(sbuf + s * kStage, srcs, tr.t0 + t + EX_STAGES, &bars[s]);
  }
  if (aborted_at >= 0 && tid == 0) drain_stages(bars, aborted_at, tr.nt, status);
#pragma unroll
  for (int c = 0; c < kAdjComps; c++)
    part[((size_t)bj * kAdjComps + c) * geo.Npad + i] = K[c].out();

  if (!last_block(tickets, bi, geo.J)) return;
  if (i >= geo.N) return;
  double acc[kAdjComps];
#pragma unroll
  for (int c = 0; c < kAdjComps; c++) acc[c] = 0.0;
  for (int b = 0; b < geo.J; b++)
#pragma unroll
    for (int c = 0; c < kAdjComps; c++) {
      const float2 v = __ldcg(&part[((size_t)b * kAdjComps + c) * geo.Npad + i]);
      acc[c] += (double)v.x + (double)v.y;
    }
  adj_epilogue(i, acc, acc + 3, acc + 6, acc + 9, acc + 12, epi);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
size_t exact_fwd_smem() { return (size_t)EX_STAGES * (EX_TILE / 2 * 3) * sizeof(float4); }
size_t exact_adj_smem() { return 2 * exact_fwd_smem(); }

cudaError_t exact_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_exact_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)exact_fwd_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_exact_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)exact_adj_smem());
}

cudaError_t launch_exact_fwd(const float4* pk, const ExactGeom& g, float2* part,
                             unsigned* tickets, const FwdEpi& e, int* status, cudaStream_t st) {
  dim3 grid(g.n_itiles, g.J);
  k_exact_fwd<<<grid, EX_NT, exact_fwd_smem(), st>>>(pk, g, part, tickets, e, status);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_exact_adj(const float4* pk, const float4* ab, const ExactGeom& g, float2* part,
                             unsigned* tickets, const AdjEpi& e, int* status, cudaStream_t st) {
  dim3 grid(g.n_itiles, g.J);
  k_exact_adj<<<grid, EX_NT, exact_adj_smem(), st>>>(pk, ab, g, part, tickets, e, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gs
