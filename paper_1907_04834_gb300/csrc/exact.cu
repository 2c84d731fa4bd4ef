// exact.cu -- exact all-pairs right-hand sides of the Hamiltonian flow
// (Sec. 2.1 Eq. 1) and of its discrete adjoint, O(N^2) per step.
//
// Source tiles of EX_TILE points are staged into shared memory by 1-D bulk
// copies (cp.async.bulk, no multicast) through an EX_STAGES-deep mbarrier
// pipeline; every thread owns one target point and streams each staged tile
// with f32x2 arithmetic, two sources per instruction, exp on MUFU ex2.  Tile
// partial sums are FP32 and folded into Kahan accumulators.
//
// Single point set: a block owns EX_NT targets and a contiguous range of
// source tiles (J splits, so the grid fills the GPU); each block writes its
// compensated partial, and the last block to finish a target tile (ticket
// counter) sums the J partials in FP64 in a fixed order and applies the
// epilogue (Euler update + next pack), so results are deterministic.
//
// Many point sets (batched): persistent blocks take (subject, target tile)
// items from a queue ordered by decreasing subject size; an item covers all
// of its subject's sources, so its epilogue follows directly.
#include "common.cuh"
#include "kernels.h"

namespace gs {

namespace {

constexpr int kFwdComps = 6;
constexpr int kAdjComps = 9;
constexpr int kTileF4 = EX_TILE / 2 * 3;  // float4 per tile of one pack

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
  constexpr unsigned kBytes = kTileF4 * sizeof(float4);
  mbar_expect_tx(bar, kBytes * NPACK);
#pragma unroll
  for (int k = 0; k < NPACK; k++)
    bulk_g2s(dst + k * kTileF4, src[k] + (size_t)t * kTileF4, kBytes, bar);
}

__device__ __forceinline__ void init_barriers(uint64_t* bars) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < EX_STAGES; s++) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
}

// Streams source tiles [t0, t0 + nt) of NPACK packs through the pipeline,
// calling body(stage) on each staged tile.  `done` counts the tiles this
// block has consumed so far (stage and phase continue across calls).  A wait
// that gives up records ST_TIMEOUT, waits (bounded) for the copies still in
// flight and returns false.
template <int NPACK, class Body>
__device__ __forceinline__ bool stream_tiles(float4* sbuf, uint64_t* bars,
                                             const float4* const* srcs, int t0, int nt,
                                             unsigned& done, int* status, Body&& body) {
  constexpr int kStage = NPACK * kTileF4;
  __syncthreads();  // the stage buffers' previous readers are done
  if (threadIdx.x == 0)
    for (int k = 0; k < EX_STAGES && k < nt; k++) {
      const unsigned u = done + k;
      issue_tile<NPACK>(sbuf + (u % EX_STAGES) * kStage, srcs, t0 + k, &bars[u % EX_STAGES]);
    }
  for (int t = 0; t < nt; t++) {
    const unsigned u = done + t;
    const int s = u % EX_STAGES;
    const bool ok = mbar_wait_bounded(&bars[s], (u / EX_STAGES) & 1u, status);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0)
        for (int v = t; v < nt && v < t + EX_STAGES; v++) {
          const unsigned uv = done + v;
          (void)mbar_wait_bounded(&bars[uv % EX_STAGES], (uv / EX_STAGES) & 1u, status,
                                  400000000LL);
        }
      done += nt;
      return false;
    }
    body(sbuf + s * kStage);
    __syncthreads();
    if (threadIdx.x == 0 && t + EX_STAGES < nt)
      issue_tile<NPACK>(sbuf + s * kStage, srcs, t0 + t + EX_STAGES, &bars[s]);
  }
  done += nt;
  return true;
}

// ---------------------------------------------------------------- tile bodies
// Forward sums of one target over one staged tile:
//   F = Sum_j g_ij p_j,  S = Sum_j (p_i.p_j) g_ij d_s,ij.
struct FwdTarget {
  f2 xi, yi, zi, ui, vi, wi;
  Kahan K[kFwdComps];
  __device__ __forceinline__ void load(const float4* pk, int64_t i) {
    float qa[3], pa[3];
    pack_read(pk, i, qa, pa);
    xi = f2_dup(qa[0]), yi = f2_dup(qa[1]), zi = f2_dup(qa[2]);
    ui = f2_dup(pa[0]), vi = f2_dup(pa[1]), wi = f2_dup(pa[2]);
#pragma unroll
    for (int c = 0; c < kFwdComps; c++) K[c].zero();
  }
  __device__ __forceinline__ void tile(const float4* stage) {
    const ulonglong2* tb = reinterpret_cast<const ulonglong2*>(stage);
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
  }
};

// Velocity of Eq. 3 at one tracer point over one staged tile:
//   v = Sum_j g(x - q_j) p_j  (the tracer is not a source).
constexpr int kVelComps = 3;
struct VelTarget {
  f2 xi, yi, zi;
  Kahan K[kVelComps];
  __device__ __forceinline__ void load(const float4* xpk, int64_t i, int64_t M) {
    const float4 r = i < M ? xpk[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi = f2_dup(r.x), yi = f2_dup(r.y), zi = f2_dup(r.z);
#pragma unroll
    for (int c = 0; c < kVelComps; c++) K[c].zero();
  }
  __device__ __forceinline__ void tile(const float4* stage) {
    const ulonglong2* tb = reinterpret_cast<const ulonglong2*>(stage);
    f2 fx = 0, fy = 0, fz = 0;
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
    }
    K[0].add(f2_sum(fx));
    K[1].add(f2_sum(fy));
    K[2].add(f2_sum(fz));
  }
};

// Adjoint sums of one target over one staged tile (a = alpha^{k+1}, b' the
// scaled beta^{k+1} of the adjoint pack, w' = b'_i - b'_j, d = d_s):
//   A13' = Sum (g (a_i.p_j + a_j.p_i) + c g (w'.d)) d,  A2' = Sum c g w',
//   B'   = Sum g (a_j + (w'.d) p_j).
struct AdjTarget {
  f2 xi, yi, zi, ui, vi, wi, axi, ayi, azi, bxi, byi, bzi;
  Kahan K[kAdjComps];
  __device__ __forceinline__ void load(const float4* pk, const float4* ab, int64_t i) {
    float qa[3], pa[3], aa[3], ba[3];
    pack_read(pk, i, qa, pa);
    pack_read(ab, i, aa, ba);
    xi = f2_dup(qa[0]), yi = f2_dup(qa[1]), zi = f2_dup(qa[2]);
    ui = f2_dup(pa[0]), vi = f2_dup(pa[1]), wi = f2_dup(pa[2]);
    axi = f2_dup(aa[0]), ayi = f2_dup(aa[1]), azi = f2_dup(aa[2]);
    bxi = f2_dup(ba[0]), byi = f2_dup(ba[1]), bzi = f2_dup(ba[2]);
#pragma unroll
    for (int c = 0; c < kAdjComps; c++) K[c].zero();
  }
  __device__ __forceinline__ void tile(const float4* stage) {
    const ulonglong2* tq = reinterpret_cast<const ulonglong2*>(stage);
    const ulonglong2* ta = tq + kTileF4;
    f2 ax = 0, ay = 0, az = 0, a2x = 0, a2y = 0, a2z = 0, bx = 0, by = 0, bz = 0;
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
      const f2 wx = f2_sub(bxi, s1v.y), wy = f2_sub(byi, s2.x), wz = f2_sub(bzi, s2.y);
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
      bx = f2_fma(g, f2_fma(wd, q1.y, s0.x), bx);
      by = f2_fma(g, f2_fma(wd, q2.x, s0.y), by);
      bz = f2_fma(g, f2_fma(wd, q2.y, s1v.x), bz);
    }
    K[0].add(f2_sum(ax));
    K[1].add(f2_sum(ay));
    K[2].add(f2_sum(az));
    K[3].add(f2_sum(a2x));
    K[4].add(f2_sum(a2y));
    K[5].add(f2_sum(a2z));
    K[6].add(f2_sum(bx));
    K[7].add(f2_sum(by));
    K[8].add(f2_sum(bz));
  }
};

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

// Next work item of a persistent block (same value in every thread).
__device__ __forceinline__ int next_item(int* queue) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
  __syncthreads();
  return s_item;
}

}  // namespace

// ---------------------------------------------------------------------------
// Single point set, split over J source ranges.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EX_NT, 3)
    k_exact_fwd(const float4* __restrict__ pk, ExactGeom geo, float2* __restrict__ part,
                unsigned* __restrict__ tickets, FwdEpi epi, int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int64_t i = (int64_t)bi * EX_NT + threadIdx.x;
  const TileRange tr = tile_range(bj, geo.J, geo.n_jtiles);
  FwdTarget tg;
  tg.load(pk, i);
  init_barriers(bars);
  const float4* srcs[1] = {pk};
  unsigned done = 0;
  stream_tiles<1>(sbuf, bars, srcs, tr.t0, tr.nt, done, status,
                  [&](const float4* st) { tg.tile(st); });
#pragma unroll
  for (int c = 0; c < kFwdComps; c++)
    part[((size_t)bj * kFwdComps + c) * geo.Npad + i] = tg.K[c].out();
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

__global__ void __launch_bounds__(EX_NT, 2)
    k_exact_adj(const float4* __restrict__ pk, const float4* __restrict__ ab, ExactGeom geo,
                float2* __restrict__ part, unsigned* __restrict__ tickets, AdjEpi epi,
                int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int64_t i = (int64_t)bi * EX_NT + threadIdx.x;
  const TileRange tr = tile_range(bj, geo.J, geo.n_jtiles);
  AdjTarget tg;
  tg.load(pk, ab, i);
  init_barriers(bars);
  const float4* srcs[2] = {pk, ab};
  unsigned done = 0;
  stream_tiles<2>(sbuf, bars, srcs, tr.t0, tr.nt, done, status,
                  [&](const float4* st) { tg.tile(st); });
#pragma unroll
  for (int c = 0; c < kAdjComps; c++)
    part[((size_t)bj * kAdjComps + c) * geo.Npad + i] = tg.K[c].out();
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
  adj_epilogue(i, acc, acc + 3, acc + 6, epi);
}

// ---------------------------------------------------------------------------
// Tracer points (Eq. 3): targets are the tracers, sources the particles'
// pack; split over J source ranges like k_exact_fwd.  tg.M tracers in
// tg.n_itiles tiles of EX_NT.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EX_NT, 3)
    k_tracer(const float4* __restrict__ pk, ExactGeom geo, const float4* __restrict__ xpk,
             TracerGeom tg, float2* __restrict__ part, unsigned* __restrict__ tickets,
             TracerEpi epi, int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int64_t i = (int64_t)bi * EX_NT + threadIdx.x;
  const TileRange tr = tile_range(bj, tg.J, geo.n_jtiles);
  VelTarget vt;
  vt.load(xpk, i, tg.M);
  init_barriers(bars);
  const float4* srcs[1] = {pk};
  unsigned done = 0;
  stream_tiles<1>(sbuf, bars, srcs, tr.t0, tr.nt, done, status,
                  [&](const float4* st) { vt.tile(st); });
#pragma unroll
  for (int c = 0; c < kVelComps; c++)
    part[((size_t)bj * kVelComps + c) * tg.Mpad + i] = vt.K[c].out();
  if (!last_block(tickets, bi, tg.J)) return;
  if (i >= tg.M) return;
  double v[kVelComps];
#pragma unroll
  for (int c = 0; c < kVelComps; c++) v[c] = 0.0;
  for (int b = 0; b < tg.J; b++)
#pragma unroll
    for (int c = 0; c < kVelComps; c++) {
      const float2 u = __ldcg(&part[((size_t)b * kVelComps + c) * tg.Mpad + i]);
      v[c] += (double)u.x + (double)u.y;
    }
  tracer_epilogue(i, v, epi);
}

// ---------------------------------------------------------------------------
// Many point sets: persistent blocks over (subject, target tile) items.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EX_NT, 3)
    k_batched_fwd(const float4* __restrict__ pk, BatchInfo bi, FwdEpi epi, int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  init_barriers(bars);
  unsigned done = 0;
  for (int it = next_item(bi.queue); it < bi.n_items; it = next_item(bi.queue)) {
    const int2 w = bi.items[it];
    const int64_t pbase = bi.poff[w.x], row0 = bi.off[w.x];
    const int n = (int)(bi.off[w.x + 1] - row0), il = w.y * EX_NT + threadIdx.x;
    const float4* sp = pk + (size_t)(pbase / 2) * 3;
    FwdTarget tg;
    tg.load(sp, il);
    const float4* srcs[1] = {sp};
    // a wait that gave up ends the block's work (the status word says so)
    if (!stream_tiles<1>(sbuf, bars, srcs, 0, bi.npad[w.x] / EX_TILE, done, status,
                         [&](const float4* st) { tg.tile(st); }))
      break;
    if (il < n) {
      double acc[kFwdComps];
#pragma unroll
      for (int c = 0; c < kFwdComps; c++) {
        const float2 v = tg.K[c].out();
        acc[c] = (double)v.x + (double)v.y;
      }
      fwd_epilogue_at(row0 + il, pbase + il, bi.centers + 3 * w.x, acc, acc + 3, epi);
    }
  }
}

__global__ void __launch_bounds__(EX_NT, 2)
    k_batched_adj(const float4* __restrict__ pk, const float4* __restrict__ ab, BatchInfo bi,
                  AdjEpi epi, int* status) {
  extern __shared__ __align__(128) float4 sbuf[];
  __shared__ uint64_t bars[EX_STAGES];
  init_barriers(bars);
  unsigned done = 0;
  for (int it = next_item(bi.queue); it < bi.n_items; it = next_item(bi.queue)) {
    const int2 w = bi.items[it];
    const int64_t pbase = bi.poff[w.x], row0 = bi.off[w.x];
    const int n = (int)(bi.off[w.x + 1] - row0), il = w.y * EX_NT + threadIdx.x;
    const float4* sp = pk + (size_t)(pbase / 2) * 3;
    const float4* sa = ab + (size_t)(pbase / 2) * 3;
    AdjTarget tg;
    tg.load(sp, sa, il);
    const float4* srcs[2] = {sp, sa};
    if (!stream_tiles<2>(sbuf, bars, srcs, 0, bi.npad[w.x] / EX_TILE, done, status,
                         [&](const float4* st) { tg.tile(st); }))
      break;
    if (il < n) {
      double acc[kAdjComps];
#pragma unroll
      for (int c = 0; c < kAdjComps; c++) {
        const float2 v = tg.K[c].out();
        acc[c] = (double)v.x + (double)v.y;
      }
      adj_epilogue_at(row0 + il, pbase + il, acc, acc + 3, acc + 6, epi);
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
size_t exact_fwd_smem() { return (size_t)EX_STAGES * kTileF4 * sizeof(float4); }
size_t exact_adj_smem() { return 2 * exact_fwd_smem(); }

cudaError_t exact_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_exact_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)exact_fwd_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_exact_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)exact_adj_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batched_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)exact_fwd_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tracer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)exact_fwd_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batched_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)exact_adj_smem());
  return e;
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

cudaError_t launch_tracer(const float4* pk, const ExactGeom& g, const float4* xpk,
                          const TracerGeom& tg, float2* part, unsigned* tickets,
                          const TracerEpi& e, int* status, cudaStream_t st) {
  dim3 grid(tg.n_itiles, tg.J);
  k_tracer<<<grid, EX_NT, exact_fwd_smem(), st>>>(pk, g, xpk, tg, part, tickets, e, status);
  note_launches(1);
  return cudaGetLastError();
}

int batched_resident_blocks(bool adjoint) {
  int n = 0;
  cudaError_t e =
      adjoint ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_adj, EX_NT,
                                                               exact_adj_smem())
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_fwd, EX_NT,
                                                               exact_fwd_smem());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_batched_fwd(const float4* pk, const BatchInfo& b, const FwdEpi& e, int* status,
                               int blocks, cudaStream_t st) {
  k_batched_fwd<<<blocks, EX_NT, exact_fwd_smem(), st>>>(pk, b, e, status);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batched_adj(const float4* pk, const float4* ab, const BatchInfo& b,
                               const AdjEpi& e, int* status, int blocks, cudaStream_t st) {
  k_batched_adj<<<blocks, EX_NT, exact_adj_smem(), st>>>(pk, ab, b, e, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gs
