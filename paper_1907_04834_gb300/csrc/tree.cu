// tree.cu -- Barnes-Hut octree of Sec. 2.2 built on the GPU every step:
//   1. FP32 bounding box of the FP32 positions (the root cell);
//   2. 10-bit quantised coordinates per axis and 30-bit Morton codes:
//      ext = hi - lo, inv = 1024 / ext, u = (x - lo) * inv, k = min(trunc(u), 1023),
//      k = 0 on a zero-extent axis (all FP32, round to nearest, no contraction);
//   3. stable LSD radix sort of (code, index): one point set in three
//      passes of 10 bits, one kernel each (decoupled look-back); a forest
//      in 8-bit passes with the subject index as the leading digits;
//   4. the compressed octree in depth-first preorder (see tree_impl.h): one
//      owner boundary per internal node, node offsets by a prefix sum of the
//      per-position depth masks, skip pointers and parents by galloping search
//      over the sorted codes;
//   5. node aggregates (count, FP32 actual range, sums of scaled positions,
//      momenta and, in the backward stage, alpha and beta as compensated
//      FP32 pairs) over each node's range of sorted points, from the points
//      and the precomputed sums of aligned chunks of 32 and 1024 points.
// The paper inserts points one at a time into a pointer tree; the node set,
// the members of every node and the depth-first order are the same here (the
// tests compare them bit for bit with the oracle's insertion tree).
//
// A forest of independent point sets (subjects) is built in the same passes:
// each subject is quantised in its own bounding box, the sort key is
// (subject, code) (extra radix passes over the subject index), and two
// sorted points of different subjects share no cell, so every subject's tree
// is the one it would have alone, placed in a contiguous preorder range.
#include <algorithm>
#include <cstdio>
#include <utility>

#include "kernels.h"
#include "tree.h"
#include "tree_impl.h"

namespace gs {

namespace {

constexpr int kBBoxThreads = 256;
constexpr int kMaxBBoxBlocks = 1024;
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 4;  // keys per thread per tile (striped)
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
// single-pass sort of one point set: three passes of 10-bit digits over the
// 30-bit codes, OS_TILE keys per tile
constexpr int OS_BITS = 10, OS_BINS = 1 << OS_BITS, OS_PASSES = 3;
constexpr int OS_THREADS = 256, OS_WARPS = OS_THREADS / 32, OS_R = 8;
constexpr int OS_TILE = OS_THREADS * OS_R;
constexpr int MORTON_PTS = 4;  // points per thread of the Morton kernel

thread_local char g_err[256] = "";

inline unsigned nblocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------- bbox, Morton
__global__ void k_bbox_partial(const float4* __restrict__ raw, int N, float* part) {
  __shared__ float sh[6][kBBoxThreads / 32];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    float4 r = raw[i];
    lo[0] = fminf(lo[0], r.x);
    lo[1] = fminf(lo[1], r.y);
    lo[2] = fminf(lo[2], r.z);
    hi[0] = fmaxf(hi[0], r.x);
    hi[1] = fmaxf(hi[1], r.y);
    hi[2] = fmaxf(hi[2], r.z);
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; a++) {
      lo[a] = fminf(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; a++) {
      sh[a][w] = lo[a];
      sh[3 + a][w] = hi[a];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kBBoxThreads / 32; k++)
      for (int a = 0; a < 3; a++) {
        sh[a][0] = fminf(sh[a][0], sh[a][k]);
        sh[3 + a][0] = fmaxf(sh[3 + a][0], sh[3 + a][k]);
      }
    for (int a = 0; a < 6; a++) part[blockIdx.x * 6 + a] = sh[a][0];
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float ext, float inv) {
  if (!(ext > 0.f)) return 0u;
  float u = __fmul_rn(__fsub_rn(x, lo), inv);
  uint32_t k = __float2uint_rz(u);
  return k > 1023u ? 1023u : k;
}

// Morton codes of one point set, MORTON_PTS points per thread: the root
// box, each point's code (into key and codes), the digit histograms of the
// three sort passes (hist, 3 x 1024, zeroed by the caller), and the node
// bit masks of the node list zeroed for its build.
__global__ void __launch_bounds__(256)
    k_morton(const float4* __restrict__ raw, int N, const float* __restrict__ part, int nparts,
             uint32_t* key, uint32_t* codes, float* bbox, uint32_t* hist, uint32_t* mask) {
  // the root box: every block folds the nparts partial boxes, all its
  // threads at once (min and max are exact: any order gives the same box)
  __shared__ float sh[6][8];
  __shared__ float box[6];
  __shared__ uint32_t s_h[OS_PASSES * OS_BINS];
  for (int k = threadIdx.x; k < OS_PASSES * OS_BINS; k += blockDim.x) s_h[k] = 0u;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = threadIdx.x; k < nparts; k += blockDim.x)
    for (int a = 0; a < 3; a++) {
      lo[a] = fminf(lo[a], part[k * 6 + a]);
      hi[a] = fmaxf(hi[a], part[k * 6 + 3 + a]);
    }
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; a++) {
      lo[a] = fminf(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; a++) sh[a][wid] = lo[a], sh[3 + a][wid] = hi[a];
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    float v = sh[a][0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++)
      v = a < 3 ? fminf(v, sh[a][k]) : fmaxf(v, sh[a][k]);
    box[a] = v;
    if (blockIdx.x == 0) bbox[a] = v;
  }
  __syncthreads();
  float ext[3], inv[3];
  for (int a = 0; a < 3; a++) {
    ext[a] = __fsub_rn(box[3 + a], box[a]);
    inv[a] = ext[a] > 0.f ? __fdiv_rn(1024.0f, ext[a]) : 0.f;
  }
  for (int r = 0; r < MORTON_PTS; r++) {
    const int i = (blockIdx.x * MORTON_PTS + r) * blockDim.x + threadIdx.x;
    if (i >= N) break;
    const float4 q = raw[i];
    const uint32_t kx = quantise(q.x, box[0], ext[0], inv[0]);
    const uint32_t ky = quantise(q.y, box[1], ext[1], inv[1]);
    const uint32_t kz = quantise(q.z, box[2], ext[2], inv[2]);
    const uint32_t c = (spread10(kx) << 2) | (spread10(ky) << 1) | spread10(kz);
    key[i] = c;
    codes[i] = c;
    mask[i] = 0u;
    for (int p = 0; p < OS_PASSES; p++)
      atomicAdd(&s_h[p * OS_BINS + ((c >> (OS_BITS * p)) & (OS_BINS - 1))], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < OS_PASSES * OS_BINS; k += blockDim.x)
    if (s_h[k]) atomicAdd(&hist[k], s_h[k]);
}

// Forest: one block per subject, its FP32 bounding box into sbox[6 s ..].
__global__ void k_bbox_subjects(const float4* __restrict__ raw, const int64_t* __restrict__ off,
                                float* sbox) {
  __shared__ float sh[6][kBBoxThreads / 32];
  const int s = blockIdx.x;
  const int a = (int)off[s], b = (int)off[s + 1];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
    const float4 r = raw[i];
    lo[0] = fminf(lo[0], r.x);
    lo[1] = fminf(lo[1], r.y);
    lo[2] = fminf(lo[2], r.z);
    hi[0] = fmaxf(hi[0], r.x);
    hi[1] = fmaxf(hi[1], r.y);
    hi[2] = fmaxf(hi[2], r.z);
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 3; k++) {
      lo[k] = fminf(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; k++) {
      sh[k][w] = lo[k];
      sh[3 + k][w] = hi[k];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    float v = sh[k][0];
    for (int m = 1; m < kBBoxThreads / 32; m++) v = k < 3 ? fminf(v, sh[k][m]) : fmaxf(v, sh[k][m]);
    sbox[6 * s + k] = v;
  }
}

// Forest: Morton code of every point in its subject's box.
__global__ void k_morton_subjects(const float4* __restrict__ raw, int N,
                                  const int64_t* __restrict__ off, int S,
                                  const float* __restrict__ sbox, uint32_t* key, uint32_t* perm,
                                  uint32_t* codes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float* box = sbox + 6 * subject_of(off, S, i);
  const float4 r = raw[i];
  float ext[3], inv[3];
  for (int a = 0; a < 3; a++) {
    ext[a] = __fsub_rn(box[3 + a], box[a]);
    inv[a] = ext[a] > 0.f ? __fdiv_rn(1024.0f, ext[a]) : 0.f;
  }
  const uint32_t kx = quantise(r.x, box[0], ext[0], inv[0]);
  const uint32_t ky = quantise(r.y, box[1], ext[1], inv[1]);
  const uint32_t kz = quantise(r.z, box[2], ext[2], inv[2]);
  const uint32_t c = (spread10(kx) << 2) | (spread10(ky) << 1) | spread10(kz);
  key[i] = c;
  perm[i] = (uint32_t)i;
  codes[i] = c;
}

// Forest: subject index of each sorted point, the key of the subject passes.
__global__ void k_subject_keys(const uint32_t* __restrict__ perm, int N,
                               const int64_t* __restrict__ off, int S, uint32_t* skey) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) skey[i] = (uint32_t)subject_of(off, S, perm[i]);
}

// Forest, after the subject passes: sorted subjects, permutation and codes.
__global__ void k_forest_finish(const uint32_t* skey, const uint32_t* sperm, int N,
                                const uint32_t* __restrict__ codes, uint32_t* key,
                                uint32_t* perm, uint32_t* ssub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t s = skey[i], v = sperm[i];
  ssub[i] = s;
  perm[i] = v;
  key[i] = codes[v];
}

// Tracers walking a tree: Morton codes in the tree's root box (points
// outside it clamp to the boundary cells), keyed with their index.
__global__ void k_tracer_codes(const float4* __restrict__ xraw, int M,
                               const float* __restrict__ bbox, uint32_t* key, uint32_t* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const float4 r = xraw[i];
  float ext[3], inv[3];
  for (int a = 0; a < 3; a++) {
    ext[a] = __fsub_rn(bbox[3 + a], bbox[a]);
    inv[a] = ext[a] > 0.f ? __fdiv_rn(1024.0f, ext[a]) : 0.f;
  }
  const uint32_t kx = quantise(r.x, bbox[0], ext[0], inv[0]);
  const uint32_t ky = quantise(r.y, bbox[1], ext[1], inv[1]);
  const uint32_t kz = quantise(r.z, bbox[2], ext[2], inv[2]);
  key[i] = (spread10(kx) << 2) | (spread10(ky) << 1) | spread10(kz);
  perm[i] = (uint32_t)i;
}

// Per tracer group: the tree leaf nearest in Morton order to its middle
// tracer (first sorted point with a code >= the tracer's), where the
// group's slices are cut.
__global__ void k_tracer_mid(const uint32_t* __restrict__ tkey, int M, const uint32_t* __restrict__ sk,
                             const uint32_t* __restrict__ offs, int N, int* mid) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 32 >= M) return;
  const uint32_t c = tkey[g * 32 + min(16, M - g * 32 - 1)];
  int lo = 0, hi = N - 1;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (sk[m] < c) lo = m + 1;
    else hi = m;
  }
  mid[g] = lo + (int)offs[lo + 1];
}

// ---------------------------------------------------------------- scans
struct Ident {
  __device__ uint32_t operator()(uint32_t v) const { return v; }
};
struct Popc {
  __device__ uint32_t operator()(uint32_t v) const { return (uint32_t)__popc(v); }
};

__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = w > 0 ? warp_tot[w - 1] : 0u;
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

template <class Op>
__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int n, uint32_t* bsum, Op op) {
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++)
    if (base + k < n) s += op(in[base + k]);
  uint32_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_bsums(uint32_t* bsum, int nb) {
  uint32_t carry = 0;
  for (int c0 = 0; c0 < nb; c0 += SCAN_THREADS) {
    const int i = c0 + threadIdx.x;
    uint32_t v = i < nb ? bsum[i] : 0u, tot;
    uint32_t ex = block_excl_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
}

template <class Op>
__global__ void k_scan_apply(const uint32_t* __restrict__ in, int n, const uint32_t* bsum,
                             uint32_t* out, Op op) {
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS], s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = base + k < n ? op(in[base + k]) : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t ex = bsum[blockIdx.x] + block_excl_scan(s, &tot);
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bsum[blockIdx.x] + tot;
}

// exclusive scan of op(in[0..n)) into out[0..n], out[n] = total
template <class Op>
cudaError_t scan(const uint32_t* in, int n, uint32_t* bsum, uint32_t* out, Op op,
                 cudaStream_t st) {
  const int nb = (int)nblocks(n, SCAN_TILE);
  k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(in, n, bsum, op);
  k_scan_bsums<<<1, SCAN_THREADS, 0, st>>>(bsum, nb);
  k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, n, bsum, out, op);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
// hist layout: digit-major, hist[d * nb + block].
__global__ void k_rs_hist(const uint32_t* __restrict__ key, int N, int shift, uint32_t* hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    const int i = base + r * RS_THREADS + threadIdx.x;
    if (i < N) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: key order within a tile is round-major then thread, i.e.
// the input order; ranks among equal digits follow it.
__global__ void k_rs_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ val,
                             int N, int shift, const uint32_t* __restrict__ hscan,
                             uint32_t* key_out, uint32_t* val_out) {
  constexpr int W = RS_THREADS / 32;
  __shared__ uint32_t run[256];     // keys of each digit placed so far in this tile
  __shared__ uint32_t wcnt[W][256]; // per-warp counts in the current round
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = 0u;
  const uint32_t goff = hscan[threadIdx.x * gridDim.x + blockIdx.x];
  __shared__ uint32_t gbase[256];
  gbase[threadIdx.x] = goff;
  const int base = blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    for (int k = 0; k < W; k++) wcnt[k][threadIdx.x] = 0u;
    __syncthreads();
    const int i = base + r * RS_THREADS + threadIdx.x;
    const bool valid = i < N;
    uint32_t k = 0, v = 0, d = 256u;
    if (valid) {
      k = key[i];
      v = val[i];
      d = (k >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank_w = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank_w == 0) wcnt[w][d] = (uint32_t)__popc(peers);
    __syncthreads();
    // thread t owns digit t: prefix over warps, then advance the running count
    {
      uint32_t acc = run[threadIdx.x];
      for (int k2 = 0; k2 < W; k2++) {
        uint32_t c = wcnt[k2][threadIdx.x];
        wcnt[k2][threadIdx.x] = acc;
        acc += c;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = gbase[d] + wcnt[w][d] + (uint32_t)rank_w;
      key_out[pos] = k;
      val_out[pos] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- single-pass sort
// Stable LSD radix sort of the 30-bit codes of one point set in three passes
// of 10 bits with one kernel per pass.  A tile of OS_TILE keys ranks its
// keys stably by digit, publishes its count of each digit and adds up the
// counts of the tiles before it by decoupled look-back (the single-pass
// prefix scan of Merrill and Garland, 2016, applied per digit as in the
// one-kernel-per-digit radix sort of Adinets and Merrill, 2022); the digit
// histograms of all three passes come from the Morton kernel.  Tiles are
// numbered in the order blocks start, so every tile a look-back waits for
// belongs to a block that is running or done.
//
// Look-back word of a (tile, digit): bits 62-63 the kind (0 nothing yet,
// LB_AGG the tile's own count, LB_PRE the count of this and every earlier
// tile), bits 0-61 the count.
constexpr unsigned long long LB_AGG = 1ull << 62, LB_PRE = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr long long LB_SPIN_CYCLES = 2000000000LL;  // about 1 s of SM clock

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Publishes the tile's own count (tile > 0; tile 0 publishes its prefix).
__device__ __forceinline__ void lb_publish(unsigned long long* word, int tile,
                                           unsigned long long cnt) {
  lb_store(word, (tile == 0 ? LB_PRE : LB_AGG) | cnt);
}

// Exclusive prefix of tile `tile` (words of tile j at stat[j * stride]),
// whose own count `cnt` is published: adds the counts of the tiles before it
// back to the first one with a published prefix, then publishes its own
// prefix.  A word that stays empty for about a second records ST_TIMEOUT in
// *status and ends the look-back (the result is then wrong, and the call
// reports the timeout; every position computed from it is bounds-checked).
__device__ unsigned long long lb_prefix(unsigned long long* stat, size_t stride, int tile,
                                        unsigned long long cnt, int* status) {
  if (tile == 0) return 0ull;
  unsigned long long excl = 0ull;
  int j = tile - 1;
  long long t0 = clock64();
  while (true) {
    const unsigned long long v = lb_load(stat + (size_t)j * stride);
    const unsigned long long kind = v & ~LB_VAL;
    if (kind == 0ull) {
      if (clock64() - t0 > LB_SPIN_CYCLES) {
        atomicOr(status, ST_TIMEOUT);
        break;
      }
      continue;
    }
    excl += v & LB_VAL;
    if (kind == LB_PRE || j == 0) break;
    j--;
    t0 = clock64();
  }
  lb_store(stat + (size_t)tile * stride, LB_PRE | (excl + cnt));
  return excl;
}

// One pass over digit (key >> shift) & 1023.  val_in NULL: the values are
// the input positions (the first pass).  ghist: the pass's 1024 digit counts
// over all keys.
__global__ void __launch_bounds__(OS_THREADS)
    k_os_pass(const uint32_t* __restrict__ key_in, const uint32_t* __restrict__ val_in, int N,
              int shift, const uint32_t* __restrict__ ghist, unsigned long long* stat, int* ctr,
              int* status, uint32_t* key_out, uint32_t* val_out) {
  __shared__ uint32_t s_wc[OS_WARPS][OS_BINS];  // per warp and digit: count, then offset
  __shared__ uint32_t s_base[OS_BINS];          // global start of the digit, then + tile's
  __shared__ uint32_t s_wsum[OS_WARPS];
  __shared__ int s_tile;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(ctr, 1);
  for (int k = tid; k < OS_WARPS * OS_BINS; k += OS_THREADS) (&s_wc[0][0])[k] = 0u;
  // global start of each digit: exclusive scan of ghist, 4 digits per thread
  constexpr int PER = OS_BINS / OS_THREADS;
  uint32_t h[PER], hs = 0u;
#pragma unroll
  for (int k = 0; k < PER; k++) {
    h[k] = ghist[PER * tid + k];
    hs += h[k];
  }
  uint32_t inc = hs;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_wsum[w] = inc;
  __syncthreads();
  uint32_t before = 0u;
  for (int k = 0; k < w; k++) before += s_wsum[k];
  uint32_t run = before + inc - hs;
#pragma unroll
  for (int k = 0; k < PER; k++) {
    s_base[PER * tid + k] = run;
    run += h[k];
  }
  __syncthreads();
  const int tile = s_tile;
  // stable ranks within the warp's keys (input order: warp, round, lane)
  const int base = tile * OS_TILE + w * (32 * OS_R);
  uint32_t kk[OS_R], vv[OS_R], rk[OS_R];
#pragma unroll
  for (int r = 0; r < OS_R; r++) {
    const int i = base + r * 32 + lane;
    const bool valid = i < N;
    kk[r] = valid ? key_in[i] : 0u;
    vv[r] = valid ? (val_in ? val_in[i] : (uint32_t)i) : 0u;
    const uint32_t d = valid ? (kk[r] >> shift) & (OS_BINS - 1) : (uint32_t)OS_BINS;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0u;
    if (valid && lane == leader) {
      old = s_wc[w][d];
      s_wc[w][d] = old + (uint32_t)__popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rk[r] = old + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    __syncwarp();
  }
  __syncthreads();
  // per digit: offsets of the warps within the tile, the tile's count,
  // published first for all of this thread's digits, then the look-back
  uint32_t cnt[PER];
#pragma unroll
  for (int k = 0; k < PER; k++) {
    const int d = tid + k * OS_THREADS;
    uint32_t acc = 0u;
    for (int ww = 0; ww < OS_WARPS; ww++) {
      const uint32_t c = s_wc[ww][d];
      s_wc[ww][d] = acc;
      acc += c;
    }
    cnt[k] = acc;
    lb_publish(stat + (size_t)tile * OS_BINS + d, tile, acc);
  }
  // the look-backs of this thread's digits advance together, each over a
  // window of LB_WIN earlier tiles at a time (all those loads in flight at
  // once); the wait gives up only when none of them advances
  constexpr int LB_WIN = 4;
  unsigned long long excl[PER];
  int jj[PER];
  bool busy[PER];
  bool any = false;
#pragma unroll
  for (int k = 0; k < PER; k++) {
    excl[k] = 0ull;
    jj[k] = tile - 1;
    busy[k] = tile > 0;
    any = any || busy[k];
  }
  long long t0 = clock64();
  while (any) {
    unsigned long long v[PER][LB_WIN];
#pragma unroll
    for (int k = 0; k < PER; k++)
#pragma unroll
      for (int u = 0; u < LB_WIN; u++)
        v[k][u] = (busy[k] && jj[k] - u >= 0)
                      ? lb_load(stat + (size_t)(jj[k] - u) * OS_BINS + tid + k * OS_THREADS)
                      : 0ull;
    any = false;
    bool moved = false;
#pragma unroll
    for (int k = 0; k < PER; k++) {
      if (!busy[k]) continue;
      int j = jj[k];
#pragma unroll
      for (int u = 0; u < LB_WIN; u++) {
        const unsigned long long kind = v[k][u] & ~LB_VAL;
        if (kind == 0ull) break;  // not published yet: wait there
        excl[k] += v[k][u] & LB_VAL;
        moved = true;
        if (kind == LB_PRE || j == 0) {
          busy[k] = false;
          break;
        }
        j--;
      }
      jj[k] = j;
      any = any || busy[k];
    }
    if (moved) {
      t0 = clock64();
    } else if (any && clock64() - t0 > LB_SPIN_CYCLES) {
      atomicOr(status, ST_TIMEOUT);
      break;
    }
  }
#pragma unroll
  for (int k = 0; k < PER; k++) {
    const int d = tid + k * OS_THREADS;
    if (tile > 0) lb_store(stat + (size_t)tile * OS_BINS + d, LB_PRE | (excl[k] + cnt[k]));
    s_base[d] += (uint32_t)excl[k];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < OS_R; r++) {
    const int i = base + r * 32 + lane;
    if (i >= N) continue;
    const uint32_t d = (kk[r] >> shift) & (OS_BINS - 1);
    const uint32_t pos = s_base[d] + s_wc[w][d] + rk[r];
    if (pos < (uint32_t)N) {
      key_out[pos] = kk[r];
      val_out[pos] = vv[r];
    }
  }
}

// Single-pass exclusive scan of popc(in[0..n)) into out[0..n], out[n] =
// total (the node offsets), with the same look-back over tiles.
__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_popc_1p(const uint32_t* __restrict__ in, int n, uint32_t* out,
                   unsigned long long* stat, int* ctr, int* status) {
  __shared__ int s_tile;
  __shared__ uint32_t s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1);
  __syncthreads();
  const int tile = s_tile;
  const int base = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS], sum = 0u;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = base + k < n ? (uint32_t)__popc(in[base + k]) : 0u;
    sum += v[k];
  }
  uint32_t tot;
  uint32_t ex = block_excl_scan(sum, &tot);
  if (threadIdx.x == 0) {
    lb_publish(stat + tile, tile, tot);
    s_excl = (uint32_t)lb_prefix(stat, 1, tile, tot, status);
  }
  __syncthreads();
  ex += s_excl;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) out[n] = s_excl + tot;
}

// ---------------------------------------------------------------- node list
// ss: NULL for one point set, else the subject of every sorted position;
// points of different subjects share no cell (split "above" the root).

// depth of the deepest cell holding sorted points i and i+1 (10: same code;
// -1: different subjects)
__device__ __forceinline__ int delta_at(const uint32_t* sk, const uint32_t* ss, int i) {
  if (ss && ss[i] != ss[i + 1]) return -1;
  const uint32_t x = sk[i] ^ sk[i + 1];
  return x == 0u ? 10 : (__clz(x) - 2) / 3;
}

__device__ __forceinline__ bool same_cell(const uint32_t* sk, const uint32_t* ss, int j,
                                          uint32_t pre, uint32_t sub, int sh) {
  return (sk[j] >> sh) == pre && (!ss || ss[j] == sub);
}

// smallest j <= i in the cell of sorted point i at shift sh
__device__ int gallop_left(const uint32_t* sk, const uint32_t* ss, int i, int sh) {
  const uint32_t pre = sk[i] >> sh, sub = ss ? ss[i] : 0u;
  int good = i, bad = -1, step = 1;
  while (true) {
    const int j = good - step;
    if (j < 0) break;
    if (same_cell(sk, ss, j, pre, sub, sh)) {
      good = j;
      step <<= 1;
    } else {
      bad = j;
      break;
    }
  }
  int L = bad + 1, R = good;
  while (L < R) {
    const int mid = (L + R) >> 1;
    if (same_cell(sk, ss, mid, pre, sub, sh)) R = mid;
    else L = mid + 1;
  }
  return L;
}

// largest j >= i in the cell of sorted point i at shift sh
__device__ int gallop_right(const uint32_t* sk, const uint32_t* ss, int i, int N, int sh) {
  const uint32_t pre = sk[i] >> sh, sub = ss ? ss[i] : 0u;
  int good = i, bad = N, step = 1;
  while (true) {
    const int j = good + step;
    if (j >= N) break;
    if (same_cell(sk, ss, j, pre, sub, sh)) {
      good = j;
      step <<= 1;
    } else {
      bad = j;
      break;
    }
  }
  int L = good, R = bad - 1;
  while (L < R) {
    const int mid = (L + R + 1) >> 1;
    if (same_cell(sk, ss, mid, pre, sub, sh)) L = mid;
    else R = mid - 1;
  }
  return L;
}

// Boundary i (between sorted i and i+1) owns the internal node of depth
// D = delta_i that it is the first depth-D split of (none between subjects).
__global__ void k_owners(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ ss, int N,
                         uint32_t* mask, int32_t* own_a, int32_t* own_b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N - 1) return;
  const int D = delta_at(sk, ss, i);
  if (D < 0) {
    own_a[i] = -1;
    return;
  }
  const int sh = 30 - 3 * D;
  const int a = gallop_left(sk, ss, i, sh);
  bool owner;
  if (D == 10) owner = (a == i);
  else owner = (sk[a] >> (sh - 3)) == (sk[i] >> (sh - 3));
  if (owner) {
    own_a[i] = a;
    own_b[i] = gallop_right(sk, ss, i + 1, N, sh);
    atomicOr(&mask[a], 1u << D);
  } else {
    own_a[i] = -1;
  }
}

__device__ __forceinline__ int node_id(const uint32_t* offs, const uint32_t* mask, int a, int D) {
  return a + (int)offs[a] + __popc(mask[a] & ((1u << D) - 1u));
}

// parent of a node spanning sorted [a, b]: the cell of depth
// Dp = max(delta_{a-1}, delta_b) that contains it (-1 when there is none)
__device__ int parent_of(const uint32_t* sk, const uint32_t* ss, const uint32_t* offs,
                         const uint32_t* mask, int N, int a, int b, int& Dp) {
  Dp = -1;
  if (a > 0) Dp = delta_at(sk, ss, a - 1);
  if (b < N - 1) Dp = max(Dp, delta_at(sk, ss, b));
  if (Dp < 0) return -1;
  const int pa = gallop_left(sk, ss, a, 30 - 3 * Dp);
  return node_id(offs, mask, pa, Dp);
}

// Leaf of every sorted point and the internal node owned by each boundary:
// {skip, count}, {depth, first}, parent, and the internal node's entry in
// the list of internal nodes (its rank among them: its preorder id minus the
// number of leaves before it, which is its first member's position).
__global__ void k_write_nodes(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ ss,
                              int N,
                              const uint32_t* __restrict__ mask, const uint32_t* __restrict__ offs,
                              const int32_t* __restrict__ own_a, const int32_t* __restrict__ own_b,
                              int2* nsc, int2* ninfo, int32_t* nparent, int32_t* inode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // the leaf of sorted point i
  const int leaf = i + (int)offs[i + 1];
  int Dp;
  nsc[leaf] = make_int2(leaf + 1, 1);
  ninfo[leaf] = make_int2(-1, i);
  nparent[leaf] = parent_of(sk, ss, offs, mask, N, i, i, Dp);
  // the internal node owned by boundary i
  if (i < N - 1 && own_a[i] >= 0) {
    const int a = own_a[i], b = own_b[i], D = delta_at(sk, ss, i);
    const int id = node_id(offs, mask, a, D);
    nsc[id] = make_int2(b + 1 + (int)offs[b + 1], b - a + 1);
    ninfo[id] = make_int2(D, a);
    nparent[id] = parent_of(sk, ss, offs, mask, N, a, b, Dp);
    inode[id - a] = id;
  }
}

// ---------------------------------------------------------------- aggregates
// Member sums are carried as unevaluated FP32 pairs (Pair, pair_add): FP64
// arithmetic is the slow path on this GPU.  Each node's pairs are added in
// a fixed order (below), so results are deterministic.
// pair_mean: (hi + lo) / n rounded to FP32.  n < 2^24 (exact in FP32): q = hi / n, then
// one correction by the remainder hi - q n (exact by FMA) plus lo.  Larger
// counts (only the top nodes of trees beyond 2^24 points) divide in FP64.
__device__ __forceinline__ float pair_mean(const Pair& s, int count) {
  if (count >= (1 << 24)) return (float)(((double)s.hi + (double)s.lo) / (double)count);
  const float n = (float)count;
  const float q = __fdiv_rn(s.hi, n);
  const float r = __fadd_rn(__fmaf_rn(-q, n, s.hi), s.lo);
  return __fadd_rn(q, __fdiv_rn(r, n));
}

// Node sums over member ranges.  A node's members are the sorted points
// [first, first + count), so its sums are taken over that range, cut at
// multiples of 32 and 1024 into at most 31 points, at most 31 chunks of 32,
// whole chunks of 1024, at most 31 chunks of 32 and at most 31 points, in
// that order; the chunks' sums are formed once per aggregation.  Every sum
// is a compensated FP32 pair (TwoSum per addition) in a fixed order, so the
// results are deterministic, and no node waits for another.
//
// ADJ: the sums of alpha and beta too (12 components, else 6: xs and p).
// BOX: also the FP32 actual ranges and the nodes' boxes (forward build);
// without, the boxes stored with this tree stay (backward-stage reuse).

// Pass 1, one thread per sorted point, a block per chunk of 1024: the
// leaf's record (and box), the sorted copy of the point's values, and the
// sums (and ranges) of its chunk of 32 and of 1024 (butterfly over lanes;
// lane 0's additions are in a fixed order).
template <bool ADJ, bool BOX>
__global__ void __launch_bounds__(1024)
    k_range_points(TreeArrays t, int N, const float4* __restrict__ raw,
                   const float4* __restrict__ pack, const float4* __restrict__ abpack) {
  constexpr int NS = ADJ ? 12 : 6;
  __shared__ float2 s_sum[32][NS];
  __shared__ float s_box[32][6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const bool valid = i < N;
  float v[NS];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int k = 0; k < NS; k++) v[k] = 0.f;
  if (valid) {
    const int o = (int)t.perm[i];
    const int x = i + (int)t.offs[i + 1];
    float a[3], b[3];
    pack_read(pack, o, a, b);
    v[0] = a[0], v[1] = a[1], v[2] = a[2], v[3] = b[0], v[4] = b[1], v[5] = b[2];
    if (ADJ) {
      pack_read(abpack, o, a, b);
      v[NS - 6] = a[0], v[NS - 5] = a[1], v[NS - 4] = a[2];
      v[NS - 3] = b[0], v[NS - 2] = b[1], v[NS - 1] = b[2];
    }
#pragma unroll
    for (int r = 0; r < NS / 3; r++) {
      const float4 f = make_float4(v[3 * r], v[3 * r + 1], v[3 * r + 2], 0.f);
      t.nrec[4 * x + r] = f;
      t.spt[4 * (size_t)i + r] = f;
    }
    if (BOX) {
      const float4 q = raw[o];
      t.nbox[2 * x] = make_float4(q.x, q.y, q.z, __int_as_float(x + 1));
      t.nbox[2 * x + 1] = make_float4(q.x, q.y, q.z, __int_as_float(1));
      t.sraw[i] = q;
      lo[0] = hi[0] = q.x, lo[1] = hi[1] = q.y, lo[2] = hi[2] = q.z;
    }
  }
  Pair S[NS];
#pragma unroll
  for (int k = 0; k < NS; k++) S[k] = Pair{v[k], 0.f};
  auto butterfly = [&]() {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
      for (int k = 0; k < NS; k++) {
        const float oh = __shfl_xor_sync(0xffffffffu, S[k].hi, d);
        const float ol = __shfl_xor_sync(0xffffffffu, S[k].lo, d);
        pair_add(S[k], make_float2(oh, ol));
      }
      if (BOX)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], d));
          hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], d));
        }
    }
  };
  butterfly();
  const int c1 = i >> 5;  // this warp's chunk of 32
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; k++) s_sum[w][k] = make_float2(S[k].hi, S[k].lo);
#pragma unroll
    for (int a = 0; a < 3; a++) s_box[w][a] = lo[a], s_box[w][3 + a] = hi[a];
    if (valid) {  // a chunk with at least one point
#pragma unroll
      for (int k = 0; k < NS; k++) t.c1sum[12 * (size_t)c1 + k] = make_float2(S[k].hi, S[k].lo);
      if (BOX) {
        t.c1box[2 * (size_t)c1] = make_float4(lo[0], lo[1], lo[2], 0.f);
        t.c1box[2 * (size_t)c1 + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
      }
    }
  }
  __syncthreads();
  if (w != 0) return;
#pragma unroll
  for (int k = 0; k < NS; k++) S[k] = Pair{s_sum[lane][k].x, s_sum[lane][k].y};
#pragma unroll
  for (int a = 0; a < 3; a++) lo[a] = s_box[lane][a], hi[a] = s_box[lane][3 + a];
  butterfly();
  if (lane == 0) {
    const size_t c2 = blockIdx.x;
#pragma unroll
    for (int k = 0; k < NS; k++) t.c2sum[12 * c2 + k] = make_float2(S[k].hi, S[k].lo);
    if (BOX) {
      t.c2box[2 * c2] = make_float4(lo[0], lo[1], lo[2], 0.f);
      t.c2box[2 * c2 + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
}

// The pieces of a member range [a, e): points [a, h1) up to a multiple of
// 32, chunks of 32 [h1, h2) up to a multiple of 1024, chunks of 1024
// [h2, h3), chunks of 32 [h3, h4), points [h4, e); item k of the range is
// the k-th piece in that order.
struct RangeCut {
  int a, h1, h2, h3, h4, e;
  __device__ __forceinline__ RangeCut(int a_, int e_) : a(a_), e(e_) {
    h1 = (a & 31) ? min(e, (a + 31) & ~31) : a;
    const int to1024 = (((h1 + 1023) & ~1023) - h1) >> 5;
    h2 = h1 + 32 * min(to1024, (e - h1) >> 5);
    h3 = (h2 & 1023) ? h2 : h2 + 1024 * ((e - h2) >> 10);
    h4 = h3 + 32 * ((e - h3) >> 5);
  }
  __device__ __forceinline__ int items() const {
    return (h1 - a) + ((h2 - h1) >> 5) + ((h3 - h2) >> 10) + ((h4 - h3) >> 5) + (e - h4);
  }
  // kind 0: sorted point, 1: chunk of 32, 2: chunk of 1024; its index
  __device__ __forceinline__ int2 item(int k) const {
    int n = h1 - a;
    if (k < n) return make_int2(0, a + k);
    k -= n, n = (h2 - h1) >> 5;
    if (k < n) return make_int2(1, (h1 >> 5) + k);
    k -= n, n = (h3 - h2) >> 10;
    if (k < n) return make_int2(2, (h2 >> 10) + k);
    k -= n, n = (h4 - h3) >> 5;
    if (k < n) return make_int2(1, (h3 >> 5) + k);
    return make_int2(0, h4 + k - n);
  }
};

template <int NS, bool BOX>
struct RangeAcc {
  Pair S[NS];
  float lo[3], hi[3];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < NS; k++) S[k] = Pair{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; a++) lo[a] = INFINITY, hi[a] = -INFINITY;
  }
  __device__ __forceinline__ void add(const TreeArrays& t, int2 it) {
    if (it.x == 0) {
#pragma unroll
      for (int q = 0; q < NS / 3; q++) {
        const float4 f = __ldcg(&t.spt[4 * (size_t)it.y + q]);
        pair_add(S[3 * q], f.x);
        pair_add(S[3 * q + 1], f.y);
        pair_add(S[3 * q + 2], f.z);
      }
      if (BOX) {
        const float4 p = __ldcg(&t.sraw[it.y]);
        lo[0] = fminf(lo[0], p.x), lo[1] = fminf(lo[1], p.y), lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x), hi[1] = fmaxf(hi[1], p.y), hi[2] = fmaxf(hi[2], p.z);
      }
    } else {
      const float2* cs = it.x == 1 ? t.c1sum : t.c2sum;
      const float4* cb = it.x == 1 ? t.c1box : t.c2box;
#pragma unroll
      for (int k = 0; k < NS; k++) pair_add(S[k], __ldcg(&cs[12 * (size_t)it.y + k]));
      if (BOX) {
        const float4 u = __ldcg(&cb[2 * (size_t)it.y]), v = __ldcg(&cb[2 * (size_t)it.y + 1]);
        lo[0] = fminf(lo[0], u.x), lo[1] = fminf(lo[1], u.y), lo[2] = fminf(lo[2], u.z);
        hi[0] = fmaxf(hi[0], v.x), hi[1] = fmaxf(hi[1], v.y), hi[2] = fmaxf(hi[2], v.z);
      }
    }
  }
  // every lane's accumulator folded into lane 0's (fixed order)
  __device__ __forceinline__ void warp_fold() {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
      for (int k = 0; k < NS; k++) {
        const float oh = __shfl_down_sync(0xffffffffu, S[k].hi, d);
        const float ol = __shfl_down_sync(0xffffffffu, S[k].lo, d);
        pair_add(S[k], make_float2(oh, ol));
      }
      if (BOX)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          lo[a] = fminf(lo[a], __shfl_down_sync(0xffffffffu, lo[a], d));
          hi[a] = fmaxf(hi[a], __shfl_down_sync(0xffffffffu, hi[a], d));
        }
    }
  }
  // the node's pair sums, record and (BOX) box with skip and count
  __device__ __forceinline__ void write(const TreeArrays& t, int id, int2 sc, bool adj) const {
    float2* isum = reinterpret_cast<float2*>(t.isum);
#pragma unroll
    for (int k = 0; k < NS; k++) isum[12 * (size_t)id + k] = pair_store(S[k]);
    const int n = sc.y;
    t.nrec[4 * id] = make_float4(pair_mean(S[0], n), pair_mean(S[1], n), pair_mean(S[2], n), 0.f);
    t.nrec[4 * id + 1] = make_float4(pair_value(S[3]), pair_value(S[4]), pair_value(S[5]), 0.f);
    if (adj) {
      t.nrec[4 * id + 2] =
          make_float4(pair_value(S[NS - 6]), pair_value(S[NS - 5]), pair_value(S[NS - 4]), 0.f);
      t.nrec[4 * id + 3] = make_float4(pair_mean(S[NS - 3], n), pair_mean(S[NS - 2], n),
                                       pair_mean(S[NS - 1], n), 0.f);
    }
    if (BOX) {
      t.nbox[2 * id] = make_float4(lo[0], lo[1], lo[2], __int_as_float(sc.x));
      t.nbox[2 * id + 1] = make_float4(hi[0], hi[1], hi[2], __int_as_float(n));
    }
  }
};

// Pass 2, one thread per internal node (preorder): a node of at most
// kRangeSmall pieces is summed by its own lane, piece after piece; a larger
// one is queued for pass 3 (its place in the queue does not change its sums).
constexpr int kRangeSmall = 8;
template <bool ADJ, bool BOX>
__global__ void __launch_bounds__(256) k_range_nodes(TreeArrays t, int N) {
  constexpr int NS = ADJ ? 12 : 6;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int nint = (int)t.offs[N];
  if (r - lane >= nint) return;  // the whole warp
  int id = 0, K = 0;
  int2 sc = make_int2(0, 0);
  RangeCut cut(0, 0);
  if (r < nint) {
    id = t.inode[r];
    const int2 inf = t.ninfo[id];
    sc = t.nsc[id];
    cut = RangeCut(inf.y, inf.y + sc.y);
    K = cut.items();
  }
  if (K > 0 && K <= kRangeSmall) {
    RangeAcc<NS, BOX> A;
    A.zero();
    for (int k = 0; k < K; k++) A.add(t, cut.item(k));
    A.write(t, id, sc, ADJ);
  }
  const unsigned big = __ballot_sync(0xffffffffu, K > kRangeSmall);
  if (big) {
    const int leader = __ffs(big) - 1;
    int at = 0;
    if (lane == leader) at = atomicAdd(t.bigc, __popc(big));
    at = __shfl_sync(0xffffffffu, at, leader) + __popc(big & ((1u << lane) - 1u));
    if (K > kRangeSmall) t.bigq[at] = id;
  }
}

// Pass 3, a warp per queued node (grid-stride over the queue): lane j takes
// pieces j, j + 32, ..., then the lanes' sums are folded in a fixed order.
template <bool ADJ, bool BOX>
__global__ void __launch_bounds__(256) k_range_big(TreeArrays t) {
  constexpr int NS = ADJ ? 12 : 6;
  const int lane = threadIdx.x & 31;
  const int nq = *t.bigc;
  const int nw = (int)(gridDim.x * blockDim.x) >> 5;
  for (int q = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += nw) {
    const int id = t.bigq[q];
    const int2 inf = t.ninfo[id], sc = t.nsc[id];
    const RangeCut cut(inf.y, inf.y + sc.y);
    const int K = cut.items();
    RangeAcc<NS, BOX> A;
    A.zero();
    for (int k = lane; k < K; k += 32) A.add(t, cut.item(k));
    A.warp_fold();
    if (lane == 0) A.write(t, id, sc, ADJ);
  }
}

void launch_aggregate(const TreeArrays& t, int N, const float4* raw, const float4* pack,
                      const float4* abpack, bool box, cudaStream_t st) {
  const unsigned nb1 = nblocks(N, 1024), nb2 = nblocks(N, 256);
  const unsigned nb3 = std::min<unsigned>(nb2, 2048);
  cudaMemsetAsync(t.bigc, 0, sizeof(int32_t), st);
  if (abpack && box) {
    k_range_points<true, true><<<nb1, 1024, 0, st>>>(t, N, raw, pack, abpack);
    k_range_nodes<true, true><<<nb2, 256, 0, st>>>(t, N);
    k_range_big<true, true><<<nb3, 256, 0, st>>>(t);
  } else if (abpack) {
    k_range_points<true, false><<<nb1, 1024, 0, st>>>(t, N, raw, pack, abpack);
    k_range_nodes<true, false><<<nb2, 256, 0, st>>>(t, N);
    k_range_big<true, false><<<nb3, 256, 0, st>>>(t);
  } else if (box) {
    k_range_points<false, true><<<nb1, 1024, 0, st>>>(t, N, raw, pack, abpack);
    k_range_nodes<false, true><<<nb2, 256, 0, st>>>(t, N);
    k_range_big<false, true><<<nb3, 256, 0, st>>>(t);
  } else {
    k_range_points<false, false><<<nb1, 1024, 0, st>>>(t, N, raw, pack, abpack);
    k_range_nodes<false, false><<<nb2, 256, 0, st>>>(t, N);
    k_range_big<false, false><<<nb3, 256, 0, st>>>(t);
  }
}

// ---------------------------------------------------------------- layout
size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

size_t n_lists(int64_t groups) { return (size_t)groups * BH_SLICES; }       // slices
size_t n_walk_lists(int64_t groups) { return (size_t)groups * BH_MAX_WK; }  // at most

// Shared scratch of one workspace (capacity n points, 2n + 2 nodes, `groups`
// walk groups); with mem == NULL only the size is computed.
size_t carve_shared(void* mem, int64_t n, int64_t groups, TreeArrays* t, BHLists* L) {
  const size_t N1 = (size_t)n + 1, M = 2 * (size_t)n + 2, nl = n_lists(groups);
  const size_t nb_rs = nblocks(n, RS_TILE), nb_bb = kMaxBBoxBlocks;
  const size_t hist_n = 256 * nb_rs + 1;
  const size_t bsum_n = nblocks((int64_t)std::max<size_t>(hist_n, N1), SCAN_TILE) + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t o_key = take(4 * N1), o_key2 = take(4 * N1), o_perm2 = take(4 * N1),
               o_codes = take(4 * N1), o_ssub = take(4 * N1), o_mask = take(4 * N1),
               o_oa = take(4 * N1),
               o_ob = take(4 * N1), o_hist = take(4 * hist_n), o_hscan = take(4 * (hist_n + 1)),
               o_bsum = take(4 * bsum_n), o_bbp = take(4 * 6 * nb_bb), o_bb = take(4 * 6),
               o_nrec = take(64 * M), o_isum = take(96 * M), o_cnt = take(16),
               o_spt = take(64 * N1), o_sraw = take(16 * N1),
               o_c1s = take(96 * (N1 / 32 + 1)), o_c1b = take(32 * (N1 / 32 + 1)),
               o_c2s = take(96 * (N1 / 1024 + 1)), o_c2b = take(32 * (N1 / 1024 + 1)),
               o_bigq = take(4 * N1), o_bigc = take(4),
               o_part = take(nl * 9 * 32 * sizeof(float2)),
               o_fb = take(nl * 9 * 32 * sizeof(float2)), o_word = take(4 * n_walk_lists(groups)),
               o_wordn = take(4), o_gtick = take(4 * (size_t)groups),
               o_ohist = take(4 * 2 * 256 * 256);
  // the single-pass sort's histograms, tile counters and look-back words and
  // the node-offset scan's look-back words, contiguous (one memset per build)
  const size_t os_tiles = nblocks(n, OS_TILE), sc_tiles = nblocks(std::max<int64_t>(n, 1), SCAN_TILE);
  const size_t os_hist_b = 4 * OS_PASSES * OS_BINS, os_ctr_b = 64;
  const size_t os_stat_b = 8 * OS_PASSES * os_tiles * OS_BINS, sc_stat_b = 8 * sc_tiles;
  const size_t o_osreg = take(os_hist_b + os_ctr_b + os_stat_b + sc_stat_b);
  if (mem) {
    char* b = static_cast<char*>(mem);
    t->key = (uint32_t*)(b + o_key);
    t->key_alt = (uint32_t*)(b + o_key2);
    t->perm_alt = (uint32_t*)(b + o_perm2);
    t->codes = (uint32_t*)(b + o_codes);
    t->ssub = (uint32_t*)(b + o_ssub);
    t->mask = (uint32_t*)(b + o_mask);
    t->own_a = (int32_t*)(b + o_oa);
    t->own_b = (int32_t*)(b + o_ob);
    t->hist = (uint32_t*)(b + o_hist);
    t->hscan = (uint32_t*)(b + o_hscan);
    t->bsum = (uint32_t*)(b + o_bsum);
    t->bbox_part = (float*)(b + o_bbp);
    t->bbox = (float*)(b + o_bb);
    t->nrec = (float4*)(b + o_nrec);
    t->isum = (double*)(b + o_isum);
    t->spt = (float4*)(b + o_spt);
    t->sraw = (float4*)(b + o_sraw);
    t->c1sum = (float2*)(b + o_c1s);
    t->c1box = (float4*)(b + o_c1b);
    t->c2sum = (float2*)(b + o_c2s);
    t->c2box = (float4*)(b + o_c2b);
    t->bigq = (int32_t*)(b + o_bigq);
    t->bigc = (int32_t*)(b + o_bigc);
    t->counts = (int64_t*)(b + o_cnt);
    L->part = (float2*)(b + o_part);
    L->fb = (float2*)(b + o_fb);
    L->worder = (int*)(b + o_word);
    L->worder_n = (int*)(b + o_wordn);
    L->gticket = (int*)(b + o_gtick);
    L->ohist = (int*)(b + o_ohist);
    t->os_hist = (uint32_t*)(b + o_osreg);
    t->os_ctr = (int*)(b + o_osreg + os_hist_b);
    t->os_stat = (unsigned long long*)(b + o_osreg + os_hist_b + os_ctr_b);
    t->sc_stat = (unsigned long long*)(b + o_osreg + os_hist_b + os_ctr_b + os_stat_b);
    t->os_bytes = os_hist_b + os_ctr_b + os_stat_b + sc_stat_b;
  }
  return o;
}

// One step's tree and interaction lists (kept for the backward stage).
size_t carve_slot(void* mem, int64_t n, int64_t groups, int64_t chunks, TreeArrays* t,
                  BHLists* L) {
  const size_t N1 = (size_t)n + 1, M = 2 * (size_t)n + 2, nl = n_lists(groups),
               nw = n_walk_lists(groups);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t o_perm = take(4 * N1), o_offs = take(4 * (N1 + 1)), o_npar = take(4 * M),
               o_inode = take(4 * N1),
               o_nsc = take(8 * M), o_ninfo = take(8 * M), o_nbox = take(32 * M),
               o_ent = take((size_t)chunks * BH_CHUNK * sizeof(int2)),
               o_next = take(4 * (size_t)chunks), o_head = take(4 * nw), o_len = take(4 * nw),
               o_ovx = take(4 * nw), o_used = take(4), o_order = take(4 * nl);
  if (mem) {
    char* b = static_cast<char*>(mem);
    t->perm = (uint32_t*)(b + o_perm);
    t->offs = (uint32_t*)(b + o_offs);
    t->nparent = (int32_t*)(b + o_npar);
    t->inode = (int32_t*)(b + o_inode);
    t->nsc = (int2*)(b + o_nsc);
    t->ninfo = (int2*)(b + o_ninfo);
    t->nbox = (float4*)(b + o_nbox);
    L->ent = (int2*)(b + o_ent);
    L->next = (int*)(b + o_next);
    L->head = (int*)(b + o_head);
    L->len = (int*)(b + o_len);
    L->ovf_x = (int*)(b + o_ovx);
    L->used = (int*)(b + o_used);
    L->order = (int*)(b + o_order);
    L->n_chunks = (int)chunks;
  }
  return o;
}

#define TRY(x)                             \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

// Steps 1-5 for one state (one point set, or the forest f).  abpack = NULL
// for the forward stage.
cudaError_t build(const TreeArrays& t, int N, const float4* raw, const float4* pack,
                  const float4* abpack, const BHForest& f, cudaStream_t st) {
  int launches = 0;
  if (f.S > 0) {
    k_bbox_subjects<<<f.S, kBBoxThreads, 0, st>>>(raw, f.off, f.sbox);
    k_morton_subjects<<<nblocks(N, 256), 256, 0, st>>>(raw, N, f.off, f.S, f.sbox, t.key, t.perm,
                                                       t.codes);
  } else {
    // one point set: codes, the three digit histograms, then the
    // single-pass sort (three kernels) and the single-pass node-offset scan
    const unsigned nbb = std::min<unsigned>(nblocks(N, kBBoxThreads), kMaxBBoxBlocks);
    TRY(cudaMemsetAsync(t.os_hist, 0, t.os_bytes, st));
    k_bbox_partial<<<nbb, kBBoxThreads, 0, st>>>(raw, N, t.bbox_part);
    // the passes alternate between the two key/value buffers and end in
    // key/perm: the codes start in the buffer that makes that so
    uint32_t *k0 = t.key, *v0 = t.perm, *k1 = t.key_alt, *v1 = t.perm_alt;
    if (OS_PASSES & 1) std::swap(k0, k1), std::swap(v0, v1);
    k_morton<<<nblocks(N, 256 * MORTON_PTS), 256, 0, st>>>(raw, N, t.bbox_part, (int)nbb, k0,
                                                             t.codes, t.bbox, t.os_hist, t.mask);
    const unsigned ntiles = nblocks(N, OS_TILE);
    const size_t stat_pass = (size_t)ntiles * OS_BINS;
    for (int p = 0; p < OS_PASSES; p++) {
      k_os_pass<<<ntiles, OS_THREADS, 0, st>>>(k0, p == 0 ? nullptr : v0, N, OS_BITS * p,
                                               t.os_hist + p * OS_BINS, t.os_stat + p * stat_pass,
                                               t.os_ctr + p, t.status, k1, v1);
      std::swap(k0, k1);
      std::swap(v0, v1);
    }
    TRY(cudaGetLastError());
    if (N > 1)
      k_owners<<<nblocks(N - 1, 256), 256, 0, st>>>(t.key, nullptr, N, t.mask, t.own_a, t.own_b);
    k_scan_popc_1p<<<nblocks(N, SCAN_TILE), SCAN_THREADS, 0, st>>>(t.mask, N, t.offs, t.sc_stat,
                                                                   t.os_ctr + OS_PASSES, t.status);
    k_write_nodes<<<nblocks(N, 256), 256, 0, st>>>(t.key, nullptr, N, t.mask, t.offs, t.own_a,
                                                   t.own_b, t.nsc, t.ninfo, t.nparent, t.inode);
    launch_aggregate(t, N, raw, pack, abpack, true, st);
    note_launches(7 + OS_PASSES + (N > 1 ? 1 : 0));
    return cudaGetLastError();
  }
  launches += 2;
  TRY(cudaGetLastError());
  // radix sort, 4 passes of 8 bits (the 30-bit codes end in key/perm)
  const int nb = (int)nblocks(N, RS_TILE);
  uint32_t *k0 = t.key, *v0 = t.perm, *k1 = t.key_alt, *v1 = t.perm_alt;
  auto pass = [&](int shift) -> cudaError_t {
    k_rs_hist<<<nb, RS_THREADS, 0, st>>>(k0, N, shift, t.hist);
    TRY(scan(t.hist, 256 * nb, t.bsum, t.hscan, Ident(), st));
    k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(k0, v0, N, shift, t.hscan, k1, v1);
    std::swap(k0, k1);
    std::swap(v0, v1);
    launches += 5;
    return cudaGetLastError();
  };
  for (int p = 0; p < 4; p++) TRY(pass(8 * p));
  // forest: stable passes over the subject index (most significant digits)
  const uint32_t* ss = nullptr;
  if (f.S > 1) {
    k_subject_keys<<<nblocks(N, 256), 256, 0, st>>>(v0, N, f.off, f.S, k0);
    launches++;
    for (int shift = 0; ((uint32_t)(f.S - 1) >> shift) != 0u; shift += 8) TRY(pass(shift));
    k_forest_finish<<<nblocks(N, 256), 256, 0, st>>>(k0, v0, N, t.codes, t.key, t.perm, t.ssub);
    launches++;
    ss = t.ssub;
  }
  // node list
  TRY(cudaMemsetAsync(t.mask, 0, sizeof(uint32_t) * (size_t)N, st));
  if (N > 1) {
    k_owners<<<nblocks(N - 1, 256), 256, 0, st>>>(t.key, ss, N, t.mask, t.own_a, t.own_b);
    launches++;
  }
  TRY(scan(t.mask, N, t.bsum, t.offs, Popc(), st));
  k_write_nodes<<<nblocks(N, 256), 256, 0, st>>>(t.key, ss, N, t.mask, t.offs, t.own_a, t.own_b,
                                                 t.nsc, t.ninfo, t.nparent, t.inode);
  launch_aggregate(t, N, raw, pack, abpack, true, st);
  note_launches(launches + 3 + 4);
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- host API
namespace {
constexpr size_t kListBudget = size_t(24) << 30;  // interaction-list pools, all slots
constexpr int64_t kMinChunksPerList = 4;
constexpr int64_t kEntriesPerPoint = 512;  // pool per slot: entries per point at most

// Views of the shared scratch and of slot `slot`.
void views(const TreeWork& w, int slot, TreeArrays* t, BHLists* L) {
  *t = TreeArrays{};
  *L = BHLists{};
  carve_shared(w.mem, w.cap_n, w.cap_groups, t, L);
  carve_slot(static_cast<char*>(w.smem) + (size_t)slot * w.slot_bytes, w.cap_n, w.cap_groups,
             w.lcap, t, L);
  t->status = w.d_status;
}

// Walk lists per slice for G groups: the request, else two when one list
// per slice would give fewer than about four waves of walk warps (48
// resident per SM), so that a small tree's walk still fills the GPU.  The
// sums do not depend on it.
int walk_split(const TreeWork& w, int64_t G) {
  if (w.wsplit_req) return w.wsplit_req;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  return G * BH_SLICES < 4 * 48 * (int64_t)sms ? 2 : 1;
}

// Walk groups of a step: the forest's table, or 32-point groups of one set.
WalkGroups walk_groups(const TreeWork& w, const BHStep& b) {
  WalkGroups g{};
  g.leaf = b.leaf;
  g.trunc = b.trunc;
  g.crit = b.crit;
  if (b.f.S > 0) {
    g.groups = b.f.groups;
    g.G = b.f.G;
    g.off = b.f.off;
    g.S = b.f.S;
    g.centers = b.f.centers;
  } else {
    g.G = (int)((b.N + 31) / 32);
  }
  g.wsplit = walk_split(w, g.G);
  return g;
}
}  // namespace

cudaError_t tree_setup() { return cudaSuccess; }

// Chunks in each slot's pool: the requested number of entries per list times
// the list count, else the slot's share of the storage budget (at most a
// quarter of the free memory) capped at kEntriesPerPoint entries per point,
// at least kMinChunksPerList chunks per list.
// The pool size only decides how many slices take the slower re-walk path,
// never the results.
static int64_t pool_chunks(const TreeWork& w, int64_t N, int64_t groups, int slots) {
  const int64_t nl = (int64_t)n_walk_lists(groups);
  if (w.lcap_req > 0) return std::max<int64_t>(1, nl * w.lcap_req / BH_CHUNK);
  size_t budget = kListBudget;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = std::min(budget, fr / 4);
  else cudaGetLastError();
  int64_t per_slot = (int64_t)(budget / (size_t)std::max(slots, 1) /
                               (BH_CHUNK * sizeof(int2) + sizeof(int)));
  per_slot = std::min(per_slot, N * kEntriesPerPoint / BH_CHUNK);
  return std::max(per_slot, nl * kMinChunksPerList);
}

gs_status tree_reserve(TreeWork& w, int64_t N, int slots, cudaStream_t st, int64_t groups) {
  (void)st;
  if (N > (int64_t(1) << 30)) return GS_ERR_INVALID_ARG;
  slots = std::max(slots, 1);
  groups = std::max(groups, (N + 31) / 32);
  if (w.mem && w.cap_n >= N && w.cap_groups >= groups && w.nslots >= slots &&
      w.lcap_req == w.lcap_from_req)
    return GS_OK;
  N = std::max<int64_t>(N, w.cap_n);
  groups = std::max<int64_t>(groups, w.cap_groups);
  slots = std::max(slots, w.nslots);
  tree_release(w);
  const int64_t cap = pool_chunks(w, N, groups, slots);
  TreeArrays t;
  BHLists L;
  const size_t sb = carve_shared(nullptr, N, groups, &t, &L);
  const size_t slb = carve_slot(nullptr, N, groups, cap, &t, &L);
  if (cudaMalloc(&w.mem, sb) != cudaSuccess ||
      cudaMalloc(&w.smem, slb * (size_t)slots) != cudaSuccess) {
    cudaGetLastError();
    tree_release(w);
    return GS_ERR_OOM;
  }
  w.bytes = sb;
  w.slot_bytes = slb;
  w.nslots = slots;
  w.cap_n = N;
  w.cap_groups = groups;
  w.lcap = cap;
  w.lcap_from_req = w.lcap_req;
  views(w, 0, &t, &L);
  w.d_counts = t.counts;
  // no walk order yet: the first walk takes its lists in index order; group
  // tickets start at zero (each combining warp puts its group's back)
  if (cudaMemset(L.worder_n, 0xff, sizeof(int)) != cudaSuccess ||
      cudaMemset(L.gticket, 0, sizeof(int) * (size_t)groups) != cudaSuccess) {
    cudaGetLastError();
    tree_release(w);
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

void tree_release(TreeWork& w) {
  if (w.mem) cudaFree(w.mem);
  if (w.smem) cudaFree(w.smem);
  w.mem = nullptr;
  w.smem = nullptr;
  w.cap_n = 0;
  w.cap_groups = 0;
  w.nslots = 0;
  w.d_counts = nullptr;
}

const char* bh_last_error() { return g_err; }

static gs_status cuda_err(cudaError_t e) {
  snprintf(g_err, sizeof g_err, "%s", cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

gs_status bh_build(TreeWork& w, const BHStep& b, const float4* abpack, bool zero_counts,
                   cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err;
  if (zero_counts && (err = cudaMemsetAsync(t.counts, 0, 16, st)) != cudaSuccess)
    return cuda_err(err);
  if ((err = build(t, (int)b.N, b.raw, b.pack, abpack, b.f, st)) != cudaSuccess)
    return cuda_err(err);
  return GS_OK;
}

gs_status bh_aggregate(TreeWork& w, const BHStep& b, const float4* abpack, bool zero_counts,
                       cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err;
  if (zero_counts && (err = cudaMemsetAsync(t.counts, 0, 16, st)) != cudaSuccess)
    return cuda_err(err);
  launch_aggregate(t, (int)b.N, b.raw, b.pack, abpack, false, st);
  note_launches(3);
  err = cudaGetLastError();
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

gs_status bh_walk(TreeWork& w, const BHStep& b, bool counts, cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = cudaMemsetAsync(L.used, 0, sizeof(int), st);
  if (err == cudaSuccess)
    err = launch_bh_walk(t, (int)b.N, b.raw, b.thr, L, walk_groups(w, b),
                         counts ? t.counts : nullptr, true, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

gs_status bh_eval_fwd(TreeWork& w, const BHStep& b, const FwdEpi& e, bool counts,
                      cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = launch_bh_eval(t, (int)b.N, b.raw, b.thr, L, walk_groups(w, b), false, e,
                                   AdjEpi{}, TracerEpi{}, counts ? t.counts : nullptr, true, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

gs_status bh_eval_adj(TreeWork& w, const BHStep& b, const AdjEpi& e, bool counts,
                      cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = launch_bh_eval(t, (int)b.N, b.raw, b.thr, L, walk_groups(w, b), true, FwdEpi{},
                                   e, TracerEpi{}, counts ? t.counts : nullptr, true, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

gs_status bh_tally(TreeWork& w, const BHStep& b, int64_t* tally, int64_t* stats,
                   cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = cudaMemsetAsync(tally, 0, sizeof(int64_t) * 5 * (size_t)b.N, st);
  if (err == cudaSuccess && stats) err = cudaMemsetAsync(stats, 0, 2 * sizeof(int64_t), st);
  if (err == cudaSuccess)
    err = launch_bh_tally(t, (int)b.N, b.raw, b.thr, walk_groups(w, b), tally, stats, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

void bh_counts(TreeWork& w, int64_t* cnt) {
  cnt[0] = cnt[1] = 0;
  if (w.d_counts) cudaMemcpy(cnt, w.d_counts, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost);
}

namespace {
__global__ void k_export_nodes(TreeArrays t, int m, int32_t* nodes, float* range) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= m) return;
  const int2 inf = t.ninfo[x], sc = t.nsc[x];
  nodes[4 * x + 0] = inf.x;
  nodes[4 * x + 1] = inf.y;
  nodes[4 * x + 2] = sc.y;
  nodes[4 * x + 3] = sc.x;
  const float4 lo = t.nbox[2 * x], hi = t.nbox[2 * x + 1];
  range[6 * x + 0] = lo.x;
  range[6 * x + 1] = lo.y;
  range[6 * x + 2] = lo.z;
  range[6 * x + 3] = hi.x;
  range[6 * x + 4] = hi.y;
  range[6 * x + 5] = hi.z;
}

// Node sums in input units (tests): per preorder node x, {sum q, sum p,
// sum alpha, sum beta} in FP64 from the FP32-pair sums of the aggregation
// (a leaf: its own FP32 record).  The pack holds (q - c) s and mu beta, so
// sum q = (sum xs) / s + n c and sum beta = (sum mu beta) / mu.
__global__ void k_export_sums(TreeArrays t, int m, const double* __restrict__ center,
                              double inv_s, double inv_mu, bool adj, double* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= m) return;
  const int skip = __float_as_int(t.nbox[2 * x].w), count = __float_as_int(t.nbox[2 * x + 1].w);
  double v[12];
  if (skip == x + 1) {
    for (int r = 0; r < 4; r++) {
      const float4 f = (r < 2 || adj) ? t.nrec[4 * x + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      v[3 * r] = f.x, v[3 * r + 1] = f.y, v[3 * r + 2] = f.z;
    }
  } else {
    const float2* isum = reinterpret_cast<const float2*>(t.isum);
    for (int k = 0; k < 12; k++) {
      const float2 pr = (k < 6 || adj) ? isum[12 * (size_t)x + k] : make_float2(0.f, 0.f);
      v[k] = (double)pr.x + (double)pr.y;
    }
  }
  double* o = out + 12 * (size_t)x;
  for (int a = 0; a < 3; a++) {
    o[a] = v[a] * inv_s + (double)count * center[a];
    o[3 + a] = v[3 + a];
    o[6 + a] = v[6 + a];
    o[9 + a] = v[9 + a] * inv_mu;
  }
}
}  // namespace

gs_status tree_export(TreeWork& w, const float4* raw, const float4* pack, int64_t N,
                      uint32_t* codes, int32_t* order, int32_t* nodes, float* range, int64_t cap,
                      int64_t* n_nodes, cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, 0, &t, &L);
  cudaError_t err;
  if ((err = build(t, (int)N, raw, pack, nullptr, BHForest{}, st)) != cudaSuccess)
    return cuda_err(err);
  uint32_t nint = 0;
  if ((err = cudaMemcpyAsync(&nint, t.offs + N, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_err(err);
  const int64_t M = N + (int64_t)nint;
  if (n_nodes) *n_nodes = M;
  if (codes && (err = cudaMemcpyAsync(codes, t.codes, 4 * N, cudaMemcpyDefault, st)) != cudaSuccess)
    return cuda_err(err);
  if (order && (err = cudaMemcpyAsync(order, t.perm, 4 * N, cudaMemcpyDefault, st)) != cudaSuccess)
    return cuda_err(err);
  const int64_t m = std::min(M, cap);
  if ((nodes || range) && m > 0) {
    int32_t* dn = nullptr;
    float* dr = nullptr;
    if ((err = cudaMalloc(&dn, 16 * m)) != cudaSuccess ||
        (err = cudaMalloc(&dr, 24 * m)) != cudaSuccess) {
      if (dn) cudaFree(dn);
      return cuda_err(err);
    }
    k_export_nodes<<<nblocks(m, 256), 256, 0, st>>>(t, (int)m, dn, dr);
    note_launches(1);
    err = cudaGetLastError();
    if (err == cudaSuccess && nodes) err = cudaMemcpyAsync(nodes, dn, 16 * m, cudaMemcpyDefault, st);
    if (err == cudaSuccess && range) err = cudaMemcpyAsync(range, dr, 24 * m, cudaMemcpyDefault, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaFree(dn);
    cudaFree(dr);
    if (err != cudaSuccess) return cuda_err(err);
  }
  return GS_OK;
}

gs_status tree_sums(TreeWork& w, const float4* raw, const float4* pack, const float4* abpack,
                    int64_t N, const double* center, double s, double mu, double* sums,
                    int64_t cap, int64_t* n_nodes, cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, 0, &t, &L);
  cudaError_t err;
  if ((err = build(t, (int)N, raw, pack, abpack, BHForest{}, st)) != cudaSuccess)
    return cuda_err(err);
  uint32_t nint = 0;
  if ((err = cudaMemcpyAsync(&nint, t.offs + N, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_err(err);
  const int64_t M = N + (int64_t)nint;
  if (n_nodes) *n_nodes = M;
  const int64_t m = std::min(M, cap);
  if (!sums || m <= 0) return GS_OK;
  double* d = nullptr;
  if ((err = cudaMalloc(&d, 96 * m)) != cudaSuccess) return cuda_err(err);
  k_export_sums<<<nblocks(m, 256), 256, 0, st>>>(t, (int)m, center, 1.0 / s, 1.0 / mu,
                                                   abpack != nullptr, d);
  note_launches(1);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(sums, d, 96 * m, cudaMemcpyDefault, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  cudaFree(d);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

// ---------------------------------------------------------------- tracers
namespace {
struct TracerScratch {
  uint32_t *key, *key2, *perm2, *hist, *hscan, *bsum;
};
size_t carve_tracers(void* mem, int64_t M, TracerScratch* x, uint32_t** perm, int** mid) {
  const size_t M1 = (size_t)M + 1, nb = nblocks(M, RS_TILE), hist_n = 256 * nb + 1;
  const size_t bsum_n = nblocks((int64_t)hist_n, SCAN_TILE) + 1, G = (size_t)(M + 31) / 32;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t o_key = take(4 * M1), o_key2 = take(4 * M1), o_perm = take(4 * M1),
               o_perm2 = take(4 * M1), o_hist = take(4 * hist_n), o_hscan = take(4 * (hist_n + 1)),
               o_bsum = take(4 * bsum_n), o_mid = take(4 * G);
  if (mem) {
    char* b = static_cast<char*>(mem);
    x->key = (uint32_t*)(b + o_key);
    x->key2 = (uint32_t*)(b + o_key2);
    x->perm2 = (uint32_t*)(b + o_perm2);
    x->hist = (uint32_t*)(b + o_hist);
    x->hscan = (uint32_t*)(b + o_hscan);
    x->bsum = (uint32_t*)(b + o_bsum);
    *perm = (uint32_t*)(b + o_perm);
    *mid = (int*)(b + o_mid);
  }
  return o;
}
}  // namespace

size_t tracer_scratch_bytes(int64_t M) {
  TracerScratch x;
  uint32_t* p;
  int* m;
  return carve_tracers(nullptr, std::max<int64_t>(M, 1), &x, &p, &m);
}

gs_status tracer_order(TreeWork& w, const BHStep& b, const float4* xraw, int64_t M,
                       void* scratch, BHTargets* out, cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  TracerScratch x;
  uint32_t* perm = nullptr;
  int* mid = nullptr;
  carve_tracers(scratch, M, &x, &perm, &mid);
  const int Mi = (int)M;
  k_tracer_codes<<<nblocks(M, 256), 256, 0, st>>>(xraw, Mi, t.bbox, x.key, perm);
  // stable radix sort of the tracer codes, 4 passes of 8 bits
  const int nb = (int)nblocks(M, RS_TILE);
  uint32_t *k0 = x.key, *v0 = perm, *k1 = x.key2, *v1 = x.perm2;
  cudaError_t err = cudaSuccess;
  for (int pass = 0; pass < 4 && err == cudaSuccess; pass++) {
    k_rs_hist<<<nb, RS_THREADS, 0, st>>>(k0, Mi, 8 * pass, x.hist);
    err = scan(x.hist, 256 * nb, x.bsum, x.hscan, Ident(), st);
    k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(k0, v0, Mi, 8 * pass, x.hscan, k1, v1);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  const int G = (int)((M + 31) / 32);
  if (err == cudaSuccess)
    k_tracer_mid<<<nblocks(G, 256), 256, 0, st>>>(k0, Mi, t.key, t.offs, (int)b.N, mid);
  note_launches(3 + 4 * 5);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_err(err);
  out->xraw = xraw;
  out->xperm = v0;  // after an even number of passes: `perm`
  out->xmid = mid;
  out->M = M;
  out->G = G;
  return GS_OK;
}

namespace {
WalkGroups target_groups(const TreeWork& w, const BHStep& b, const BHTargets& x) {
  WalkGroups g = walk_groups(w, b);
  g.groups = nullptr;
  g.G = x.G;
  g.wsplit = walk_split(w, g.G);
  g.xraw = x.xraw;
  g.xrec = x.xrec;
  g.xperm = x.xperm;
  g.xmid = x.xmid;
  g.xM = (int)x.M;
  return g;
}
}  // namespace

gs_status bh_walk_targets(TreeWork& w, const BHStep& b, const BHTargets& x, cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = cudaMemsetAsync(L.used, 0, sizeof(int), st);
  if (err == cudaSuccess)
    err = launch_bh_walk(t, (int)b.N, b.raw, b.thr, L, target_groups(w, b, x), nullptr, false,
                         st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

gs_status bh_eval_targets(TreeWork& w, const BHStep& b, const BHTargets& x, const TracerEpi& e,
                          cudaStream_t st) {
  TreeArrays t;
  BHLists L;
  views(w, b.slot, &t, &L);
  cudaError_t err = launch_bh_eval(t, (int)b.N, b.raw, b.thr, L, target_groups(w, b, x), false,
                                   FwdEpi{}, AdjEpi{}, e, nullptr, false, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

// ---------------------------------------------------------------- cell grid
// Uniform grid of the truncation variant.  The FP32 bounding box of the
// positions; cells of side h = 0.51 r, doubled while the grid would have more
// than grid_cells(N) cells; cell coordinates k = min(trunc((x - lo) * (1/h)),
// n - 1) in FP32; a stable radix sort of (cell id, index).  A pair that passes
// the FP32 truncation test is less than r (1 + 1e-6) apart on every axis,
// i.e. less than 1.97 cells, so its cells differ by at most GRID_REACH = 2.
namespace {
int64_t grid_cells(int64_t N) { return std::min<int64_t>(8 * N + 4096, int64_t(1) << 30); }

struct GridScratch {
  uint32_t *key, *key2, *perm, *perm2, *hist, *hscan, *bsum;
  float *part, *geo;
  int *dims, *cstart;
};

size_t carve_grid(void* mem, int64_t N, GridScratch* g) {
  const size_t N1 = (size_t)N + 1, nb = nblocks(N, RS_TILE), hist_n = 256 * nb + 1;
  const size_t bsum_n = nblocks((int64_t)hist_n, SCAN_TILE) + 1;
  const size_t C1 = (size_t)grid_cells(N) + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t o_key = take(4 * N1), o_key2 = take(4 * N1), o_perm = take(4 * N1),
               o_perm2 = take(4 * N1), o_hist = take(4 * hist_n), o_hscan = take(4 * (hist_n + 1)),
               o_bsum = take(4 * bsum_n), o_part = take(4 * 6 * (size_t)kMaxBBoxBlocks),
               o_geo = take(4 * 4), o_dims = take(4 * 4), o_cstart = take(4 * C1);
  if (mem) {
    char* b = static_cast<char*>(mem);
    g->key = (uint32_t*)(b + o_key);
    g->key2 = (uint32_t*)(b + o_key2);
    g->perm = (uint32_t*)(b + o_perm);
    g->perm2 = (uint32_t*)(b + o_perm2);
    g->hist = (uint32_t*)(b + o_hist);
    g->hscan = (uint32_t*)(b + o_hscan);
    g->bsum = (uint32_t*)(b + o_bsum);
    g->part = (float*)(b + o_part);
    g->geo = (float*)(b + o_geo);
    g->dims = (int*)(b + o_dims);
    g->cstart = (int*)(b + o_cstart);
  }
  return o;
}

// One thread folds the partial boxes and picks the cell side: geo = {lo,
// 1/h}, dims = {nx, ny, nz, C}.  Extents are capped at 1e6 cells before the
// product is taken; a side that cannot be made large enough (a vanishing r)
// puts every point in one cell, which is still correct.
__global__ void k_grid_geometry(const float* __restrict__ part, int nparts, float r, int64_t cap,
                                float* geo, int* dims) {
  if (threadIdx.x != 0) return;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < nparts; k++)
    for (int a = 0; a < 3; a++) {
      lo[a] = fminf(lo[a], part[6 * k + a]);
      hi[a] = fmaxf(hi[a], part[6 * k + 3 + a]);
    }
  float inv = 1.0f / (0.51f * r);
  long long n[3] = {1, 1, 1}, C = 1;
  bool fits = false;
  for (int it = 0; it < 80 && !fits; it++) {
    C = 1;
    for (int a = 0; a < 3; a++) {
      double u = (double)__fmul_rn(__fsub_rn(hi[a], lo[a]), inv);
      if (!(u >= 0.0)) u = 0.0;  // NaN, or an empty box
      if (u > 1e6) u = 1e6;
      n[a] = (long long)u + 1;
      C *= n[a];
    }
    fits = C <= cap;
    if (!fits) inv *= 0.5f;
  }
  if (!fits) n[0] = n[1] = n[2] = 1, C = 1, inv = 0.f;
  for (int a = 0; a < 3; a++) geo[a] = lo[a];
  geo[3] = inv;
  for (int a = 0; a < 3; a++) dims[a] = (int)n[a];
  dims[3] = (int)C;
}

// Cell id of every point (input order) and the identity permutation.
__global__ void k_grid_keys(const float4* __restrict__ raw, int N, const float* __restrict__ geo,
                            const int* __restrict__ dims, uint32_t* key, uint32_t* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 r = raw[i];
  const float x[3] = {r.x, r.y, r.z};
  int c[3];
  for (int a = 0; a < 3; a++) {
    const float u = __fmul_rn(__fsub_rn(x[a], geo[a]), geo[3]);
    const int k = u >= 0.f ? (int)fminf(u, 2.0e9f) : 0;  // NaN -> 0
    c[a] = min(k, dims[a] - 1);
  }
  key[i] = (uint32_t)(((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0]);
  perm[i] = (uint32_t)i;
}

// cstart[c] = the first sorted position whose cell id is >= c, c in [0, C]:
// each sorted position fills the ids after its predecessor's up to its own,
// the last one also those up to C.
__global__ void k_grid_starts(const uint32_t* __restrict__ key, int N, const int* __restrict__ dims,
                              int* cstart) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int64_t cur = key[s], prev = s > 0 ? (int64_t)key[s - 1] : -1;
  for (int64_t c = prev + 1; c <= cur; c++) cstart[c] = s;
  if (s == N - 1)
    for (int64_t c = cur + 1; c <= (int64_t)dims[3]; c++) cstart[c] = N;
}
}  // namespace

size_t grid_scratch_bytes(int64_t N) {
  GridScratch g;
  return carve_grid(nullptr, std::max<int64_t>(N, 1), &g);
}

gs_status grid_rhs(void* scratch, int64_t N, const float4* raw, const float4* pack,
                   const float4* abpack, float r, float thr, bool adj, const FwdEpi& fe,
                   const AdjEpi& ae, int64_t* counts, cudaStream_t st) {
  GridScratch g;
  carve_grid(scratch, N, &g);
  const int Ni = (int)N;
  cudaError_t err = cudaSuccess;
  if (counts && (err = cudaMemsetAsync(counts, 0, 16, st)) != cudaSuccess) return cuda_err(err);
  const unsigned nbb = std::min<unsigned>(nblocks(N, kBBoxThreads), kMaxBBoxBlocks);
  k_bbox_partial<<<nbb, kBBoxThreads, 0, st>>>(raw, Ni, g.part);
  k_grid_geometry<<<1, 32, 0, st>>>(g.part, (int)nbb, r, grid_cells(N), g.geo, g.dims);
  k_grid_keys<<<nblocks(N, 256), 256, 0, st>>>(raw, Ni, g.geo, g.dims, g.key, g.perm);
  err = cudaGetLastError();
  // stable radix sort of the 32-bit cell ids, 4 passes of 8 bits
  const int nb = (int)nblocks(N, RS_TILE);
  uint32_t *k0 = g.key, *v0 = g.perm, *k1 = g.key2, *v1 = g.perm2;
  for (int pass = 0; pass < 4 && err == cudaSuccess; pass++) {
    k_rs_hist<<<nb, RS_THREADS, 0, st>>>(k0, Ni, 8 * pass, g.hist);
    err = scan(g.hist, 256 * nb, g.bsum, g.hscan, Ident(), st);
    k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(k0, v0, Ni, 8 * pass, g.hscan, k1, v1);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  if (err == cudaSuccess) {
    k_grid_starts<<<nblocks(N, 256), 256, 0, st>>>(k0, Ni, g.dims, g.cstart);
    err = cudaGetLastError();
  }
  note_launches(4 + 4 * 5);
  if (err != cudaSuccess) return cuda_err(err);
  GridView v;
  v.perm = v0;
  v.key = k0;
  v.cstart = g.cstart;
  v.dims = g.dims;
  err = launch_grid_eval(v, Ni, pack, abpack, raw, thr, adj, fe, ae, counts, st);
  return err == cudaSuccess ? GS_OK : cuda_err(err);
}

}  // namespace gs
