// util.cu -- small per-point kernels: recentring, packing, adjoint
// initialisation, deterministic FP64 reductions, finiteness checks.
#include <atomic>
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace gs {

namespace {

constexpr int kRedThreads = 1024;
constexpr int kBoxThreads = 256;

// Block-wide sum with a fixed reduction tree (deterministic).
__device__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Bounding-box centre of q [N][3] in two launches: k_bbox_part gives each of
// G blocks the min and max of a grid-stride share of the points
// (part[6b..6b+2] low corner, part[6b+3..6b+5] high corner), k_bbox_fin
// folds the G partials.  Min and max are exact, so the centre does not
// depend on the split.
__global__ void k_bbox_part(const double* __restrict__ q, int64_t N, double* __restrict__ part) {
  __shared__ double sh[6][kBoxThreads / 32];
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < 3; a++) {
      const double x = q[3 * i + a];
      lo[a] = fmin(lo[a], x);
      hi[a] = fmax(hi[a], x);
    }
  for (int a = 0; a < 3; a++)
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fmin(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; a++) sh[a][w] = lo[a], sh[3 + a][w] = hi[a];
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    double v = sh[a][0];
    for (int k = 1; k < kBoxThreads / 32; k++) v = a < 3 ? fmin(v, sh[a][k]) : fmax(v, sh[a][k]);
    part[6 * blockIdx.x + a] = v;
  }
}

__global__ void k_bbox_fin(const double* __restrict__ part, int G, double* center) {
  const int l = threadIdx.x;
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int b = l; b < G; b += 32)
    for (int a = 0; a < 3; a++) {
      lo[a] = fmin(lo[a], part[6 * b + a]);
      hi[a] = fmax(hi[a], part[6 * b + 3 + a]);
    }
  for (int a = 0; a < 3; a++)
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fmin(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
  if (l == 0)
    for (int a = 0; a < 3; a++) center[a] = 0.5 * (lo[a] + hi[a]);
}

// Failure-detection self-test: one thread waits, with the bounded wait the
// bulk-copy pipelines use, on an mbarrier that nothing arrives at.  The wait
// gives up after `limit` SM clocks and records ST_TIMEOUT in the status word,
// exactly as a wait on a copy that never lands would; the kernel then ends.
__global__ void k_wait_selftest(int* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) (void)mbar_wait_bounded(&bar, 0u, status, limit);
}

__global__ void k_pack(const double* __restrict__ q, const double* __restrict__ p, int64_t N,
                       const double* __restrict__ center, double s, float4* pack, float4* raw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const PackScale ps{center[0], center[1], center[2], s};
  if (pack) pack_state(pack, i, q + 3 * i, p + 3 * i, ps);
  if (raw)
    raw[i] = make_float4((float)q[3 * i], (float)q[3 * i + 1], (float)q[3 * i + 2], 0.f);
}

__global__ void k_pad_zero(float4* base, size_t slot_f4, int64_t N, int64_t Npad) {
  const int64_t i = N + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  pack_write(base + (size_t)blockIdx.y * slot_f4, i, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
}

// Adjoint pack: alpha, and beta scaled by mu (the pair kernels' convention).
__global__ void k_pack_ab(const double* __restrict__ al, const double* __restrict__ be,
                          int64_t N, double mu, float4* abpack) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  pack_write(abpack, i, (float)al[3 * i], (float)al[3 * i + 1], (float)al[3 * i + 2],
             (float)(mu * be[3 * i]), (float)(mu * be[3 * i + 1]), (float)(mu * be[3 * i + 2]));
}

__global__ void k_adjoint_init(const double* __restrict__ q, const double* __restrict__ X,
                               int64_t N, double lambda, double* al, double* be, float4* abpack,
                               double* r2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double a[3], s = 0.0;
  for (int c = 0; c < 3; c++) {
    double r = q[3 * i + c] - X[3 * i + c];
    s += r * r;
    a[c] = 2.0 * lambda * r;
    al[3 * i + c] = a[c];
    be[3 * i + c] = 0.0;
  }
  r2[i] = s;
  pack_write(abpack, i, (float)a[0], (float)a[1], (float)a[2], 0.f, 0.f, 0.f);
}

__global__ void k_sum(const double* __restrict__ x, int64_t n, double scale, double* out) {
  // each thread sums a contiguous chunk in order, then a fixed tree
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t a = (int64_t)threadIdx.x * chunk;
  const int64_t b = a + chunk < n ? a + chunk : n;
  double v = 0.0;
  for (int64_t i = a; i < b; i++) v += x[i];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = scale * v;
}

__global__ void k_energy(const double* H, const double* data, double* E) {
  E[0] = *H + *data;
  E[1] = *H;
  E[2] = *data;
}

__global__ void k_axpy_grad(const double* be, const double* F0, int64_t n3, double* grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) grad[i] = be[i] + F0[i];
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t n, int* status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// one block per subject: centre of its bounding box
__global__ void k_batch_centers(const double* __restrict__ q, const int64_t* __restrict__ off,
                                double* centers) {
  __shared__ double smin[3][32], smax[3][32];
  const int s = blockIdx.x;
  const int64_t a = off[s], b = off[s + 1];
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x)
    for (int c = 0; c < 3; c++) {
      lo[c] = fmin(lo[c], q[3 * i + c]);
      hi[c] = fmax(hi[c], q[3 * i + c]);
    }
  for (int c = 0; c < 3; c++)
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = fmin(lo[c], __shfl_down_sync(0xffffffffu, lo[c], o));
      hi[c] = fmax(hi[c], __shfl_down_sync(0xffffffffu, hi[c], o));
    }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 3; c++) {
      smin[c][w] = lo[c];
      smax[c][w] = hi[c];
    }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) {
      double mn = smin[c][0], mx = smax[c][0];
      for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
        mn = fmin(mn, smin[c][k]);
        mx = fmax(mx, smax[c][k]);
      }
      centers[3 * s + c] = 0.5 * (mn + mx);
    }
}

__global__ void k_batch_pack(const double* __restrict__ q, const double* __restrict__ p,
                             int64_t N, const int64_t* __restrict__ off,
                             const int64_t* __restrict__ poff, int S,
                             const double* __restrict__ centers, double sc, float4* pack,
                             float4* raw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int s = subject_of(off, S, i);
  const PackScale ps{centers[3 * s], centers[3 * s + 1], centers[3 * s + 2], sc};
  const int64_t e = poff[s] + (i - off[s]);
  pack_state(pack, e, q + 3 * i, p + 3 * i, ps);
  if (raw) raw[e] = make_float4((float)q[3 * i], (float)q[3 * i + 1], (float)q[3 * i + 2], 0.f);
}

// one block per (subject, pack slot): zero the subject's padding entries
__global__ void k_batch_pad_zero(float4* base, size_t slot_f4, const int64_t* __restrict__ off,
                                 const int64_t* __restrict__ poff, const int* __restrict__ npad) {
  const int s = blockIdx.x;
  float4* pk = base + (size_t)blockIdx.y * slot_f4;
  const int64_t n = off[s + 1] - off[s];
  for (int64_t j = n + threadIdx.x; j < npad[s]; j += blockDim.x)
    pack_write(pk, poff[s] + j, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
}

__global__ void k_batch_adjoint_init(const double* __restrict__ q, const double* __restrict__ X,
                                     int64_t N, const int64_t* __restrict__ off,
                                     const int64_t* __restrict__ poff, int S, double lambda,
                                     double* al, double* be, float4* abpack, double* r2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int s = subject_of(off, S, i);
  double a[3], t = 0.0;
  for (int c = 0; c < 3; c++) {
    const double r = q[3 * i + c] - X[3 * i + c];
    t += r * r;
    a[c] = 2.0 * lambda * r;
    al[3 * i + c] = a[c];
    be[3 * i + c] = 0.0;
  }
  r2[i] = t;
  pack_write(abpack, poff[s] + (i - off[s]), (float)a[0], (float)a[1], (float)a[2], 0.f, 0.f,
             0.f);
}

// one block per subject; each thread sums a contiguous chunk, then a fixed tree
__global__ void k_segment_sum(const double* __restrict__ x, const int64_t* __restrict__ off,
                              double scale, double* out, int stride) {
  const int s = blockIdx.x;
  const int64_t a = off[s], b = off[s + 1], n = b - a;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t c0 = a + (int64_t)threadIdx.x * chunk;
  const int64_t c1 = c0 + chunk < b ? c0 + chunk : b;
  double v = 0.0;
  for (int64_t i = c0; i < c1; i++) v += x[i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[(size_t)s * stride] = scale * v;
}

__global__ void k_pack_points(const double* __restrict__ x, int64_t M,
                              const double* __restrict__ c, double s, float4* xpk, float4* xraw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  xpk[i] = make_float4((float)((x[3 * i] - c[0]) * s), (float)((x[3 * i + 1] - c[1]) * s),
                       (float)((x[3 * i + 2] - c[2]) * s), 0.f);
  if (xraw) xraw[i] = make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f);
}

// a . b over n values: each thread sums a contiguous chunk in order, then a
// fixed tree (deterministic)
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                      double* out) {
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t c0 = (int64_t)threadIdx.x * chunk;
  const int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
  double v = 0.0;
  for (int64_t i = c0; i < c1; i++) v += a[i] * b[i];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

__global__ void k_scale(double* y, const double* __restrict__ x, double a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

__global__ void k_axpy(double* y, const double* __restrict__ x, double a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __dadd_rn(y[i], __dmul_rn(a, x[i]));  // rounded product, then sum
}

__global__ void k_batch_energy(double* E, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) E[3 * s] = E[3 * s + 1] + E[3 * s + 2];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

std::atomic<long long> g_launches{0};

}  // namespace

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_batch_centers(const double* q, const int64_t* off, int S, double* centers,
                                 cudaStream_t st) {
  k_batch_centers<<<S, 256, 0, st>>>(q, off, centers);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_pack(const double* q, const double* p, int64_t N, const int64_t* off,
                              const int64_t* poff, int S, const double* centers, double s,
                              float4* pack, float4* raw, cudaStream_t st) {
  k_batch_pack<<<blocks_for(N, 256), 256, 0, st>>>(q, p, N, off, poff, S, centers, s, pack, raw);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_pad_zero(float4* base, size_t slot_f4, int slots, const int64_t* off,
                                  const int64_t* poff, const int* npad, int S, cudaStream_t st) {
  dim3 grid((unsigned)S, (unsigned)slots);
  k_batch_pad_zero<<<grid, 256, 0, st>>>(base, slot_f4, off, poff, npad);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_adjoint_init(const double* q, const double* X, int64_t N,
                                      const int64_t* off, const int64_t* poff, int S,
                                      double lambda, double* al, double* be, float4* abpack,
                                      double* r2, cudaStream_t st) {
  k_batch_adjoint_init<<<blocks_for(N, 256), 256, 0, st>>>(q, X, N, off, poff, S, lambda, al, be,
                                                           abpack, r2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_segment_sum(const double* x, const int64_t* off, int S, double scale,
                               double* out, int stride, cudaStream_t st) {
  k_segment_sum<<<S, kRedThreads, 0, st>>>(x, off, scale, out, stride);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(const double* x, int64_t M, const double* center, double s,
                               float4* xpk, float4* xraw, cudaStream_t st) {
  if (M > 0) {
    k_pack_points<<<blocks_for(M, 256), 256, 0, st>>>(x, M, center, s, xpk, xraw);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* out,
                       cudaStream_t st) {
  k_dot<<<1, kRedThreads, 0, st>>>(a, b, n, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* y, const double* x, double a, int64_t n, cudaStream_t st) {
  k_scale<<<blocks_for(n, 256), 256, 0, st>>>(y, x, a, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t st) {
  k_axpy<<<blocks_for(n, 256), 256, 0, st>>>(y, x, a, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_energy(double* E, int S, cudaStream_t st) {
  k_batch_energy<<<blocks_for(S, 256), 256, 0, st>>>(E, S);
  note_launches(1);
  return cudaGetLastError();
}

int bbox_blocks(int64_t N) {
  const int64_t need = (N + kBoxThreads - 1) / kBoxThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(kBoxBlocks, need));
}

cudaError_t launch_bbox_center(const double* q, int64_t N, double* center, double* part,
                               cudaStream_t st) {
  const int G = bbox_blocks(N);
  k_bbox_part<<<G, kBoxThreads, 0, st>>>(q, N, part);
  k_bbox_fin<<<1, 32, 0, st>>>(part, G, center);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* status, long long limit, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* q, const double* p, int64_t N, const double* center,
                        double s, float4* pack, float4* raw, cudaStream_t st) {
  k_pack<<<blocks_for(N, 256), 256, 0, st>>>(q, p, N, center, s, pack, raw);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pad_zero(float4* base, size_t slot_f4, int slots, int64_t N, int64_t Npad,
                            cudaStream_t st) {
  if (Npad <= N || slots <= 0) return cudaSuccess;
  dim3 grid(blocks_for(Npad - N, 256), (unsigned)slots);
  k_pad_zero<<<grid, 256, 0, st>>>(base, slot_f4, N, Npad);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_ab(const double* al, const double* be, int64_t N, double mu,
                           float4* abpack, cudaStream_t st) {
  k_pack_ab<<<blocks_for(N, 256), 256, 0, st>>>(al, be, N, mu, abpack);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const double* q, const double* X, int64_t N, double lambda,
                                double* al, double* be, float4* abpack, double* r2,
                                cudaStream_t st) {
  k_adjoint_init<<<blocks_for(N, 256), 256, 0, st>>>(q, X, N, lambda, al, be, abpack, r2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* x, int64_t n, double scale, double* out, cudaStream_t st) {
  k_sum<<<1, kRedThreads, 0, st>>>(x, n, scale, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_energy(const double* H, const double* data, double* E, cudaStream_t st) {
  k_energy<<<1, 1, 0, st>>>(H, data, E);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_axpy_grad(const double* be, const double* F0, int64_t n3, double* grad,
                             cudaStream_t st) {
  k_axpy_grad<<<blocks_for(n3, 256), 256, 0, st>>>(be, F0, n3, grad);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int64_t n, int* status, cudaStream_t st) {
  unsigned b = blocks_for(n, 256);
  if (b > 1024) b = 1024;
  if (b == 0) b = 1;
  k_check_finite<<<b, 256, 0, st>>>(x, n, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gs
