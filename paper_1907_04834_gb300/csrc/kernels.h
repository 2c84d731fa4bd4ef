// kernels.h -- host-side declarations of the libgs kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gs {

// Process-wide count of kernel launches issued by this library (every
// launcher adds the number of kernels it enqueues).
void note_launches(int n);
long long launches_total();

// ---- exact all-pairs kernels (exact.cu)
constexpr int EX_NT = 256;     // target points per block (one per thread)
constexpr int EX_TILE = 512;   // source points per shared-memory tile
constexpr int EX_STAGES = 3;   // bulk-copy pipeline depth

struct ExactGeom {
  int64_t N;     // points
  int64_t Npad;  // N rounded up to EX_TILE (padding sources have p = 0)
  int n_itiles;  // Npad / EX_NT
  int n_jtiles;  // Npad / EX_TILE
  int J;         // source splits per target tile (1 <= J <= n_jtiles)
};

// Many point sets ("subjects") in one launch: work items (subject, target
// tile) in decreasing subject size, taken from `queue` by persistent blocks.
// Subject s owns rows [off[s], off[s+1]) of the state and pack entries
// [poff[s], poff[s] + npad[s]) (npad a multiple of EX_TILE, padding sources
// with zero momentum).
struct BatchInfo {
  const int2* items;      // {subject, target tile}
  int n_items;
  const int64_t* off;     // S + 1 row offsets
  const int64_t* poff;    // S pack offsets
  const int* npad;        // S padded sizes
  const double* centers;  // S x 3 recentring points
  int* queue;             // next item (zeroed before each launch)
};

cudaError_t exact_setup();
cudaError_t launch_exact_fwd(const float4* pk, const ExactGeom& g, float2* part,
                             unsigned* tickets, const FwdEpi& e, int* status, cudaStream_t st);
cudaError_t launch_exact_adj(const float4* pk, const float4* ab, const ExactGeom& g, float2* part,
                             unsigned* tickets, const AdjEpi& e, int* status, cudaStream_t st);

// Tracer points of the velocity field (Eq. 3): M targets in n_itiles tiles
// of EX_NT (Mpad = n_itiles * EX_NT), J splits of the particle source tiles.
struct TracerGeom {
  int64_t M, Mpad;
  int n_itiles, J;
};
// part: J x 3 x Mpad float2; tickets: n_itiles (zero, reset by the kernel)
cudaError_t launch_tracer(const float4* pk, const ExactGeom& g, const float4* xpk,
                          const TracerGeom& tg, float2* part, unsigned* tickets,
                          const TracerEpi& e, int* status, cudaStream_t st);

// resident blocks per SM of the persistent batched kernels
int batched_resident_blocks(bool adjoint);
cudaError_t launch_batched_fwd(const float4* pk, const BatchInfo& b, const FwdEpi& e, int* status,
                               int blocks, cudaStream_t st);
cudaError_t launch_batched_adj(const float4* pk, const float4* ab, const BatchInfo& b,
                               const AdjEpi& e, int* status, int blocks, cudaStream_t st);

// ---- batched helpers (util.cu)
// centers[s] = bounding-box centre of subject s (one block per subject)
cudaError_t launch_batch_centers(const double* q, const int64_t* off, int S, double* centers,
                                 cudaStream_t st);
// pack entries of every subject (raw: NULL or FP32 positions at the same
// entries)
cudaError_t launch_batch_pack(const double* q, const double* p, int64_t N, const int64_t* off,
                              const int64_t* poff, int S, const double* centers, double s,
                              float4* pack, float4* raw, cudaStream_t st);
cudaError_t launch_batch_pad_zero(float4* base, size_t slot_f4, int slots, const int64_t* off,
                                  const int64_t* poff, const int* npad, int S, cudaStream_t st);
// alpha = 2 lambda (q - X), beta = 0, adjoint pack; r2[i] = |q_i - X_i|^2
cudaError_t launch_batch_adjoint_init(const double* q, const double* X, int64_t N,
                                      const int64_t* off, const int64_t* poff, int S,
                                      double lambda, double* al, double* be, float4* abpack,
                                      double* r2, cudaStream_t st);
// out[s * stride] = scale * Sum over rows of subject s of x (fixed order)
cudaError_t launch_segment_sum(const double* x, const int64_t* off, int S, double scale,
                               double* out, int stride, cudaStream_t st);
// tracer records {(x - c) s, 0} of M points (xraw: NULL or FP32 positions)
cudaError_t launch_pack_points(const double* x, int64_t M, const double* center, double s,
                               float4* xpk, float4* xraw, cudaStream_t st);
// *out = a . b (FP64, fixed order)
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* out, cudaStream_t st);
// y = a x (y may be x)
cudaError_t launch_scale(double* y, const double* x, double a, int64_t n, cudaStream_t st);
// y += a x (product rounded, then the sum: no fused multiply-add)
cudaError_t launch_axpy(double* y, const double* x, double a, int64_t n, cudaStream_t st);
// E[s] = {H[s] + D[s], H[s], D[s]} from E[s*3+1] = H, E[s*3+2] = D
cudaError_t launch_batch_energy(double* E, int S, cudaStream_t st);

// ---- small helpers (util.cu)
// Centre of the bounding box of q [N][3]; part is scratch for 6 * kBoxBlocks
// doubles.
constexpr int kBoxBlocks = 304;
cudaError_t launch_bbox_center(const double* q, int64_t N, double* center, double* part,
                               cudaStream_t st);
cudaError_t launch_pack(const double* q, const double* p, int64_t N, const double* center,
                        double s, float4* pack, float4* raw, cudaStream_t st);
// zero the padding points [N, Npad) of `slots` consecutive packs
cudaError_t launch_pad_zero(float4* base, size_t slot_f4, int slots, int64_t N, int64_t Npad,
                            cudaStream_t st);
// failure-detection self-test: a bounded wait that cannot complete (ST_TIMEOUT)
cudaError_t launch_wait_selftest(int* status, long long limit, cudaStream_t st);
// adjoint pack of (alpha, mu beta) as FP32 (mu = adj_beta_scale(s))
cudaError_t launch_pack_ab(const double* al, const double* be, int64_t N, double mu,
                           float4* abpack, cudaStream_t st);
// alpha = 2 lambda (q - X), beta = 0, adjoint pack; r2[i] = |q_i - X_i|^2
cudaError_t launch_adjoint_init(const double* q, const double* X, int64_t N, double lambda,
                                double* al, double* be, float4* abpack, double* r2,
                                cudaStream_t st);
// out[slot] = scale * Sum_{i<n} x[i] (single block, fixed order)
cudaError_t launch_sum(const double* x, int64_t n, double scale, double* out, cudaStream_t st);
// E = {H + data, H, data} from two sums
cudaError_t launch_energy(const double* H, const double* data, double* E, cudaStream_t st);
// grad = beta + F0 (when the adjoint had no steps to fuse it into)
cudaError_t launch_axpy_grad(const double* be, const double* F0, int64_t n3, double* grad,
                             cudaStream_t st);
cudaError_t launch_check_finite(const double* x, int64_t n, int* status, cudaStream_t st);

}  // namespace gs
