// peaks.cu -- measured issue rates of the arithmetic units the pair kernels
// are bound by: scalar FP32 FMA, packed f32x2 FMA, and MUFU ex2.  Each thread
// runs 8 independent dependency chains so latency is hidden; rates are
// lane-operations per second over the whole device.
#include "common.cuh"
#include "gs.h"

namespace gs {
namespace {

constexpr int kIters = 4096;

__global__ void k_ffma(float* out, float b, float c) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = threadIdx.x * 1e-6f + k;
  for (int it = 0; it < kIters; it++)
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = fmaf(a[k], b, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; k++) s += a[k];
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void k_ffma2(float* out, float b, float c) {
  f2 a[8];
  const f2 B = f2_dup(b), C = f2_dup(c);
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = f2_make(threadIdx.x * 1e-6f + k, k * 0.5f);
  for (int it = 0; it < kIters; it++)
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = f2_fma(a[k], B, C);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; k++) s += f2_sum(a[k]);
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void k_ex2(float* out) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = (threadIdx.x & 7) * 0.01f + k * 0.1f;
  for (int it = 0; it < kIters; it++)
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = ex2_neg(a[k]);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; k++) s += a[k];
  if (s == 12345.678f) out[threadIdx.x] = s;
}

}  // namespace
}  // namespace gs

using namespace gs;

// out[0] = FP32 FMA lane-ops/s (scalar), out[1] = FP32 lane-ops/s with f32x2
// FMA (2 per lane per instruction), out[2] = MUFU ex2 lane-ops/s.
extern "C" gs_status gs_alu_peaks(int device, double* out) {
  if (!out) return GS_ERR_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GS_ERR_INVALID_ARG;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float* buf = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gs_status rc = GS_OK;
  if (cudaMalloc(&buf, 1024 * sizeof(float)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = GS_ERR_CUDA;
  } else {
    const int threads = 256, blocks = sms * 8;
    const double lanes = (double)threads * blocks * kIters * 8;
    for (int which = 0; which < 3 && rc == GS_OK; which++) {
      float best = 1e30f;
      for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, st);
        if (which == 0) k_ffma<<<blocks, threads, 0, st>>>(buf, 0.9999999f, 1e-7f);
        if (which == 1) k_ffma2<<<blocks, threads, 0, st>>>(buf, 0.9999999f, 1e-7f);
        if (which == 2) k_ex2<<<blocks, threads, 0, st>>>(buf);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = GS_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
      }
      out[which] = lanes * (which == 1 ? 2.0 : 1.0) / (best * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (buf) cudaFree(buf);
  cudaSetDevice(prev);
  return rc;
}
