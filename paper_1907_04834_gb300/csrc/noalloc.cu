// noalloc.cu -- gs_rhs_exact_noalloc: the exact forward right-hand side
// (F, Phi) for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: applications whose device
// memory is owned entirely by their own pool allocator (which forbids other
// allocations), and latency-critical loops in which an allocation's implicit
// device synchronisation is not acceptable.  This entry point allocates
// nothing: its scratch (recentring point, status word, tickets, the source
// pack, the split partial sums and the bounding-box partials) lives in one
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.  Inputs and outputs are the caller's device
// buffers.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gs.h"
#include "kernels.h"

namespace gs {
namespace {

constexpr int64_t kMaxN = GS_RHS_NOALLOC_MAX_N;
constexpr int kMaxJ = 8;  // source splits per target tile
constexpr size_t kOffCenter = 0;
constexpr size_t kOffStatus = 256;
constexpr size_t kOffTickets = 512;
constexpr size_t kOffPack = kOffTickets + 4 * (kMaxN / EX_NT) + 256;
constexpr size_t kOffPart = kOffPack + sizeof(float4) * 3 * (kMaxN / 2);
constexpr size_t kOffBox = kOffPart + sizeof(float2) * 6 * kMaxJ * kMaxN;
constexpr size_t kScratchBytes = kOffBox + sizeof(double) * 6 * kBoxBlocks;
static_assert(kMaxN % EX_TILE == 0, "the maximum size must be a whole number of tiles");

// The scratch itself.  Host code must not use this name as an address: the
// device address comes from cudaGetSymbolAddress (per device, below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
  bool ready = false;
  char* scratch = nullptr;  // device address of g_scratch on this device
  int num_sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mutex;

// First call on a device (that device current): resolve the scratch's device
// address and configure the kernel's shared-memory limit.
gs_status setup(int dev, DeviceState** out) {
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& d = g_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return GS_ERR_CUDA;
    }
    if (exact_setup() != cudaSuccess ||
        cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return GS_ERR_CUDA;
    }
    d.scratch = static_cast<char*>(ptr);
    d.ready = true;
  }
  *out = &d;
  return GS_OK;
}

bool on_device(const void* ptr, int dev) {
  if (!ptr || reinterpret_cast<uintptr_t>(ptr) % 8 != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_rhs_exact_noalloc(const double* q, const double* p, int64_t N,
                                          double sigma, double* F, double* Phi, void* stream) {
  if (N < 1 || N > kMaxN) return GS_ERR_INVALID_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return GS_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GS_ERR_CUDA;
  }
  if (!on_device(q, dev) || !on_device(p, dev) || !on_device(F, dev) || !on_device(Phi, dev))
    return GS_ERR_INVALID_ARG;
  DeviceState* d = nullptr;
  gs_status s = setup(dev, &d);
  if (s != GS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;

  ExactGeom g;
  g.N = N;
  g.Npad = (N + EX_TILE - 1) / EX_TILE * EX_TILE;
  g.n_itiles = (int)(g.Npad / EX_NT);
  g.n_jtiles = (int)(g.Npad / EX_TILE);
  const int want = (3 * d->num_sms * 2 + g.n_itiles - 1) / g.n_itiles;  // about two waves
  g.J = std::max(1, std::min(std::min(want, kMaxJ), g.n_jtiles));

  double* center = reinterpret_cast<double*>(d->scratch + kOffCenter);
  int* status = reinterpret_cast<int*>(d->scratch + kOffStatus);
  unsigned* tickets = reinterpret_cast<unsigned*>(d->scratch + kOffTickets);
  float4* pack = reinterpret_cast<float4*>(d->scratch + kOffPack);
  float2* part = reinterpret_cast<float2*>(d->scratch + kOffPart);
  double* box = reinterpret_cast<double*>(d->scratch + kOffBox);
  const double sc = std::sqrt(1.4426950408889634 / (2.0 * sigma * sigma));

  // The scratch keeps the previous call's contents: clear what must start at
  // zero (status, tickets, padding sources of the pack).
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, sizeof(unsigned) * g.n_itiles, st);
  if (e == cudaSuccess) e = launch_bbox_center(q, N, center, box, st);
  if (e == cudaSuccess) e = launch_pad_zero(pack, (size_t)(g.Npad / 2) * 3, 1, N, g.Npad, st);
  if (e == cudaSuccess) e = launch_pack(q, p, N, center, sc, pack, nullptr, st);
  if (e == cudaSuccess) {
    FwdEpi ep{};
    ep.q = const_cast<double*>(q);  // not written: h = 0
    ep.p = const_cast<double*>(p);
    ep.F_out = F;
    ep.Phi_out = Phi;
    ep.center = center;
    ep.s = sc;
    ep.phi_scale = 1.0 / (sigma * sigma * sc);
    ep.h = 0.0;
    ep.N = N;
    e = launch_exact_fwd(pack, g, part, tickets, ep, status, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GS_ERR_CUDA;
  }
  return GS_OK;
}
