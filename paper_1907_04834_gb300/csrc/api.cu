// api.cu -- the C ABI of libgs (include/gs.h): contexts, argument checks,
// host/device pointer handling, workspace, and the step drivers that chain
// the kernels for shooting, the adjoint and the single-step calls.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gs.h"
#include "kernels.h"
#include "tree.h"

namespace gs {

// Owning device buffer that only grows.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace gs

using namespace gs;

struct gs_ctx {
  // kernel timing (gs_timing): events around each timed launch group
  struct Timed {
    int cls;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
  long long launch_mark = 0;
  int device = 0;
  int num_sms = 0;
  // source splits of the exact single-set kernels (gs_set_option
  // "exact_splits_fwd" / "exact_splits_adj"; 0 = choose_J)
  int xs_fwd = 0, xs_adj = 0;
  std::string err;
  int* d_status = nullptr;  // device status word (ST_* bits)
  // staging of host inputs / outputs
  DevMem in_q, in_p, in_a, in_b, in_X, out_a, out_b;
  // solver state
  DevMem q, p, al, be, F0, pf, r2, scal;
  DevMem packs, raws, abpacks, ckpt, st64, rho;
  DevMem part, tickets;
  size_t tickets_n = 0;
  // many-subject calls: per-subject layout, queues, energies and gradients
  DevMem bmeta, bout, gd_p, gd_E;
  std::vector<int64_t> bmeta_key;  // layout currently held by bmeta
  // CUDA graphs of the step loops (one cached executable per entry point)
  struct GraphCache {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;  // kernels per replay
  };
  GraphCache g_shoot, g_grad, g_batch, g_flow;
  // tracer points of the velocity field (gs_flow, gs_velocity)
  DevMem in_x, xs, xpks, xpart, xtickets, xraws, xsort;
  DevMem lb;  // L-BFGS vectors
  DevMem grid;  // cell grid of the truncation variant (option "trunc_grid")
  size_t xtickets_n = 0;
  cudaStream_t cap = nullptr;  // capture stream
  bool graphs = true;
  bool trunc_grid = false;  // GS_TRUNC on one point set: uniform grid, not the octree
  TreeWork tree;  // Barnes-Hut workspace (tree.h)
};

namespace {

// Brackets the launches of one kernel class with events on `st` when the
// context's timing is on.
struct KTimer {
  gs_ctx* c;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  static cudaEvent_t get(gs_ctx* c) {
    if (!c->pool.empty()) {
      cudaEvent_t e = c->pool.back();
      c->pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  KTimer(gs_ctx* c_, int cls_, cudaStream_t st_) : c(c_), cls(cls_), st(st_) {
    if (c->timing && (a = get(c))) cudaEventRecord(a, st);
  }
  ~KTimer() {
    if (!a) return;
    cudaEvent_t b = get(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->pending.push_back({cls, a, b});
  }
};

// scal slots (doubles)
enum { SC_CENTER = 0, SC_H0 = 3, SC_H1 = 4, SC_DATA = 5, SC_E = 6, SC_BOX = 16,
       SC_N = SC_BOX + 6 * kBoxBlocks };

constexpr double kLog2e = 1.4426950408889634;

gs_status fail(gs_ctx* c, gs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

gs_status cuda_fail(gs_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Identity of a captured step loop: sizes, parameters and every device
// address the captured launches use.  A graph is replayed only for an equal
// key; anything else is captured again.
struct Key {
  std::vector<unsigned char> b;
  template <class T>
  void add(const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
  void params(const gs_params* prm) {
    add(prm->sigma), add(prm->lambda), add(prm->thresh_sigmas);
    add(prm->T), add(prm->mode), add(prm->ckpt_every), add(prm->flags), add(prm->leaf_size);
    add(prm->criterion), add(prm->sympl_iters);
  }
  void workspace(const gs_ctx* c) {
    for (const DevMem* m : {&c->in_q, &c->in_p, &c->in_X, &c->out_a, &c->out_b, &c->q, &c->p,
                            &c->al, &c->be, &c->F0, &c->pf, &c->r2, &c->scal, &c->packs, &c->raws,
                            &c->abpacks, &c->ckpt, &c->part, &c->tickets, &c->bmeta, &c->bout,
                            &c->gd_p, &c->in_x, &c->xs, &c->xpks, &c->xpart, &c->xtickets,
                            &c->lb, &c->xraws, &c->xsort, &c->grid, &c->st64, &c->rho})
      add(m->p), add(m->bytes);
    add(c->tree.mem), add(c->tree.smem), add(c->tree.lcap), add(c->tree.cap_n);
    add(c->tree.cap_groups), add(c->tree.nslots), add(c->tree.slot_bytes), add(c->d_status);
    add(c->tree.wsplit_req), add(c->xs_fwd), add(c->xs_adj), add(c->trunc_grid);
  }
};

// Runs work(stream): directly, or (graphs on, timing off) as a CUDA graph
// captured on the context's capture stream the first time a key is seen and
// replayed on `st` afterwards.  Work must only enqueue (no allocation, no
// synchronisation).
template <class F>
gs_status run_graphed(gs_ctx* c, gs_ctx::GraphCache& gc, const Key& k, cudaStream_t st, F&& work) {
  if (!c->graphs || c->timing) return work(st);
  if (!(gc.exec && gc.key == k.b)) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
    gc.key.clear();
    if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "stream create");
    const long long l0 = launches_total();
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
    gs_status s = work(c->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    const int n = (int)(launches_total() - l0);
    note_launches(-n);  // captured, not run
    if (s != GS_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s != GS_OK ? s : cuda_fail(c, e, "graph capture");
    }
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gc.exec = nullptr;
      return cuda_fail(c, e, "graph instantiate");
    }
    gc.key = k.b;
    gc.launches = n;
  }
  CK(cudaGraphLaunch(gc.exec, st), "graph launch");
  note_launches(gc.launches);
  return GS_OK;
}

gs_status check_params(gs_ctx* c, const gs_params* prm, bool need_lambda,
                       bool sympl_ok = false) {
  if (!prm) return fail(c, GS_ERR_INVALID_ARG, "params is NULL");
  if (!(prm->sigma > 0.0) || !std::isfinite(prm->sigma))
    return fail(c, GS_ERR_INVALID_ARG, "sigma must be finite and > 0 (got %g)", prm->sigma);
  if (prm->T < 1 || prm->T > 1000000)
    return fail(c, GS_ERR_INVALID_ARG, "T must be in [1, 1e6] (got %d)", prm->T);
  if (prm->mode != GS_EXACT && prm->mode != GS_BH && prm->mode != GS_TRUNC)
    return fail(c, GS_ERR_INVALID_ARG, "mode must be GS_EXACT, GS_BH or GS_TRUNC (got %d)",
                prm->mode);
  if (prm->mode != GS_EXACT && (!(prm->thresh_sigmas > 0.0) || std::isnan(prm->thresh_sigmas)))
    return fail(c, GS_ERR_INVALID_ARG, "thresh_sigmas must be > 0 (got %g)", prm->thresh_sigmas);
  if (need_lambda && (!(prm->lambda >= 0.0) || !std::isfinite(prm->lambda)))
    return fail(c, GS_ERR_INVALID_ARG, "lambda must be finite and >= 0 (got %g)", prm->lambda);
  if (prm->ckpt_every < -1)
    return fail(c, GS_ERR_INVALID_ARG, "ckpt_every must be >= -1 (got %d)", prm->ckpt_every);
  if (prm->flags != 0) return fail(c, GS_ERR_INVALID_ARG, "flags must be 0");
  if (prm->leaf_size < 0 || prm->leaf_size > 32)
    return fail(c, GS_ERR_INVALID_ARG, "leaf_size must be in [0, 32] (got %d)", prm->leaf_size);
  if (prm->criterion != 0 && prm->criterion != 1)
    return fail(c, GS_ERR_INVALID_ARG, "criterion must be 0 or 1 (got %d)", prm->criterion);
  if (prm->criterion == 1 && (prm->mode != GS_BH || !(prm->thresh_sigmas <= 1.0)))
    return fail(c, GS_ERR_INVALID_ARG,
                "criterion 1 (opening angle) needs GS_BH and theta = thresh_sigmas in (0, 1]");
  if (prm->reserved != 0) return fail(c, GS_ERR_INVALID_ARG, "reserved must be 0");
  if (prm->sympl_iters < 0 || prm->sympl_iters > 64)
    return fail(c, GS_ERR_INVALID_ARG, "sympl_iters must be in [0, 64] (got %d)",
                prm->sympl_iters);
  if (prm->sympl_iters != 0 && !sympl_ok)
    return fail(c, GS_ERR_UNSUPPORTED,
                "sympl_iters != 0 (semi-implicit symplectic Euler) is supported by gs_shoot, "
                "gs_shoot_traj and gs_shoot_grad only");
  return GS_OK;
}

gs_status check_n(gs_ctx* c, int64_t N) {
  if (N < 1 || N > (int64_t(1) << 30))
    return fail(c, GS_ERR_INVALID_ARG, "N must be in [1, 2^30] (got %lld)", (long long)N);
  return GS_OK;
}

// Is `ptr` device memory of this context's device?  Host memory (pageable or
// pinned) is reported as host.
gs_status locate(gs_ctx* c, const void* ptr, const char* name, bool* on_device) {
  if (!ptr) return fail(c, GS_ERR_INVALID_ARG, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(ptr) % 8 != 0)
    return fail(c, GS_ERR_INVALID_ARG, "%s is not 8-byte aligned", name);
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *on_device = false;
    return GS_OK;
  }
  if (a.type == cudaMemoryTypeDevice) {
    if (a.device != c->device)
      return fail(c, GS_ERR_INVALID_ARG, "%s lives on device %d, context on %d", name, a.device,
                  c->device);
    *on_device = true;
  } else {
    *on_device = (a.type == cudaMemoryTypeManaged);
  }
  return GS_OK;
}

// Device view of an input array of n doubles (staged if it is host memory).
gs_status input(gs_ctx* c, const double* user, size_t n, const char* name, DevMem& stage,
                cudaStream_t st, const double** out) {
  bool dev = false;
  gs_status s = locate(c, user, name, &dev);
  if (s != GS_OK) return s;
  if (dev) {
    *out = user;
    return GS_OK;
  }
  CK(stage.ensure(n * sizeof(double)), "staging allocation");
  CK(cudaMemcpyAsync(stage.p, user, n * sizeof(double), cudaMemcpyHostToDevice, st), "H2D copy");
  *out = stage.as<double>();
  return GS_OK;
}

// Output check: returns whether `user` is host memory (then the call syncs).
gs_status output(gs_ctx* c, const void* user, const char* name, bool* host) {
  bool dev = false;
  gs_status s = locate(c, user, name, &dev);
  if (s != GS_OK) return s;
  *host = !dev;
  return GS_OK;
}

gs_status copy_out(gs_ctx* c, void* user, const void* src, size_t bytes, cudaStream_t st) {
  CK(cudaMemcpyAsync(user, src, bytes, cudaMemcpyDefault, st), "result copy");
  return GS_OK;
}

gs_status read_status(gs_ctx* c, cudaStream_t st) {
  int h = 0;
  CK(cudaStreamSynchronize(st), "stream synchronize");
  CK(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (h) CK(cudaMemset(c->d_status, 0, sizeof(int)), "status reset");
  if (h & ST_TIMEOUT)
    return fail(c, GS_ERR_TIMEOUT, "a bounded device-side wait gave up (data not delivered)");
  if (h & ST_NONFINITE) return fail(c, GS_ERR_NONFINITE, "non-finite value in a result");
  return GS_OK;
}

// ------------------------------------------------------------------ solver
struct Batch;

struct Solver {
  gs_ctx* c;
  cudaStream_t st;
  int64_t N, Npad;
  int T, mode;
  double sigma, s, h, lambda;
  float thr;  // Barnes-Hut threshold (r*r, FP32)
  float rcut = 0.f;  // truncation radius r (FP32), grid cell size
  bool grid = false;  // truncation over the uniform cell grid
  int leaf;   // Barnes-Hut leaf size (1 = the paper's rule)
  int crit;   // far test: 0 the paper's distance rule, 1 opening angle
  int iters = 0;  // fixed-point passes per step (semi-implicit symplectic Euler)
  ExactGeom gf, ga;
  size_t pack_f4;  // float4 per pack slot
  int slots;       // pack slots allocated
  // Many subjects (exact mode): subject s owns rows [off[s], off[s+1]) and
  // pack entries [poff[s], poff[s] + npad[s]); persistent launches take
  // their work-queue head from `queues` (one zeroed counter per launch).
  const Batch* batch = nullptr;

  float4* pack(int k) const { return c->packs.as<float4>() + (size_t)k * pack_f4; }
  float4* raw(int k) const { return c->raws.as<float4>() + (size_t)k * Npad; }
  float4* abpack(int k) const { return c->abpacks.as<float4>() + (size_t)k * pack_f4; }
  double* scal(int k) const { return c->scal.as<double>() + k; }
};

// Layout of a many-subject call (host copy and device arrays in c->bmeta).
// Exact mode pads every subject's pack to whole source tiles; Barnes-Hut
// mode packs the subjects back to back (pack entry = row) and builds one
// forest per step.
struct Batch {
  int S = 0;
  bool padded = true;
  int64_t N = 0, Ppad = 0;
  std::vector<int64_t> off, poff;
  std::vector<int> npad;
  std::vector<int2> items;   // exact: {subject, target tile}, largest subjects first
  std::vector<int4> groups;  // Barnes-Hut: walk groups {first, count, off[s], off[s+1]}
  BatchInfo dev{};           // device views (queue unset)
  const int4* dgroups = nullptr;
  float* sbox = nullptr;     // Barnes-Hut: 6 S floats of per-subject boxes
  double* E = nullptr;       // S x 3 energies (device)
  int* queues = nullptr;
  int n_queues = 0, next_queue = 0;
  int fwd_blocks = 0, adj_blocks = 0;
};

// Host checks of the offsets and the per-subject layout (padded: exact mode).
gs_status batch_plan(gs_ctx* c, int32_t S, const int64_t* offsets, bool padded, Batch& b) {
  if (S < 1 || S > (1 << 20)) return fail(c, GS_ERR_INVALID_ARG, "S must be in [1, 2^20]");
  if (!offsets) return fail(c, GS_ERR_INVALID_ARG, "offsets is NULL");
  bool dev = false;
  gs_status s = locate(c, offsets, "offsets", &dev);
  if (s != GS_OK) return s;
  if (dev) return fail(c, GS_ERR_INVALID_ARG, "offsets must be host memory");
  if (offsets[0] != 0) return fail(c, GS_ERR_INVALID_ARG, "offsets[0] must be 0");
  b.S = S;
  b.padded = padded;
  b.off.assign(offsets, offsets + S + 1);
  b.poff.resize(S);
  b.npad.resize(S);
  int64_t pp = 0;
  for (int k = 0; k < S; k++) {
    const int64_t n = b.off[k + 1] - b.off[k];
    if (n < 1 || n > (int64_t(1) << 30))
      return fail(c, GS_ERR_INVALID_ARG, "subject %d has %lld points (need 1 .. 2^30)", k,
                  (long long)n);
    b.poff[k] = padded ? pp : b.off[k];
    b.npad[k] = padded ? (int)((n + EX_TILE - 1) / EX_TILE * EX_TILE) : (int)n;
    pp += b.npad[k];
  }
  b.N = b.off[S];
  if (b.N > (int64_t(1) << 30)) return fail(c, GS_ERR_INVALID_ARG, "offsets[S] must be <= 2^30");
  b.Ppad = padded ? pp : (b.N + EX_TILE - 1) / EX_TILE * EX_TILE;
  b.items.clear();
  b.groups.clear();
  if (!padded) {
    for (int k = 0; k < S; k++)
      for (int64_t f = b.off[k]; f < b.off[k + 1]; f += 32)
        b.groups.push_back(make_int4((int)f, (int)std::min<int64_t>(32, b.off[k + 1] - f),
                                     (int)b.off[k], (int)b.off[k + 1]));
    return GS_OK;
  }
  std::vector<int> order(S);
  for (int k = 0; k < S; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b2) { return b.npad[a] > b.npad[b2]; });
  for (int k : order)
    for (int t = 0; t < b.npad[k] / EX_NT; t++) b.items.push_back(make_int2(k, t));
  return GS_OK;
}

// Device copy of the layout, the energies and `n_queues` queue heads (zeroed
// by batch_zero_queues).  The copy is skipped when bmeta already holds it.
gs_status batch_upload(gs_ctx* c, Batch& b, int n_queues, cudaStream_t st) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t S = (size_t)b.S;
  const size_t o_off = 0, o_poff = o_off + up(8 * (S + 1)), o_cen = o_poff + up(8 * S),
               o_E = o_cen + up(24 * S), o_npad = o_E + up(24 * S),
               o_items = o_npad + up(4 * S), o_grp = o_items + up(8 * b.items.size()),
               o_sbox = o_grp + up(16 * b.groups.size()), o_q = o_sbox + up(24 * S),
               total = o_q + up(4 * (size_t)n_queues);
  std::vector<int64_t> key(b.off);
  key.push_back(b.padded);
  key.push_back(n_queues);
  key.push_back(c->num_sms);
  const void* before = c->bmeta.p;
  CK(c->bmeta.ensure(total), "workspace");
  char* base = c->bmeta.as<char>();
  if (c->bmeta.p != before || key != c->bmeta_key) {
    std::vector<char> h(o_q);
    memcpy(h.data() + o_off, b.off.data(), 8 * (S + 1));
    memcpy(h.data() + o_poff, b.poff.data(), 8 * S);
    memcpy(h.data() + o_npad, b.npad.data(), 4 * S);
    memcpy(h.data() + o_items, b.items.data(), 8 * b.items.size());
    memcpy(h.data() + o_grp, b.groups.data(), 16 * b.groups.size());
    // synchronous copy: `h` is freed on return
    CK(cudaStreamSynchronize(st), "stream synchronize");
    CK(cudaMemcpy(base, h.data(), o_q, cudaMemcpyHostToDevice), "layout upload");
    c->bmeta_key = key;
  }
  b.dev.items = reinterpret_cast<const int2*>(base + o_items);
  b.dev.n_items = (int)b.items.size();
  b.dev.off = reinterpret_cast<const int64_t*>(base + o_off);
  b.dev.poff = reinterpret_cast<const int64_t*>(base + o_poff);
  b.dev.npad = reinterpret_cast<const int*>(base + o_npad);
  b.dev.centers = reinterpret_cast<const double*>(base + o_cen);
  b.dev.queue = nullptr;
  b.E = reinterpret_cast<double*>(base + o_E);
  b.dgroups = b.groups.empty() ? nullptr : reinterpret_cast<const int4*>(base + o_grp);
  b.sbox = reinterpret_cast<float*>(base + o_sbox);
  b.queues = reinterpret_cast<int*>(base + o_q);
  b.n_queues = n_queues;
  b.next_queue = 0;
  b.fwd_blocks = std::max(1, std::min(b.dev.n_items, c->num_sms * batched_resident_blocks(false)));
  b.adj_blocks = std::max(1, std::min(b.dev.n_items, c->num_sms * batched_resident_blocks(true)));
  return GS_OK;
}

gs_status batch_zero_queues(gs_ctx* c, Batch& b, cudaStream_t st) {
  b.next_queue = 0;
  if (b.n_queues > 0)
    CK(cudaMemsetAsync(b.queues, 0, sizeof(int) * (size_t)b.n_queues, st), "memset");
  return GS_OK;
}

// Queue head for the next persistent launch.
gs_status batch_take_queue(gs_ctx* c, Batch& b, BatchInfo* bi) {
  if (b.next_queue >= b.n_queues) return fail(c, GS_ERR_INVALID_ARG, "internal: queue heads exhausted");
  *bi = b.dev;
  bi->queue = b.queues + b.next_queue++;
  return GS_OK;
}

constexpr int kMaxSplits = 4096;  // source splits an option or the autotuner may ask for

int choose_J(int n_itiles, int n_jtiles, int slots) {
  // smallest J giving >= 2 full waves, then the J (up to 4 waves) whose last
  // wave is fullest
  int best = 1;
  double best_eff = -1.0;
  int jmin = std::max(1, (2 * slots + n_itiles - 1) / n_itiles);
  int jmax = std::max(jmin, (6 * slots + n_itiles - 1) / n_itiles);
  jmin = std::min(jmin, n_jtiles);
  jmax = std::min(jmax, n_jtiles);
  for (int J = jmin; J <= jmax; J++) {
    double waves = (double)n_itiles * J / slots;
    double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = J;
    }
  }
  return std::max(1, std::min(best, n_jtiles));
}

// slots: pack slots; tree_slots: Barnes-Hut tree/list slots kept at once.
// Zero every pack slot's padding sources (p = 0, and a = b = 0).
gs_status pad_packs(Solver& S, float4* base, int nslots) {
  gs_ctx* c = S.c;
  if (S.batch)
    CK(launch_batch_pad_zero(base, S.pack_f4, nslots, S.batch->dev.off, S.batch->dev.poff,
                             S.batch->dev.npad, S.batch->S, S.st),
       "pad");
  else
    CK(launch_pad_zero(base, S.pack_f4, nslots, S.N, S.Npad, S.st), "pad");
  return GS_OK;
}

// batch: NULL for one point set; else the many-subject layout (exact mode).
gs_status solver_init(gs_ctx* c, Solver& S, int64_t N, const gs_params* prm, int slots,
                      bool adjoint, cudaStream_t st, int tree_slots = 1,
                      const Batch* batch = nullptr) {
  S.c = c;
  S.st = st;
  S.N = N;
  S.batch = batch;
  S.Npad = batch ? batch->Ppad : (N + EX_TILE - 1) / EX_TILE * EX_TILE;
  S.T = prm->T;
  S.mode = prm->mode;
  S.sigma = prm->sigma;
  S.s = std::sqrt(kLog2e / (2.0 * prm->sigma * prm->sigma));
  S.h = 1.0 / (double)prm->T;
  S.lambda = prm->lambda;
  S.crit = prm->criterion;
  S.iters = prm->sympl_iters;
  if (S.crit == 1) {  // opening angle: theta^2
    float th = (float)prm->thresh_sigmas;
    S.thr = th * th;
  } else {
    float r = (float)(prm->thresh_sigmas * prm->sigma);
    S.thr = r * r;
  }
  S.leaf = std::max(1, (int)prm->leaf_size);
  S.pack_f4 = (size_t)(S.Npad / 2) * 3;
  S.slots = slots;
  ExactGeom g;
  g.N = N;
  g.Npad = S.Npad;
  g.n_itiles = (int)(S.Npad / EX_NT);
  g.n_jtiles = (int)(S.Npad / EX_TILE);
  g.J = c->xs_fwd > 0 ? std::min(c->xs_fwd, g.n_jtiles)
                      : choose_J(g.n_itiles, g.n_jtiles, 3 * c->num_sms);
  S.gf = g;
  g.J = c->xs_adj > 0 ? std::min(c->xs_adj, g.n_jtiles)
                      : choose_J(g.n_itiles, g.n_jtiles, 2 * c->num_sms);
  S.ga = g;
  const size_t n3 = (size_t)N * 3;
  CK(c->q.ensure(n3 * 8), "workspace");
  CK(c->p.ensure(n3 * 8), "workspace");
  CK(c->F0.ensure(n3 * 8), "workspace");
  CK(c->pf.ensure((size_t)N * 8), "workspace");
  CK(c->scal.ensure(SC_N * 8), "workspace");
  // pack slots: zero-filled so padding sources carry p = 0 (and a = b = 0)
  size_t pbytes = (size_t)slots * S.pack_f4 * sizeof(float4);
  CK(c->packs.ensure(pbytes), "workspace");
  gs_status ps = pad_packs(S, c->packs.as<float4>(), slots);
  if (ps != GS_OK) return ps;
  if (S.mode != GS_EXACT) {
    size_t rb = (size_t)slots * S.Npad * sizeof(float4);
    CK(c->raws.ensure(rb), "workspace");
  }
  if (adjoint) {
    CK(c->al.ensure(n3 * 8), "workspace");
    CK(c->be.ensure(n3 * 8), "workspace");
    CK(c->r2.ensure((size_t)N * 8), "workspace");
    size_t ab = 2 * S.pack_f4 * sizeof(float4);
    CK(c->abpacks.ensure(ab), "workspace");
    if ((ps = pad_packs(S, c->abpacks.as<float4>(), 2)) != GS_OK) return ps;
  }
  if (batch && batch->padded != (S.mode == GS_EXACT))
    return fail(c, GS_ERR_INVALID_ARG, "internal: batch layout does not match the mode");
  if (S.mode == GS_EXACT && batch) {
    // persistent kernels: no split partials
  } else if (S.mode == GS_EXACT) {
    int J = std::max(S.gf.J, S.ga.J);
    CK(c->part.ensure((size_t)J * 9 * S.Npad * sizeof(float2)), "workspace");
    size_t tn = (size_t)S.gf.n_itiles;
    if (c->tickets_n < tn) {
      CK(c->tickets.ensure(tn * sizeof(unsigned)), "workspace");
      c->tickets_n = tn;
    }
    CK(cudaMemsetAsync(c->tickets.p, 0, tn * sizeof(unsigned), st), "memset");
  } else {
    // the grid variant keeps no trees (one slot holds the pair counters)
    S.grid = S.mode == GS_TRUNC && c->trunc_grid && !batch;
    S.rcut = (float)(prm->thresh_sigmas * prm->sigma);
    gs_status s = tree_reserve(c->tree, N, S.grid ? 1 : tree_slots, st,
                               batch ? (int64_t)batch->groups.size() : 0);
    if (s != GS_OK) return fail(c, s, "Barnes-Hut workspace allocation failed");
    if (S.grid) CK(c->grid.ensure(grid_scratch_bytes(N)), "grid workspace");
  }
  return GS_OK;
}

// Loads (q, p) into the state, computes the recentring point and the pack of
// slot 0 (and its raw FP32 positions in Barnes-Hut mode).
// Pack of the current state into pack slot `slot`.
gs_status solver_pack(Solver& S, int slot) {
  gs_ctx* c = S.c;
  if (S.batch) {
    const Batch& b = *S.batch;
    CK(launch_batch_pack(c->q.as<double>(), c->p.as<double>(), S.N, b.dev.off, b.dev.poff, b.S,
                         b.dev.centers, S.s, S.pack(slot),
                         S.mode != GS_EXACT ? S.raw(slot) : nullptr, S.st),
       "pack");
    return GS_OK;
  }
  CK(launch_pack(c->q.as<double>(), c->p.as<double>(), S.N, S.scal(SC_CENTER), S.s, S.pack(slot),
                 S.mode != GS_EXACT ? S.raw(slot) : nullptr, S.st),
     "pack");
  return GS_OK;
}

gs_status solver_load(Solver& S, const double* q0, const double* p0, int slot) {
  gs_ctx* c = S.c;
  size_t b = (size_t)S.N * 3 * sizeof(double);
  CK(cudaMemcpyAsync(c->q.p, q0, b, cudaMemcpyDeviceToDevice, S.st), "state copy");
  CK(cudaMemcpyAsync(c->p.p, p0, b, cudaMemcpyDeviceToDevice, S.st), "state copy");
  if (S.batch)
    CK(launch_batch_centers(c->q.as<double>(), S.batch->dev.off, S.batch->S,
                            const_cast<double*>(S.batch->dev.centers), S.st),
       "center");
  else
    CK(launch_bbox_center(c->q.as<double>(), S.N, S.scal(SC_CENTER), S.scal(SC_BOX), S.st),
       "center");
  return solver_pack(S, slot);
}

// The forest of a Barnes-Hut batch (S = 0: one point set).
BHForest bh_forest(const Solver& S) {
  BHForest f;
  if (S.batch) {
    const Batch& b = *S.batch;
    f.S = b.S;
    f.off = b.dev.off;
    f.groups = b.dgroups;
    f.G = (int)b.groups.size();
    f.sbox = b.sbox;
    f.centers = b.dev.centers;
  }
  return f;
}

FwdEpi fwd_epi(const Solver& S, int next_slot, double h) {
  FwdEpi e{};
  e.q = S.c->q.as<double>();
  e.p = S.c->p.as<double>();
  e.pack_next = next_slot >= 0 ? S.pack(next_slot) : nullptr;
  e.raw_next = (next_slot >= 0 && S.mode != GS_EXACT) ? S.raw(next_slot) : nullptr;
  e.center = S.scal(SC_CENTER);
  e.s = S.s;
  e.phi_scale = 1.0 / (S.sigma * S.sigma * S.s);
  e.h = h;
  e.N = S.N;
  return e;
}

// One forward right-hand side on pack slot `slot` with epilogue `e`
// (Barnes-Hut: tree and interaction lists built in tree slot `tslot`).
gs_status forward_rhs(Solver& S, int slot, const FwdEpi& e, int64_t* counts, int tslot = 0) {
  gs_ctx* c = S.c;
  if (S.batch && S.mode == GS_EXACT) {
    Batch& bt = *const_cast<Batch*>(S.batch);
    BatchInfo bi;
    gs_status qs = batch_take_queue(c, bt, &bi);
    if (qs != GS_OK) return qs;
    KTimer tm(c, GS_K_EXACT_FWD, S.st);
    CK(launch_batched_fwd(S.pack(slot), bi, e, c->d_status, bt.fwd_blocks, S.st),
       "batched forward kernel");
    return GS_OK;
  }
  if (S.mode == GS_EXACT) {
    KTimer tm(c, GS_K_EXACT_FWD, S.st);
    CK(launch_exact_fwd(S.pack(slot), S.gf, c->part.as<float2>(), c->tickets.as<unsigned>(), e,
                        c->d_status, S.st),
       "exact forward kernel");
    if (counts) {
      counts[0] = S.N * S.N;
      counts[1] = 0;
    }
    return GS_OK;
  }
  if (S.grid) {
    KTimer tm(c, GS_K_BH_FWD, S.st);
    gs_status s = grid_rhs(c->grid.p, S.N, S.raw(slot), S.pack(slot), nullptr, S.rcut, S.thr,
                           false, e, AdjEpi{}, counts ? c->tree.d_counts : nullptr, S.st);
    if (s != GS_OK) return fail(c, s, "truncation grid step failed: %s", bh_last_error());
    return GS_OK;
  }
  BHStep b{tslot, S.N, S.Npad, S.s, S.thr, S.pack(slot), S.raw(slot), bh_forest(S), S.leaf,
           S.mode == GS_TRUNC, S.crit};
  gs_status s;
  {
    KTimer tm(c, GS_K_TREE_BUILD, S.st);
    s = bh_build(c->tree, b, nullptr, counts != nullptr, S.st);
  }
  if (s == GS_OK) {
    KTimer tm(c, GS_K_BH_WALK, S.st);
    s = bh_walk(c->tree, b, counts != nullptr, S.st);
  }
  if (s == GS_OK) {
    KTimer tm(c, GS_K_BH_FWD, S.st);
    s = bh_eval_fwd(c->tree, b, e, counts != nullptr, S.st);
  }
  if (s != GS_OK) return fail(c, s, "Barnes-Hut forward step failed: %s", bh_last_error());
  return GS_OK;
}

// Another forward right-hand side at the positions of the last forward_rhs
// (a fixed-point pass of a semi-implicit step), momenta from pack slot
// `slot`.  Barnes-Hut: the tree and interaction lists of tree slot 0 stay
// valid (the decisions depend on the positions only); only the node sums are
// recomputed before the lists are evaluated.
gs_status forward_rhs_same_q(Solver& S, int slot, const FwdEpi& e, int tslot = 0) {
  gs_ctx* c = S.c;
  if (S.mode == GS_EXACT || S.batch || S.grid) return forward_rhs(S, slot, e, nullptr, tslot);
  BHStep b{tslot, S.N, S.Npad, S.s, S.thr, S.pack(slot), S.raw(slot), bh_forest(S), S.leaf,
           S.mode == GS_TRUNC, S.crit};
  gs_status s;
  {
    KTimer tm(c, GS_K_TREE_BUILD, S.st);
    s = bh_aggregate(c->tree, b, nullptr, false, S.st);
  }
  if (s == GS_OK) {
    KTimer tm(c, GS_K_BH_FWD, S.st);
    s = bh_eval_fwd(c->tree, b, e, false, S.st);
  }
  if (s != GS_OK) return fail(c, s, "Barnes-Hut forward pass failed: %s", bh_last_error());
  return GS_OK;
}

AdjEpi adj_epi(const Solver& S, int next_ab, double h, bool last, double* grad) {
  AdjEpi e{};
  e.al = S.c->al.as<double>();
  e.be = S.c->be.as<double>();
  e.pack_next = next_ab >= 0 ? S.abpack(next_ab) : nullptr;
  e.F0 = last ? S.c->F0.as<double>() : nullptr;
  e.grad = grad;
  e.inv_s2 = 1.0 / (S.sigma * S.sigma);
  e.inv_s = 1.0 / S.s;
  e.mu = adj_beta_scale(S.s);
  e.h = h;
  e.N = S.N;
  return e;
}

// One adjoint right-hand side.  Barnes-Hut: with reuse, tree slot `tslot`
// holds the forward stage's tree and lists for this same state; only the
// sums of alpha and beta are recomputed.  Without, everything is rebuilt.
gs_status adjoint_rhs(Solver& S, int slot, int ab, const AdjEpi& e, int64_t* counts,
                      int tslot = 0, bool reuse = false) {
  gs_ctx* c = S.c;
  if (S.batch && S.mode == GS_EXACT) {
    Batch& bt = *const_cast<Batch*>(S.batch);
    BatchInfo bi;
    gs_status qs = batch_take_queue(c, bt, &bi);
    if (qs != GS_OK) return qs;
    KTimer tm(c, GS_K_EXACT_ADJ, S.st);
    CK(launch_batched_adj(S.pack(slot), S.abpack(ab), bi, e, c->d_status, bt.adj_blocks, S.st),
       "batched adjoint kernel");
    return GS_OK;
  }
  if (S.mode == GS_EXACT) {
    KTimer tm(c, GS_K_EXACT_ADJ, S.st);
    CK(launch_exact_adj(S.pack(slot), S.abpack(ab), S.ga, c->part.as<float2>(),
                        c->tickets.as<unsigned>(), e, c->d_status, S.st),
       "exact adjoint kernel");
    if (counts) {
      counts[0] = S.N * S.N;
      counts[1] = 0;
    }
    return GS_OK;
  }
  if (S.grid) {  // the grid is rebuilt for the state: it is cheap beside the sums
    KTimer tm(c, GS_K_BH_ADJ, S.st);
    gs_status s = grid_rhs(c->grid.p, S.N, S.raw(slot), S.pack(slot), S.abpack(ab), S.rcut,
                           S.thr, true, FwdEpi{}, e, counts ? c->tree.d_counts : nullptr, S.st);
    if (s != GS_OK) return fail(c, s, "truncation grid step failed: %s", bh_last_error());
    return GS_OK;
  }
  BHStep b{tslot, S.N, S.Npad, S.s, S.thr, S.pack(slot), S.raw(slot), bh_forest(S), S.leaf,
           S.mode == GS_TRUNC, S.crit};
  gs_status s;
  if (reuse) {
    KTimer tm(c, GS_K_TREE_BUILD, S.st);
    s = bh_aggregate(c->tree, b, S.abpack(ab), counts != nullptr, S.st);
  } else {
    {
      KTimer tm(c, GS_K_TREE_BUILD, S.st);
      s = bh_build(c->tree, b, S.abpack(ab), counts != nullptr, S.st);
    }
    if (s == GS_OK) {
      KTimer tm(c, GS_K_BH_WALK, S.st);
      s = bh_walk(c->tree, b, counts != nullptr, S.st);
    }
  }
  if (s == GS_OK) {
    KTimer tm(c, GS_K_BH_ADJ, S.st);
    s = bh_eval_adj(c->tree, b, e, counts != nullptr, S.st);
  }
  if (s != GS_OK) return fail(c, s, "Barnes-Hut adjoint step failed: %s", bh_last_error());
  return GS_OK;
}

// Objective and gradient (Eq. 2 and the discrete adjoint) of one point set
// of N rows (batch NULL) or of every subject of `batch`: grad_setup sizes
// the workspace (allocations, never captured), grad_enqueue enqueues the
// whole forward and backward pass on `st` (capturable).  Inputs are device
// arrays; E receives 3 doubles per subject, grad N x 3, q1 (optional) q(1).
struct GradRun {
  Solver S;
  Batch* batch = nullptr;
  int T = 0, ck = 0, nck = 0;
  double* ckq = nullptr;
  // semi-implicit scheme (M = S.iters passes per step): the FP64 state of
  // every step of a segment, and M pack slots for the passes' momenta
  double* st64 = nullptr;
  int pass0 = 0;  // first pack slot of the passes
};

gs_status grad_setup(gs_ctx* c, int64_t N, const gs_params* prm, Batch* batch, cudaStream_t st,
                     GradRun& R) {
  gs_status s;
  R.batch = batch;
  R.T = prm->T;
  // -1: every round(sqrt(T))-th state, the spacing that minimises the kept
  // states plus a segment's recomputed ones, T/k + k
  const int ce = prm->ckpt_every < 0 ? std::max(1, (int)std::lround(std::sqrt((double)R.T)))
                                     : prm->ckpt_every;
  R.ck = ce > 0 && ce < R.T ? ce : 0;
  // pack slots: every step (store-all) or one segment (checkpointing)
  const int steps = R.ck ? R.ck + 1 : R.T + 1;
  const int M = prm->sympl_iters;
  const int slots = steps + M;
  R.pass0 = steps;
  // Barnes-Hut: one tree slot per step kept for the backward stage (a
  // segment's steps with checkpointing)
  const int tslots = prm->mode != GS_EXACT ? (R.ck ? R.ck : R.T) : 1;
  if ((s = solver_init(c, R.S, N, prm, slots, true, st, tslots, batch))) return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  R.nck = R.ck ? (R.T + R.ck - 1) / R.ck : 0;
  if (R.ck) CK(c->ckpt.ensure((size_t)R.nck * 2 * b3), "checkpoint allocation");
  R.ckq = R.ck ? c->ckpt.as<double>() : nullptr;
  if (M > 0) {
    CK(c->st64.ensure((size_t)(steps - 1) * 2 * b3 + (size_t)N * 3 * sizeof(double)),
       "state allocation");
    R.st64 = c->st64.as<double>();
    CK(c->rho.ensure(b3), "workspace");
  }
  return GS_OK;
}

gs_status grad_enqueue(GradRun& R, const double* dq0, const double* dp0, const double* dX,
                       double* E, double* grad, double* q1, cudaStream_t st) {
  gs_status s;
  Solver& S = R.S;
  S.st = st;
  gs_ctx* c = S.c;
  Batch* batch = R.batch;
  const int64_t N = S.N;
  const int T = R.T, ck = R.ck, nck = R.nck;
  double* ckq = R.ckq;
  const size_t n3 = (size_t)N * 3, b3 = n3 * sizeof(double);
  if (batch && (s = batch_zero_queues(c, *batch, st))) return s;
  if ((s = solver_load(S, dq0, dp0, 0))) return s;

  const int M = S.iters;
  // FP64 state j of the semi-implicit scheme's backward sweep (the passes'
  // epilogues form p^k + h Phi from it)
  auto save_state = [&](int j) -> gs_status {
    if (M == 0) return GS_OK;
    double* dst = R.st64 + (size_t)j * 2 * n3;
    CK(cudaMemcpyAsync(dst, c->q.p, b3, cudaMemcpyDeviceToDevice, st), "state copy");
    CK(cudaMemcpyAsync(dst + n3, c->p.p, b3, cudaMemcpyDeviceToDevice, st), "state copy");
    return GS_OK;
  };
  // One step from pack slot `in` (tree slot ts), the next state's pack into
  // `outs`; first: also F(q0, p0) and p0.F.  Semi-implicit: M passes at
  // fixed q (pack slots pass0 ..), then the update with the last pass.
  auto fwd_step = [&](int in, int outs, int ts, bool first) -> gs_status {
    for (int m = 0; m <= M; m++) {
      const bool last = m == M;
      FwdEpi e = fwd_epi(S, last ? outs : R.pass0 + m, S.h);
      e.iterate = !last;
      if (first && m == 0) {
        e.F_out = c->F0.as<double>();
        e.pf_part = c->pf.as<double>();
      }
      const int from = m == 0 ? in : R.pass0 + m - 1;
      gs_status r = m == 0 ? forward_rhs(S, from, e, nullptr, ts)
                           : forward_rhs_same_q(S, from, e, ts);
      if (r) return r;
    }
    return GS_OK;
  };

  // ---- forward pass
  for (int k = 0; k < T; k++) {
    int in = ck ? (k & 1) : k, outs = ck ? ((k + 1) & 1) : k + 1;
    if (ck && k % ck == 0) {
      double* dst = ckq + (size_t)(k / ck) * 2 * n3;
      CK(cudaMemcpyAsync(dst, c->q.p, b3, cudaMemcpyDeviceToDevice, st), "checkpoint");
      CK(cudaMemcpyAsync(dst + n3, c->p.p, b3, cudaMemcpyDeviceToDevice, st), "checkpoint");
    }
    if (!ck && (s = save_state(k))) return s;
    if ((s = fwd_step(in, outs, ck ? 0 : k, k == 0))) return s;
  }
  if (q1) CK(cudaMemcpyAsync(q1, c->q.p, b3, cudaMemcpyDeviceToDevice, st), "q1 copy");
  // ---- adjoint initialisation and objective
  if (batch) {
    CK(launch_batch_adjoint_init(c->q.as<double>(), dX, N, batch->dev.off, batch->dev.poff,
                                 batch->S, S.lambda, c->al.as<double>(), c->be.as<double>(),
                                 S.abpack(0), c->r2.as<double>(), st),
       "adjoint init");
    CK(launch_segment_sum(c->pf.as<double>(), batch->dev.off, batch->S, 0.5, E + 1, 3, st), "sum");
    CK(launch_segment_sum(c->r2.as<double>(), batch->dev.off, batch->S, S.lambda, E + 2, 3, st),
       "sum");
    CK(launch_batch_energy(E, batch->S, st), "energy");
  } else {
    CK(launch_sum(c->pf.as<double>(), N, 0.5, S.scal(SC_H0), st), "sum");
    CK(launch_adjoint_init(c->q.as<double>(), dX, N, S.lambda, c->al.as<double>(),
                           c->be.as<double>(), S.abpack(0), c->r2.as<double>(), st),
       "adjoint init");
    CK(launch_sum(c->r2.as<double>(), N, S.lambda, S.scal(SC_DATA), st), "sum");
    CK(launch_energy(S.scal(SC_H0), S.scal(SC_DATA), E, st), "energy");
  }
  // ---- backward pass
  int ab = 0;
  // Backward step k on pack and tree slot `slot` (state j of st64).
  // Semi-implicit: the passes r_1 .. r_M are recomputed from state k, then
  // the adjoint terms at r_M with (alpha, beta) and at r_{m-1} with (0,
  // rho_m), m = M .. 1; alpha and beta accumulate dE/dq^k and dE/dp^k (the
  // discrete adjoint of the step, as the oracle's gsref_shoot_grad_sympl).
  auto back_step = [&](int k, int slot, int j) -> gs_status {
    if (M == 0) {
      AdjEpi e = adj_epi(S, ab ^ 1, S.h, k == 0, grad);
      gs_status r = adjoint_rhs(S, slot, ab, e, nullptr, slot, true);
      ab ^= 1;
      return r;
    }
    const double* src = R.st64 + (size_t)j * 2 * n3;
    CK(cudaMemcpyAsync(c->q.p, src, b3, cudaMemcpyDeviceToDevice, st), "state copy");
    CK(cudaMemcpyAsync(c->p.p, src + n3, b3, cudaMemcpyDeviceToDevice, st), "state copy");
    for (int m = 1; m <= M; m++) {
      FwdEpi e = fwd_epi(S, R.pass0 + m - 1, S.h);
      e.iterate = true;
      gs_status r = forward_rhs_same_q(S, m == 1 ? slot : R.pass0 + m - 2, e, slot);
      if (r) return r;
    }
    for (int m = M; m >= 0; m--) {
      AdjEpi e = adj_epi(S, ab ^ 1, S.h, k == 0 && m == 0, grad);
      e.rho = c->rho.as<double>();
      e.pack_rho = m > 0;
      gs_status r = adjoint_rhs(S, m == 0 ? slot : R.pass0 + m - 1, ab, e, nullptr, slot, true);
      ab ^= 1;
      if (r) return r;
    }
    return GS_OK;
  };
  if (!ck) {
    for (int k = T - 1; k >= 0; k--)
      if ((s = back_step(k, k, k))) return s;
  } else {
    for (int seg = nck - 1; seg >= 0; seg--) {
      const int k0 = seg * ck, k1 = std::min(T, k0 + ck);
      const double* src = ckq + (size_t)seg * 2 * n3;
      CK(cudaMemcpyAsync(c->q.p, src, b3, cudaMemcpyDeviceToDevice, st), "restore");
      CK(cudaMemcpyAsync(c->p.p, src + n3, b3, cudaMemcpyDeviceToDevice, st), "restore");
      if ((s = solver_pack(S, 0))) return s;
      for (int k = k0; k < k1; k++) {
        if ((s = save_state(k - k0))) return s;
        // the last step of the segment only builds its tree and lists
        // (its state update is not needed): the adjoint reuses them
        if (k < k1 - 1) {
          if ((s = fwd_step(k - k0, k - k0 + 1, k - k0, false))) return s;
        } else if (S.mode != GS_EXACT) {
          FwdEpi e = fwd_epi(S, -1, 0.0);
          if ((s = forward_rhs(S, k - k0, e, nullptr, k - k0))) return s;
        }
      }
      for (int k = k1 - 1; k >= k0; k--)
        if ((s = back_step(k, k - k0, k - k0))) return s;
    }
  }
  return GS_OK;
}

// Objective and gradient of every subject of b (layout uploaded): energies
// into b.E, gradients into dgrad.
gs_status batched_grad(gs_ctx* c, Batch& b, const double* dq0, const double* dp0,
                       const double* dX, const gs_params* prm, double* dgrad, cudaStream_t st) {
  gs_status s;
  GradRun R;
  if ((s = grad_setup(c, b.N, prm, &b, st, R))) return s;
  Key k;
  k.add(b.N), k.params(prm), k.add(dq0), k.add(dp0), k.add(dX), k.add(dgrad), k.workspace(c);
  for (int64_t v : c->bmeta_key) k.add(v);
  return run_graphed(c, c->g_batch, k, st, [&](cudaStream_t s2) {
    return grad_enqueue(R, dq0, dp0, dX, b.E, dgrad, nullptr, s2);
  });
}

// Forward shooting of one point set: state left in c->q, c->p; with H,
// H(q0, p0) and H(q1, p1) in scal[SC_H0], scal[SC_H1] (capturable).
// qtraj, ptraj: NULL or (T + 1) x N x 3 outputs receiving every step's state
// (not captured: gs_shoot_traj launches eagerly).
gs_status shoot_enqueue(Solver& S, const double* dq0, const double* dp0, bool H,
                        cudaStream_t st, double* qtraj = nullptr, double* ptraj = nullptr) {
  gs_status s;
  gs_ctx* c = S.c;
  S.st = st;
  const int64_t N = S.N;
  if ((s = solver_load(S, dq0, dp0, 0))) return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  auto keep = [&](int k) -> gs_status {
    if (qtraj)
      CK(cudaMemcpyAsync(qtraj + (size_t)k * N * 3, c->q.p, b3, cudaMemcpyDefault, st),
         "trajectory copy");
    if (ptraj)
      CK(cudaMemcpyAsync(ptraj + (size_t)k * N * 3, c->p.p, b3, cudaMemcpyDefault, st),
         "trajectory copy");
    return GS_OK;
  };
  if ((s = keep(0))) return s;
  // Each step: S.iters fixed-point passes (the epilogue writes the next pack
  // with (q^k, p^k + h Phi) and leaves the state), then the update pass; with
  // S.iters = 0 the explicit Euler step.  Packs alternate between two slots.
  int cur = 0;
  for (int k = 0; k < S.T; k++) {
    for (int m = 0; m <= S.iters; m++) {
      FwdEpi e = fwd_epi(S, cur ^ 1, S.h);
      e.iterate = m < S.iters;
      const bool h0 = k == 0 && m == 0 && H;
      if (h0) e.pf_part = c->pf.as<double>();
      if ((s = m == 0 ? forward_rhs(S, cur, e, nullptr) : forward_rhs_same_q(S, cur, e)))
        return s;
      if (h0) CK(launch_sum(c->pf.as<double>(), N, 0.5, S.scal(SC_H0), st), "sum");
      cur ^= 1;
    }
    if ((s = keep(k + 1))) return s;
  }
  if (H) {
    FwdEpi e = fwd_epi(S, -1, 0.0);
    e.pf_part = c->pf.as<double>();
    if ((s = forward_rhs(S, cur, e, nullptr))) return s;
    CK(launch_sum(c->pf.as<double>(), N, 0.5, S.scal(SC_H1), st), "sum");
  }
  return GS_OK;
}

// Tracer points (Eq. 3) moving with the particles of solver S: workspace
// for M points (tracer_setup, never captured) and one step of them
// (tracer_step: targets = tracer records of slot k & 1, sources = the
// particles' pack slot k & 1, next records into slot (k + 1) & 1).
struct Tracers {
  int64_t M = 0;
  TracerGeom tg{};
  bool tree = false;  // Barnes-Hut: tracers walk the particles' tree
  float4* xpk(const gs_ctx* c, int k) const { return c->xpks.as<float4>() + (size_t)k * tg.Mpad; }
  float4* xraw(const gs_ctx* c, int k) const {
    return c->xraws.as<float4>() + (size_t)k * tg.Mpad;
  }
};

gs_status tracer_setup(gs_ctx* c, const Solver& S, int64_t M, cudaStream_t st, Tracers& X) {
  X.M = M;
  X.tg.M = M;
  X.tg.n_itiles = (int)((std::max<int64_t>(M, 1) + EX_NT - 1) / EX_NT);
  X.tg.Mpad = (int64_t)X.tg.n_itiles * EX_NT;
  X.tg.J = choose_J(X.tg.n_itiles, S.gf.n_jtiles, 3 * c->num_sms);
  CK(c->xs.ensure((size_t)std::max<int64_t>(M, 1) * 24), "workspace");
  CK(c->xpks.ensure(2 * (size_t)X.tg.Mpad * sizeof(float4)), "workspace");
  CK(c->xpart.ensure((size_t)X.tg.J * 3 * X.tg.Mpad * sizeof(float2)), "workspace");
  const size_t tn = (size_t)X.tg.n_itiles;
  if (c->xtickets_n < tn) {
    CK(c->xtickets.ensure(tn * sizeof(unsigned)), "workspace");
    c->xtickets_n = tn;
  }
  CK(cudaMemsetAsync(c->xtickets.p, 0, tn * sizeof(unsigned), st), "memset");
  X.tree = S.mode == GS_BH;
  if (X.tree) {
    // FP32 tracer positions, the tracer sort's scratch, list room for the
    // tracer groups
    CK(c->xraws.ensure(2 * (size_t)X.tg.Mpad * sizeof(float4)), "workspace");
    CK(c->xsort.ensure(tracer_scratch_bytes(M)), "workspace");
    gs_status s = tree_reserve(c->tree, S.N, 1, st, (M + 31) / 32);
    if (s != GS_OK) return fail(c, s, "Barnes-Hut workspace allocation failed");
  }
  return GS_OK;
}

// Barnes-Hut tracer step k on the particles' tree of state k (tree slot 0,
// built by the particle step that precedes it).
gs_status tracer_bh_step(const Solver& S, const Tracers& X, int k, double h, double* v_out,
                         cudaStream_t st) {
  gs_ctx* c = S.c;
  if (X.M == 0) return GS_OK;
  BHStep b{0, S.N, S.Npad, S.s, S.thr, S.pack(k & 1), S.raw(k & 1), BHForest{}, S.leaf, false,
           S.crit};
  BHTargets x;
  gs_status s;
  {
    KTimer tm(c, GS_K_TREE_BUILD, st);
    s = tracer_order(c->tree, b, X.xraw(c, k & 1), X.M, c->xsort.p, &x, st);
  }
  x.xrec = X.xpk(c, k & 1);
  if (s == GS_OK) {
    KTimer tm(c, GS_K_BH_WALK, st);
    s = bh_walk_targets(c->tree, b, x, st);
  }
  if (s == GS_OK) {
    TracerEpi e{};
    e.x = c->xs.as<double>();
    e.xpk_next = h != 0.0 ? X.xpk(c, (k + 1) & 1) : nullptr;
    e.xraw_next = h != 0.0 ? X.xraw(c, (k + 1) & 1) : nullptr;
    e.v_out = v_out;
    e.center = S.scal(SC_CENTER);
    e.s = S.s;
    e.h = h;
    e.M = X.M;
    KTimer tm(c, GS_K_BH_FWD, st);
    s = bh_eval_targets(c->tree, b, x, e, st);
  }
  if (s != GS_OK) return fail(c, s, "Barnes-Hut tracer step failed: %s", bh_last_error());
  return GS_OK;
}

gs_status tracer_step(const Solver& S, const Tracers& X, int k, double h, double* v_out,
                      cudaStream_t st) {
  gs_ctx* c = S.c;
  if (X.M == 0) return GS_OK;
  TracerEpi e{};
  e.x = c->xs.as<double>();
  e.xpk_next = h != 0.0 ? X.xpk(c, (k + 1) & 1) : nullptr;
  e.v_out = v_out;
  e.center = S.scal(SC_CENTER);
  e.s = S.s;
  e.h = h;
  e.M = X.M;
  KTimer tm(c, GS_K_EXACT_FWD, st);
  CK(launch_tracer(S.pack(k & 1), S.gf, X.xpk(c, k & 1), X.tg, c->xpart.as<float2>(),
                   c->xtickets.as<unsigned>(), e, c->d_status, st),
     "tracer kernel");
  return GS_OK;
}

// Shooting with tracers (capturable): particles as shoot_enqueue without H,
// tracers x0 carried along; final tracer positions left in c->xs.
gs_status flow_enqueue(Solver& S, const Tracers& X, const double* dq0, const double* dp0,
                       const double* dx0, cudaStream_t st) {
  gs_status s;
  gs_ctx* c = S.c;
  S.st = st;
  if ((s = solver_load(S, dq0, dp0, 0))) return s;
  if (X.M > 0) {
    CK(cudaMemcpyAsync(c->xs.p, dx0, (size_t)X.M * 24, cudaMemcpyDeviceToDevice, st), "copy");
    CK(launch_pack_points(c->xs.as<double>(), X.M, S.scal(SC_CENTER), S.s, X.xpk(c, 0),
                          X.tree ? X.xraw(c, 0) : nullptr, st),
       "pack");
  }
  for (int k = 0; k < S.T; k++) {
    FwdEpi e = fwd_epi(S, (k + 1) & 1, S.h);
    if (X.tree) {
      // the particle step builds state k's tree; the tracers walk it after
      if ((s = forward_rhs(S, k & 1, e, nullptr))) return s;
      if ((s = tracer_bh_step(S, X, k, S.h, nullptr, st))) return s;
    } else {
      // both read step k's particle pack; the particle step writes slot k+1
      if ((s = tracer_step(S, X, k, S.h, nullptr, st))) return s;
      if ((s = forward_rhs(S, k & 1, e, nullptr))) return s;
    }
  }
  return GS_OK;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

gs_status gs_create(int device, gs_ctx** out) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return GS_ERR_INVALID_ARG;
  }
  gs_ctx* c = new gs_ctx();
  c->device = device;
  DeviceGuard g(device);
  if (!g.ok) {
    delete c;
    return GS_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess || exact_setup() != cudaSuccess ||
      tree_setup() != cudaSuccess) {
    cudaGetLastError();
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return GS_ERR_CUDA;
  }
  c->tree.d_status = c->d_status;
  *out = c;
  return GS_OK;
}

void gs_destroy(gs_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (DevMem* m : {&c->in_q, &c->in_p, &c->in_a, &c->in_b, &c->in_X, &c->out_a, &c->out_b,
                      &c->q, &c->p, &c->al, &c->be, &c->F0, &c->pf, &c->r2, &c->scal, &c->packs,
                      &c->raws, &c->abpacks, &c->ckpt, &c->part, &c->tickets, &c->bmeta, &c->bout,
                      &c->gd_p, &c->gd_E, &c->in_x, &c->xs, &c->xpks, &c->xpart, &c->xtickets,
                      &c->lb, &c->xraws, &c->xsort, &c->grid, &c->st64, &c->rho})
      m->release();
    for (auto* gc : {&c->g_shoot, &c->g_grad, &c->g_batch, &c->g_flow})
      if (gc->exec) cudaGraphExecDestroy(gc->exec);
    if (c->cap) cudaStreamDestroy(c->cap);
    tree_release(c->tree);
    for (auto& t : c->pending) {
      cudaEventDestroy(t.a);
      cudaEventDestroy(t.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->d_status) cudaFree(c->d_status);
  }
  delete c;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->err.c_str() : "no context"; }

gs_status gs_set_option(gs_ctx* c, const char* name, int64_t value) {
  if (!c || !name) return GS_ERR_INVALID_ARG;
  if (strcmp(name, "bh_list_cap") == 0) {
    if (value < 0 || value > (int64_t(1) << 24))
      return fail(c, GS_ERR_INVALID_ARG, "bh_list_cap must be in [0, 2^24]");
    c->tree.lcap_req = (int)value;
    return GS_OK;
  }
  if (strcmp(name, "bh_walk_split") == 0) {
    if (value != 0 && value != 1 && value != 2 && value != 4)
      return fail(c, GS_ERR_INVALID_ARG, "bh_walk_split must be 0, 1, 2 or 4");
    c->tree.wsplit_req = (int)value;
    return GS_OK;
  }
  if (strcmp(name, "graphs") == 0) {
    if (value != 0 && value != 1) return fail(c, GS_ERR_INVALID_ARG, "graphs must be 0 or 1");
    c->graphs = value != 0;
    return GS_OK;
  }
  if (strcmp(name, "trunc_grid") == 0) {
    if (value != 0 && value != 1) return fail(c, GS_ERR_INVALID_ARG, "trunc_grid must be 0 or 1");
    c->trunc_grid = value != 0;
    return GS_OK;
  }
  const bool xf = strcmp(name, "exact_splits_fwd") == 0, xa = strcmp(name, "exact_splits_adj") == 0;
  if (xf || xa) {
    if (value < 0 || value > kMaxSplits)
      return fail(c, GS_ERR_INVALID_ARG, "%s must be in [0, %d]", name, kMaxSplits);
    (xf ? c->xs_fwd : c->xs_adj) = (int)value;
    return GS_OK;
  }
  return fail(c, GS_ERR_INVALID_ARG, "unknown option '%s'", name);
}

gs_status gs_timing(gs_ctx* c, int enable) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->timing = enable != 0;
  return GS_OK;
}

gs_status gs_timing_read(gs_ctx* c, int64_t* launches, double* ms, int64_t* total_launches) {
  if (!c || !launches || !ms) return GS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  for (int k = 0; k < GS_K_COUNT; k++) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  gs_status rc = GS_OK;
  for (auto& t : c->pending) {
    float v = 0.f;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&v, t.a, t.b) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(c, GS_ERR_CUDA, "timing event failed");
    }
    if (t.cls >= 0 && t.cls < GS_K_COUNT) {
      launches[t.cls] += 1;
      ms[t.cls] += v;
    }
    c->pool.push_back(t.a);
    c->pool.push_back(t.b);
  }
  c->pending.clear();
  const long long now = launches_total();
  if (total_launches) *total_launches = now - c->launch_mark;
  c->launch_mark = now;
  return rc;
}

gs_status gs_sync(gs_ctx* c, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  return read_status(c, (cudaStream_t)stream);
}

gs_status gs_selftest_timeout(gs_ctx* c, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_wait_selftest(c->d_status, 2000000LL, st), "self-test kernel");
  return read_status(c, st);
}

gs_status gs_shoot(gs_ctx* c, const double* q0, const double* p0, int64_t N,
                   const gs_params* prm, double* q1, double* p1, double* H, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false, true))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hq = false, hp = false, hh = false;
  if (q1 && (s = output(c, q1, "q1", &hq))) return s;
  if (p1 && (s = output(c, p1, "p1", &hp))) return s;
  if (H && (s = output(c, H, "H", &hh))) return s;
  const double *dq0, *dp0;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, p0, (size_t)N * 3, "p0", c->in_p, st, &dp0)))
    return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 2, false, st))) return s;
  {
    Key k;
    k.add(N), k.params(prm), k.add(dq0), k.add(dp0), k.add(H != nullptr), k.workspace(c);
    s = run_graphed(c, c->g_shoot, k, st,
                    [&](cudaStream_t s2) { return shoot_enqueue(S, dq0, dp0, H != nullptr, s2); });
    if (s) return s;
  }
  if (H) {
    CK(launch_check_finite(S.scal(SC_H0), 2, c->d_status, st), "check");
    if ((s = copy_out(c, H, S.scal(SC_H0), 2 * sizeof(double), st))) return s;
  }
  size_t b = (size_t)N * 3 * sizeof(double);
  if (q1) {
    CK(launch_check_finite(c->q.as<double>(), N * 3, c->d_status, st), "check");
    if ((s = copy_out(c, q1, c->q.p, b, st))) return s;
  }
  if (p1) {
    CK(launch_check_finite(c->p.as<double>(), N * 3, c->d_status, st), "check");
    if ((s = copy_out(c, p1, c->p.p, b, st))) return s;
  }
  if (hq || hp || hh) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_shoot_grad(gs_ctx* c, const double* q0, const double* p0, const double* X,
                        int64_t N, const gs_params* prm, double* E, double* grad, double* q1,
                        void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, true, true))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hE = false, hg = false, hq = false;
  if ((s = output(c, E, "E", &hE)) || (s = output(c, grad, "grad", &hg))) return s;
  if (q1 && (s = output(c, q1, "q1", &hq))) return s;
  const double *dq0, *dp0, *dX;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, p0, (size_t)N * 3, "p0", c->in_p, st, &dp0)) ||
      (s = input(c, X, (size_t)N * 3, "X", c->in_X, st, &dX)))
    return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  CK(c->out_a.ensure(b3), "workspace");
  CK(c->out_b.ensure(b3), "workspace");
  CK(c->scal.ensure(SC_N * 8), "workspace");
  double* dE = c->scal.as<double>() + SC_E;
  GradRun R;
  if ((s = grad_setup(c, N, prm, nullptr, st, R))) return s;
  double* dgrad = c->out_a.as<double>();
  double* dq1 = q1 ? c->out_b.as<double>() : nullptr;
  Key k;
  k.add(N), k.params(prm), k.add(dq0), k.add(dp0), k.add(dX), k.add(dq1), k.workspace(c);
  s = run_graphed(c, c->g_grad, k, st, [&](cudaStream_t s2) {
    return grad_enqueue(R, dq0, dp0, dX, dE, dgrad, dq1, s2);
  });
  if (s) return s;
  CK(launch_check_finite(dE, 3, c->d_status, st), "check");
  CK(launch_check_finite(c->out_a.as<double>(), N * 3, c->d_status, st), "check");
  if ((s = copy_out(c, E, dE, 3 * sizeof(double), st))) return s;
  if ((s = copy_out(c, grad, c->out_a.p, b3, st))) return s;
  if (q1 && (s = copy_out(c, q1, c->out_b.p, b3, st))) return s;
  if (hE || hg || hq) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_shoot_batched(gs_ctx* c, int32_t S, const int64_t* offsets, const double* q0,
                           const double* p0, const double* X, const gs_params* prm, double* E,
                           double* grad, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_params(c, prm, true))) return s;
  Batch b;
  if ((s = batch_plan(c, S, offsets, prm->mode == GS_EXACT, b))) return s;
  const int64_t N = b.N;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hE = false, hg = false;
  if ((s = output(c, E, "E", &hE)) || (s = output(c, grad, "grad", &hg))) return s;
  const double *dq0, *dp0, *dX;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, p0, (size_t)N * 3, "p0", c->in_p, st, &dp0)) ||
      (s = input(c, X, (size_t)N * 3, "X", c->in_X, st, &dX)))
    return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  // per-launch queue heads: forward steps, checkpoint recomputation, adjoint
  const int T = prm->T;
  if ((s = batch_upload(c, b, prm->mode == GS_EXACT ? 3 * T + 2 : 0, st))) return s;
  CK(c->bout.ensure(b3), "workspace");
  double* dgrad = c->bout.as<double>();
  // exact: persistent launches over (subject, tile) items; Barnes-Hut: one
  // forest of all subjects per step
  if ((s = batched_grad(c, b, dq0, dp0, dX, prm, dgrad, st))) return s;
  CK(launch_check_finite(b.E, 3 * (int64_t)S, c->d_status, st), "check");
  CK(launch_check_finite(dgrad, N * 3, c->d_status, st), "check");
  if ((s = copy_out(c, E, b.E, 3 * (size_t)S * sizeof(double), st))) return s;
  if ((s = copy_out(c, grad, dgrad, b3, st))) return s;
  if (hE || hg) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_descend_batched(gs_ctx* c, int32_t S, const int64_t* offsets, const double* q0,
                             double* p0, const double* X, const gs_params* prm, double step,
                             int32_t iters, double* E_hist, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_params(c, prm, true))) return s;
  if (!std::isfinite(step)) return fail(c, GS_ERR_INVALID_ARG, "step must be finite");
  if (iters < 0 || iters > 1000000)
    return fail(c, GS_ERR_INVALID_ARG, "iters must be in [0, 1e6] (got %d)", iters);
  Batch b;
  if ((s = batch_plan(c, S, offsets, prm->mode == GS_EXACT, b))) return s;
  const int64_t N = b.N;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hp = false, hE = false;
  if ((s = output(c, p0, "p0", &hp))) return s;
  if (E_hist && (s = output(c, E_hist, "E_hist", &hE))) return s;
  const double *dq0, *dX;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, X, (size_t)N * 3, "X", c->in_X, st, &dX)))
    return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double), eb = 3 * (size_t)S * sizeof(double);
  CK(c->gd_p.ensure(b3), "workspace");
  CK(c->gd_E.ensure(std::max<size_t>(eb * (size_t)iters, 8)), "workspace");
  CK(c->bout.ensure(b3), "workspace");
  CK(cudaMemcpyAsync(c->gd_p.p, p0, b3, cudaMemcpyDefault, st), "p0 copy");
  if ((s = batch_upload(c, b, prm->mode == GS_EXACT ? 3 * prm->T + 2 : 0, st))) return s;
  double* dp = c->gd_p.as<double>();
  double* dgrad = c->bout.as<double>();
  for (int it = 0; it < iters; it++) {
    if ((s = batched_grad(c, b, dq0, dp, dX, prm, dgrad, st))) return s;
    CK(cudaMemcpyAsync(c->gd_E.as<char>() + eb * it, b.E, eb, cudaMemcpyDeviceToDevice, st),
       "energy copy");
    CK(launch_axpy(dp, dgrad, -step, N * 3, st), "update");
  }
  if (iters > 0) CK(launch_check_finite(c->gd_E.as<double>(), 3 * (int64_t)S * iters, c->d_status, st), "check");
  CK(launch_check_finite(dp, N * 3, c->d_status, st), "check");
  if ((s = copy_out(c, p0, dp, b3, st))) return s;
  if (E_hist && iters > 0 && (s = copy_out(c, E_hist, c->gd_E.p, eb * iters, st))) return s;
  if (hp || hE) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_flow(gs_ctx* c, const double* q0, const double* p0, int64_t N, const double* x0,
                  int64_t M, const gs_params* prm, double* q1, double* p1, double* x1,
                  void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  if (M < 0 || M > (int64_t(1) << 30))
    return fail(c, GS_ERR_INVALID_ARG, "M must be in [0, 2^30] (got %lld)", (long long)M);
  if (prm->mode == GS_TRUNC)
    return fail(c, GS_ERR_UNSUPPORTED, "tracer points: GS_EXACT or GS_BH");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hq = false, hp = false, hx = false;
  if (q1 && (s = output(c, q1, "q1", &hq))) return s;
  if (p1 && (s = output(c, p1, "p1", &hp))) return s;
  if (M > 0 && (s = output(c, x1, "x1", &hx))) return s;
  const double *dq0, *dp0, *dx0 = nullptr;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, p0, (size_t)N * 3, "p0", c->in_p, st, &dp0)))
    return s;
  if (M > 0 && (s = input(c, x0, (size_t)M * 3, "x0", c->in_x, st, &dx0))) return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 2, false, st))) return s;
  Tracers X;
  if ((s = tracer_setup(c, S, M, st, X))) return s;
  {
    Key k;
    k.add(N), k.add(M), k.params(prm), k.add(dq0), k.add(dp0), k.add(dx0), k.workspace(c);
    s = run_graphed(c, c->g_flow, k, st,
                    [&](cudaStream_t s2) { return flow_enqueue(S, X, dq0, dp0, dx0, s2); });
    if (s) return s;
  }
  const size_t b = (size_t)N * 3 * sizeof(double);
  if (q1) {
    CK(launch_check_finite(c->q.as<double>(), N * 3, c->d_status, st), "check");
    if ((s = copy_out(c, q1, c->q.p, b, st))) return s;
  }
  if (p1) {
    CK(launch_check_finite(c->p.as<double>(), N * 3, c->d_status, st), "check");
    if ((s = copy_out(c, p1, c->p.p, b, st))) return s;
  }
  if (M > 0) {
    CK(launch_check_finite(c->xs.as<double>(), M * 3, c->d_status, st), "check");
    if ((s = copy_out(c, x1, c->xs.p, (size_t)M * 24, st))) return s;
  }
  if (hq || hp || hx) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_velocity(gs_ctx* c, const double* q, const double* p, int64_t N, const double* x,
                      int64_t M, const gs_params* prm, double* v, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  if (prm->mode == GS_TRUNC)
    return fail(c, GS_ERR_UNSUPPORTED, "velocity field: GS_EXACT or GS_BH");
  if (M < 1 || M > (int64_t(1) << 30))
    return fail(c, GS_ERR_INVALID_ARG, "M must be in [1, 2^30] (got %lld)", (long long)M);
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hv = false;
  if ((s = output(c, v, "v", &hv))) return s;
  const double *dq, *dp, *dx;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)) ||
      (s = input(c, x, (size_t)M * 3, "x", c->in_x, st, &dx)))
    return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 1, false, st))) return s;
  if ((s = solver_load(S, dq, dp, 0))) return s;
  Tracers X;
  if ((s = tracer_setup(c, S, M, st, X))) return s;
  CK(c->out_a.ensure((size_t)M * 24), "workspace");
  CK(cudaMemcpyAsync(c->xs.p, dx, (size_t)M * 24, cudaMemcpyDeviceToDevice, st), "copy");
  CK(launch_pack_points(c->xs.as<double>(), M, S.scal(SC_CENTER), S.s, X.xpk(c, 0),
                        X.tree ? X.xraw(c, 0) : nullptr, st),
     "pack");
  if (X.tree) {
    // the particles' tree of (q, p), then the tracers walk it
    BHStep b{0, S.N, S.Npad, S.s, S.thr, S.pack(0), S.raw(0), BHForest{}, S.leaf, false, S.crit};
    {
      KTimer tm(c, GS_K_TREE_BUILD, st);
      if ((s = bh_build(c->tree, b, nullptr, false, st)))
        return fail(c, s, "Barnes-Hut build failed: %s", bh_last_error());
    }
    if ((s = tracer_bh_step(S, X, 0, 0.0, c->out_a.as<double>(), st))) return s;
  } else if ((s = tracer_step(S, X, 0, 0.0, c->out_a.as<double>(), st))) {
    return s;
  }
  if ((s = copy_out(c, v, c->out_a.p, (size_t)M * 24, st))) return s;
  if (hv) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_lbfgs(gs_ctx* c, const double* q0, double* p0, const double* X, int64_t N,
                   const gs_params* prm, int32_t m, int32_t iters, double gtol, double* E_hist,
                   int32_t* n_done, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, true))) return s;
  if (m < 1 || m > 64) return fail(c, GS_ERR_INVALID_ARG, "m must be in [1, 64] (got %d)", m);
  if (iters < 0 || iters > 100000)
    return fail(c, GS_ERR_INVALID_ARG, "iters must be in [0, 1e5] (got %d)", iters);
  if (!(gtol >= 0.0) || !std::isfinite(gtol))
    return fail(c, GS_ERR_INVALID_ARG, "gtol must be finite and >= 0");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hp = false, hE = false;
  if ((s = output(c, p0, "p0", &hp))) return s;
  if (E_hist && (s = output(c, E_hist, "E_hist", &hE))) return s;
  const double *dq0, *dX;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, X, (size_t)N * 3, "X", c->in_X, st, &dX)))
    return s;
  const int64_t n3 = N * 3;
  const size_t b3 = (size_t)n3 * sizeof(double);
  // iterate x, gradient g, direction d, trial point xt and its gradient gt,
  // the m most recent pairs s = x_{k+1} - x_k, y = g_{k+1} - g_k, a scalar
  CK(c->lb.ensure((size_t)(5 + 2 * m) * b3 + 64), "workspace");
  double* x = c->lb.as<double>();
  double *gv = x + n3, *d = gv + n3, *xt = d + n3, *gt = xt + n3, *Sv = gt + n3,
         *Yv = Sv + (size_t)m * n3, *sc = Yv + (size_t)m * n3;
  CK(c->scal.ensure(SC_N * 8), "workspace");
  double* dE = c->scal.as<double>() + SC_E;
  CK(cudaMemcpyAsync(x, p0, b3, cudaMemcpyDefault, st), "p0 copy");
  GradRun R;
  if ((s = grad_setup(c, N, prm, nullptr, st, R))) return s;

  // E and gradient at xt (into gt): the gradient graph, replayed
  auto evaluate = [&](double* E) -> gs_status {
    Key k;
    k.add(N), k.params(prm), k.add(dq0), k.add((const double*)xt), k.add(dX), k.add(gt);
    k.workspace(c);
    gs_status r = run_graphed(c, c->g_grad, k, st, [&](cudaStream_t s2) {
      return grad_enqueue(R, dq0, xt, dX, dE, gt, nullptr, s2);
    });
    if (r) return r;
    CK(cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, st), "energy read");
    CK(cudaStreamSynchronize(st), "stream synchronize");
    return GS_OK;
  };
  auto dot = [&](const double* a, const double* b, double* out) -> gs_status {
    CK(launch_dot(a, b, n3, sc, st), "dot");
    CK(cudaMemcpyAsync(out, sc, sizeof(double), cudaMemcpyDeviceToHost, st), "dot read");
    CK(cudaStreamSynchronize(st), "stream synchronize");
    return GS_OK;
  };
  auto copy = [&](double* dst, const double* src) -> gs_status {
    CK(cudaMemcpyAsync(dst, src, b3, cudaMemcpyDeviceToDevice, st), "copy");
    return GS_OK;
  };
#define LB(call)          \
  do {                    \
    if ((s = (call))) return s; \
  } while (0)
  double E = 0.0, gg = 0.0;
  LB(copy(xt, x));
  LB(evaluate(&E));
  LB(copy(gv, gt));
  LB(dot(gv, gv, &gg));
  std::vector<double> Eh{E}, rho(m), alpha(m);
  const double g0 = std::sqrt(gg);
  int stored = 0, head = 0, it = 0;
  for (; it < iters; it++) {
    if (!(std::sqrt(gg) > gtol * std::max(1.0, g0))) break;
    // two-loop recursion: d = -H g with H from the stored pairs
    LB(copy(d, gv));
    for (int j = 0; j < stored; j++) {  // newest to oldest
      const int i = (head - 1 - j + m) % m;
      double sq = 0.0;
      LB(dot(Sv + (size_t)i * n3, d, &sq));
      alpha[i] = rho[i] * sq;
      CK(launch_axpy(d, Yv + (size_t)i * n3, -alpha[i], n3, st), "axpy");
    }
    double gamma = 1.0 / std::max(std::sqrt(gg), 1e-300);
    if (stored > 0) {
      const int i = (head - 1 + m) % m;
      double yy = 0.0;
      LB(dot(Yv + (size_t)i * n3, Yv + (size_t)i * n3, &yy));
      gamma = 1.0 / (rho[i] * yy);  // s.y / y.y
    }
    CK(launch_scale(d, d, gamma, n3, st), "scale");
    for (int j = stored - 1; j >= 0; j--) {  // oldest to newest
      const int i = (head - 1 - j + m) % m;
      double yr = 0.0;
      LB(dot(Yv + (size_t)i * n3, d, &yr));
      CK(launch_axpy(d, Sv + (size_t)i * n3, alpha[i] - rho[i] * yr, n3, st), "axpy");
    }
    CK(launch_scale(d, d, -1.0, n3, st), "scale");
    double gd = 0.0;
    LB(dot(gv, d, &gd));
    if (!(gd < 0.0)) {  // not a descent direction: restart from -g / |g|
      stored = 0;
      CK(launch_scale(d, gv, -1.0 / std::sqrt(gg), n3, st), "scale");
      gd = -std::sqrt(gg);
    }
    // backtracking line search (Armijo, c1 = 1e-4), unit step first
    double t = 1.0, Et = 0.0;
    bool ok = false;
    for (int ls = 0; ls < 50; ls++) {
      LB(copy(xt, x));
      CK(launch_axpy(xt, d, t, n3, st), "axpy");
      LB(evaluate(&Et));
      if (std::isfinite(Et) && Et <= E + 1e-4 * t * gd) {
        ok = true;
        break;
      }
      t *= 0.5;
    }
    if (!ok) break;
    // new pair s = t d, y = gt - g
    double* Si = Sv + (size_t)head * n3;
    double* Yi = Yv + (size_t)head * n3;
    CK(launch_scale(Si, d, t, n3, st), "scale");
    LB(copy(Yi, gt));
    CK(launch_axpy(Yi, gv, -1.0, n3, st), "axpy");
    double sy = 0.0, ss = 0.0, yy = 0.0;
    LB(dot(Si, Yi, &sy));
    LB(dot(Si, Si, &ss));
    LB(dot(Yi, Yi, &yy));
    LB(copy(x, xt));
    LB(copy(gv, gt));
    E = Et;
    Eh.push_back(E);
    LB(dot(gv, gv, &gg));
    if (sy > 1e-12 * std::sqrt(ss * yy)) {  // curvature condition: keep the pair
      rho[head] = 1.0 / sy;
      head = (head + 1) % m;
      stored = std::min(stored + 1, m);
    }
  }
#undef LB
  if (n_done) *n_done = it;
  CK(launch_check_finite(x, n3, c->d_status, st), "check");
  if ((s = copy_out(c, p0, x, b3, st))) return s;
  if (E_hist) {
    std::vector<double> out((size_t)iters + 1, std::nan(""));
    std::copy(Eh.begin(), Eh.end(), out.begin());
    CK(cudaMemcpyAsync(E_hist, out.data(), out.size() * sizeof(double), cudaMemcpyDefault, st),
       "E_hist copy");
    CK(cudaStreamSynchronize(st), "stream synchronize");  // `out` is freed on return
  }
  return read_status(c, st);
}

gs_status gs_autotune(gs_ctx* c, const double* q, const double* p, int64_t N,
                      const gs_params* prm, const int32_t* cand, int32_t n_cand, int32_t* best,
                      double* ms, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  if (prm->mode == GS_EXACT)
    return fail(c, GS_ERR_INVALID_ARG, "gs_autotune tunes the tree modes (GS_BH, GS_TRUNC)");
  static const int32_t kDefault[] = {1, 2, 4, 8, 16, 32};
  if (!cand) {
    cand = kDefault;
    n_cand = 6;
  }
  if (n_cand < 1 || n_cand > 32) return fail(c, GS_ERR_INVALID_ARG, "n_cand must be in [1, 32]");
  for (int k = 0; k < n_cand; k++)
    if (cand[k] < 1 || cand[k] > 32)
      return fail(c, GS_ERR_INVALID_ARG, "candidate leaf sizes must be in [1, 32]");
  if (!best) return fail(c, GS_ERR_INVALID_ARG, "best is NULL");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const double *dq, *dp;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)))
    return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, GS_ERR_CUDA, "event create failed");
  }
  double best_ms = 0.0;
  int32_t best_l = cand[0];
  gs_status rc = GS_OK;
  const bool was_timing = c->timing;
  c->timing = false;
  for (int k = 0; k < n_cand && rc == GS_OK; k++) {
    gs_params pk = *prm;
    pk.leaf_size = cand[k];
    Solver S;
    if ((rc = solver_init(c, S, N, &pk, 1, true, st))) break;
    if ((rc = solver_load(S, dq, dp, 0))) break;
    // one forward and one adjoint right-hand side on (q, p), adjoint
    // variables zero (their values do not change the work)
    if (cudaMemsetAsync(c->al.p, 0, (size_t)N * 24, st) != cudaSuccess ||
        cudaMemsetAsync(c->be.p, 0, (size_t)N * 24, st) != cudaSuccess ||
        launch_pack_ab(c->al.as<double>(), c->be.as<double>(), N, adj_beta_scale(S.s),
                       S.abpack(0), st) !=
            cudaSuccess) {
      rc = cuda_fail(c, cudaGetLastError(), "autotune setup");
      break;
    }
    float best_k = 0.f;
    for (int rep = 0; rep < 4 && rc == GS_OK; rep++) {  // first run is a warm-up
      cudaEventRecord(e0, st);
      if ((rc = forward_rhs(S, 0, fwd_epi(S, -1, 0.0), nullptr, 0))) break;
      if ((rc = adjoint_rhs(S, 0, 0, adj_epi(S, -1, 0.0, false, nullptr), nullptr, 0, true)))
        break;
      cudaEventRecord(e1, st);
      float t = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        rc = cuda_fail(c, cudaGetLastError(), "autotune timing");
        break;
      }
      if (rep == 1 || (rep > 1 && t < best_k)) best_k = t;
    }
    if (rc != GS_OK) break;
    if (ms) ms[k] = best_k;
    if (k == 0 || best_k < best_ms) {
      best_ms = best_k;
      best_l = cand[k];
    }
  }
  c->timing = was_timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GS_OK) return rc;
  *best = best_l;
  return read_status(c, st);
}

gs_status gs_autotune_exact(gs_ctx* c, const double* q, const double* p, int64_t N,
                            const gs_params* prm, const int32_t* cand, int32_t n_cand,
                            int32_t* best, double* ms, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  if (prm->mode != GS_EXACT)
    return fail(c, GS_ERR_INVALID_ARG, "gs_autotune_exact tunes the exact mode (GS_EXACT)");
  static const int32_t kDefault[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  if (!cand) {
    cand = kDefault;
    n_cand = 10;
  }
  if (n_cand < 1 || n_cand > 64) return fail(c, GS_ERR_INVALID_ARG, "n_cand must be in [1, 64]");
  for (int k = 0; k < n_cand; k++)
    if (cand[k] < 1 || cand[k] > kMaxSplits)
      return fail(c, GS_ERR_INVALID_ARG, "candidate splits must be in [1, %d]", kMaxSplits);
  if (!best) return fail(c, GS_ERR_INVALID_ARG, "best is NULL");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const double *dq, *dp;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)))
    return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, GS_ERR_CUDA, "event create failed");
  }
  // best of three launches after a warm-up
  auto time_best = [&](auto&& enqueue, float* out) -> gs_status {
    float bt = 0.f;
    for (int rep = 0; rep < 4; rep++) {
      cudaEventRecord(e0, st);
      if (gs_status r = enqueue()) return r;
      cudaEventRecord(e1, st);
      float t = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "autotune timing");
      if (rep == 1 || (rep > 1 && t < bt)) bt = t;
    }
    *out = bt;
    return GS_OK;
  };
  const int keep_f = c->xs_fwd, keep_a = c->xs_adj;
  const bool was_timing = c->timing;
  c->timing = false;
  float bf = 0.f, ba = 0.f;
  int32_t jf = 1, ja = 1;
  gs_status rc = GS_OK;
  for (int k = 0; k < n_cand && rc == GS_OK; k++) {
    c->xs_fwd = c->xs_adj = cand[k];
    Solver S;
    if ((rc = solver_init(c, S, N, prm, 1, true, st))) break;
    if ((rc = solver_load(S, dq, dp, 0))) break;
    // adjoint variables zero (their values do not change the work)
    if (cudaMemsetAsync(c->al.p, 0, (size_t)N * 24, st) != cudaSuccess ||
        cudaMemsetAsync(c->be.p, 0, (size_t)N * 24, st) != cudaSuccess ||
        launch_pack_ab(c->al.as<double>(), c->be.as<double>(), N, adj_beta_scale(S.s),
                       S.abpack(0), st) != cudaSuccess) {
      rc = cuda_fail(c, cudaGetLastError(), "autotune setup");
      break;
    }
    float tf = 0.f, ta = 0.f;
    if ((rc = time_best([&] { return forward_rhs(S, 0, fwd_epi(S, -1, 0.0), nullptr, 0); }, &tf)))
      break;
    if ((rc = time_best(
             [&] {
               return adjoint_rhs(S, 0, 0, adj_epi(S, -1, 0.0, false, nullptr), nullptr, 0, true);
             },
             &ta)))
      break;
    if (ms) ms[2 * k] = tf, ms[2 * k + 1] = ta;
    if (k == 0 || tf < bf) bf = tf, jf = S.gf.J;
    if (k == 0 || ta < ba) ba = ta, ja = S.ga.J;
  }
  c->xs_fwd = keep_f, c->xs_adj = keep_a;
  c->timing = was_timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GS_OK) return rc;
  best[0] = jf, best[1] = ja;
  return read_status(c, st);
}

gs_status gs_rhs(gs_ctx* c, const double* q, const double* p, int64_t N, const gs_params* prm,
                 double* F, double* Phi, int64_t* counts, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hF = false, hP = false;
  if ((s = output(c, F, "F", &hF)) || (s = output(c, Phi, "Phi", &hP))) return s;
  const double *dq, *dp;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)))
    return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 1, false, st))) return s;
  if ((s = solver_load(S, dq, dp, 0))) return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  CK(c->out_a.ensure(b3), "workspace");
  CK(c->out_b.ensure(b3), "workspace");
  FwdEpi e = fwd_epi(S, -1, 0.0);
  e.F_out = c->out_a.as<double>();
  e.Phi_out = c->out_b.as<double>();
  int64_t cnt[2] = {0, 0};
  // (no counts asked for: the lean walk, which lists the same entries)
  if ((s = forward_rhs(S, 0, e, counts ? cnt : nullptr))) return s;
  if ((s = copy_out(c, F, c->out_a.p, b3, st)) || (s = copy_out(c, Phi, c->out_b.p, b3, st)))
    return s;
  if (counts) {
    CK(cudaStreamSynchronize(st), "stream synchronize");
    if (S.mode != GS_EXACT) bh_counts(c->tree, cnt);
    counts[0] = cnt[0];
    counts[1] = cnt[1];
  }
  if (hF || hP || counts) return read_status(c, st);
  return GS_OK;
}

gs_status gs_adj_rhs(gs_ctx* c, const double* q, const double* p, const double* al,
                     const double* be, int64_t N, const gs_params* prm, double* dA, double* dB,
                     int64_t* counts, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hA = false, hB = false;
  if ((s = output(c, dA, "dA", &hA)) || (s = output(c, dB, "dB", &hB))) return s;
  const double *dq, *dp, *da, *db;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)) ||
      (s = input(c, al, (size_t)N * 3, "al", c->in_a, st, &da)) ||
      (s = input(c, be, (size_t)N * 3, "be", c->in_b, st, &db)))
    return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 1, true, st))) return s;
  if ((s = solver_load(S, dq, dp, 0))) return s;
  const size_t b3 = (size_t)N * 3 * sizeof(double);
  CK(cudaMemcpyAsync(c->al.p, da, b3, cudaMemcpyDeviceToDevice, st), "copy");
  CK(cudaMemcpyAsync(c->be.p, db, b3, cudaMemcpyDeviceToDevice, st), "copy");
  // adjoint pack: alpha and the scaled beta as FP32
  CK(launch_pack_ab(c->al.as<double>(), c->be.as<double>(), N, adj_beta_scale(S.s),
                    S.abpack(0), st),
     "pack");
  CK(c->out_a.ensure(b3), "workspace");
  CK(c->out_b.ensure(b3), "workspace");
  AdjEpi e = adj_epi(S, -1, 0.0, false, nullptr);
  e.dA_out = c->out_a.as<double>();
  e.dB_out = c->out_b.as<double>();
  int64_t cnt[2] = {0, 0};
  if ((s = adjoint_rhs(S, 0, 0, e, counts ? cnt : nullptr))) return s;
  if ((s = copy_out(c, dA, c->out_a.p, b3, st)) || (s = copy_out(c, dB, c->out_b.p, b3, st)))
    return s;
  if (counts) {
    CK(cudaStreamSynchronize(st), "stream synchronize");
    if (S.mode != GS_EXACT) bh_counts(c->tree, cnt);
    counts[0] = cnt[0];
    counts[1] = cnt[1];
  }
  if (hA || hB || counts) return read_status(c, st);
  return GS_OK;
}

gs_status gs_tree(gs_ctx* c, const double* q, int64_t N, uint32_t* codes, int32_t* order,
                  int32_t* nodes, float* range, int64_t cap, int64_t* n_nodes, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N))) return s;
  if (cap < 0) return fail(c, GS_ERR_INVALID_ARG, "cap must be >= 0");
  bool h;
  if (codes && (s = output(c, codes, "codes", &h))) return s;
  if (order && (s = output(c, order, "order", &h))) return s;
  if (nodes && (s = output(c, nodes, "nodes", &h))) return s;
  if (range && (s = output(c, range, "range", &h))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const double* dq;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq))) return s;
  gs_params prm{1.0, 0.0, 3.0, 1, GS_BH, 0, 0, 0, 0, 0, 0};
  Solver S;
  if ((s = solver_init(c, S, N, &prm, 1, false, st))) return s;
  if ((s = solver_load(S, dq, dq, 0))) return s;
  s = tree_export(c->tree, S.raw(0), S.pack(0), N, codes, order, nodes, range, cap, n_nodes, st);
  if (s != GS_OK) return fail(c, s, "tree export failed: %s", bh_last_error());
  return read_status(c, st);
}

gs_status gs_shoot_traj(gs_ctx* c, const double* q0, const double* p0, int64_t N,
                        const gs_params* prm, double* qtraj, double* ptraj, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false, true))) return s;
  if (!qtraj && !ptraj) return fail(c, GS_ERR_INVALID_ARG, "qtraj and ptraj are both NULL");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool hq = false, hp = false;
  if (qtraj && (s = output(c, qtraj, "qtraj", &hq))) return s;
  if (ptraj && (s = output(c, ptraj, "ptraj", &hp))) return s;
  const double *dq0, *dp0;
  if ((s = input(c, q0, (size_t)N * 3, "q0", c->in_q, st, &dq0)) ||
      (s = input(c, p0, (size_t)N * 3, "p0", c->in_p, st, &dp0)))
    return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 2, false, st))) return s;
  if ((s = shoot_enqueue(S, dq0, dp0, false, st, qtraj, ptraj))) return s;
  CK(launch_check_finite(c->q.as<double>(), N * 3, c->d_status, st), "check");
  CK(launch_check_finite(c->p.as<double>(), N * 3, c->d_status, st), "check");
  if (hq || hp) return read_status(c, st);
  CK(cudaGetLastError(), "launch");
  return GS_OK;
}

gs_status gs_bh_tally(gs_ctx* c, const double* q, int64_t N, const gs_params* prm,
                      int64_t* tally, int64_t* stats, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N)) || (s = check_params(c, prm, false))) return s;
  if (prm->mode != GS_BH) return fail(c, GS_ERR_UNSUPPORTED, "gs_bh_tally needs mode GS_BH");
  if (!tally) return fail(c, GS_ERR_INVALID_ARG, "tally is NULL");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool ht = false, hs = false;
  if ((s = output(c, tally, "tally", &ht))) return s;
  if (stats && (s = output(c, stats, "stats", &hs))) return s;
  const double* dq;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq))) return s;
  Solver S;
  if ((s = solver_init(c, S, N, prm, 1, false, st))) return s;
  if ((s = solver_load(S, dq, dq, 0))) return s;  // decisions depend on positions only
  const size_t bytes = (size_t)N * 5 * sizeof(int64_t);
  CK(c->out_a.ensure(bytes + 2 * sizeof(int64_t)), "workspace");
  int64_t* dstats = c->out_a.as<int64_t>() + (size_t)N * 5;
  BHStep b{0, S.N, S.Npad, S.s, S.thr, S.pack(0), S.raw(0), BHForest{}, S.leaf, false, S.crit};
  s = bh_build(c->tree, b, nullptr, false, st);
  if (s == GS_OK) s = bh_tally(c->tree, b, c->out_a.as<int64_t>(), stats ? dstats : nullptr, st);
  if (s != GS_OK) return fail(c, s, "decision tally failed: %s", bh_last_error());
  if ((s = copy_out(c, tally, c->out_a.p, bytes, st))) return s;
  if (stats && (s = copy_out(c, stats, dstats, 2 * sizeof(int64_t), st))) return s;
  if (ht || hs) return read_status(c, st);
  return GS_OK;
}

gs_status gs_tree_sums(gs_ctx* c, const double* q, const double* p, const double* al,
                       const double* be, int64_t N, double* sums, int64_t cap,
                       int64_t* n_nodes, void* stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->err.clear();
  gs_status s;
  if ((s = check_n(c, N))) return s;
  if (cap < 0) return fail(c, GS_ERR_INVALID_ARG, "cap must be >= 0");
  if ((al == nullptr) != (be == nullptr))
    return fail(c, GS_ERR_INVALID_ARG, "al and be must both be given or both be NULL");
  bool h;
  if (sums && (s = output(c, sums, "sums", &h))) return s;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const bool adj = al != nullptr;
  const double *dq, *dp, *da = nullptr, *db = nullptr;
  if ((s = input(c, q, (size_t)N * 3, "q", c->in_q, st, &dq)) ||
      (s = input(c, p, (size_t)N * 3, "p", c->in_p, st, &dp)))
    return s;
  if (adj && ((s = input(c, al, (size_t)N * 3, "al", c->in_a, st, &da)) ||
              (s = input(c, be, (size_t)N * 3, "be", c->in_b, st, &db))))
    return s;
  gs_params prm{1.0, 0.0, 3.0, 1, GS_BH, 0, 0, 0, 0, 0, 0};
  Solver S;
  if ((s = solver_init(c, S, N, &prm, 1, adj, st))) return s;
  if ((s = solver_load(S, dq, dp, 0))) return s;
  const double mu = adj_beta_scale(S.s);
  if (adj) {
    const size_t b3 = (size_t)N * 3 * sizeof(double);
    CK(cudaMemcpyAsync(c->al.p, da, b3, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->be.p, db, b3, cudaMemcpyDeviceToDevice, st), "copy");
    CK(launch_pack_ab(c->al.as<double>(), c->be.as<double>(), N, mu, S.abpack(0), st), "pack");
  }
  s = tree_sums(c->tree, S.raw(0), S.pack(0), adj ? S.abpack(0) : nullptr, N, S.scal(SC_CENTER),
                S.s, mu, sums, cap, n_nodes, st);
  if (s != GS_OK) return fail(c, s, "tree sums export failed: %s", bh_last_error());
  return read_status(c, st);
}

}  // extern "C"
