// common.cuh -- device helpers shared by the libgs kernels (sm_103a).
//
// Packed FP32 pairs: the pair kernels process two source points per
// instruction with the Blackwell f32x2 arithmetic (add/sub/mul/fma .f32x2),
// a 64-bit register holding {low = even source, high = odd source}.
// exp(-r^2 / (2 sigma^2)) is evaluated as ex2(-|d_s|^2) on the MUFU unit,
// with positions pre-scaled by s = sqrt(log2(e) / (2 sigma^2)) so that the
// exponent's constant folds into the coordinates (exp(x) = 2^(x log2 e)).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

// ---------------------------------------------------------------- status bits
enum : int {
  ST_NONFINITE = 1,  // a result was NaN/Inf
  ST_TIMEOUT = 2,    // a bounded wait (mbarrier / queue) gave up
};

// ---------------------------------------------------------------- f32x2 ops
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_make(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2 f2_dup(float v) { return f2_make(v, v); }
__device__ __forceinline__ void f2_split(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float f2_sum(f2 v) {
  float a, b;
  f2_split(v, a, b);
  return a + b;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// 2^(-x) on the MUFU ex2 unit (x >= 0 here; large x flushes to 0).
__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}
// Gaussian weights of a packed pair of squared scaled distances.
__device__ __forceinline__ f2 gauss2(f2 r2) {
  float a, b;
  f2_split(r2, a, b);
  return f2_make(ex2_neg(a), ex2_neg(b));
}

// Compensated (Kahan) accumulation of FP32 tile partials.
struct Kahan {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float t) {
    float y = t - c;
    float u = s + y;
    c = (u - s) - y;
    s = u;
  }
  __device__ __forceinline__ float2 out() const { return make_float2(s, -c); }
};

// ---------------------------------------------------------------- smem / TMA
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (non-multicast), completing on `bar`.
// src and dst 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~`limit_cycles` SM clocks, records ST_TIMEOUT
// and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* status,
                                                  long long limit_cycles = 4000000000LL) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit_cycles) {
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Subject of row i in a set of subjects with offsets off[0..S]: the last s
// with off[s] <= i.
__device__ __forceinline__ int subject_of(const int64_t* off, int S, int64_t i) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- packing
// Pair layout of the per-step source arrays ("packs"): point pair m = j/2
// occupies 3 float4 = {x0,x1,y0,y1}, {z0,z1,u0,u1}, {v0,v1,w0,w1}, where
// (x,y,z) are the scaled recentred coordinates and (u,v,w) the momentum
// (or, in the adjoint pack, (x,y,z) = alpha and (u,v,w) = beta).
struct PackScale {
  double cx, cy, cz;  // recentring point
  double s;           // sqrt(log2(e) / (2 sigma^2))
};

__device__ __forceinline__ void pack_write(float4* pk, int64_t i, float a0, float a1, float a2,
                                           float b0, float b1, float b2) {
  float* b = reinterpret_cast<float*>(pk + (i >> 1) * 3);
  int o = (int)(i & 1);
  b[0 + o] = a0;
  b[2 + o] = a1;
  b[4 + o] = a2;
  b[6 + o] = b0;
  b[8 + o] = b1;
  b[10 + o] = b2;
}
__device__ __forceinline__ void pack_read(const float4* pk, int64_t i, float* a, float* b) {
  const float* f = reinterpret_cast<const float*>(pk + (i >> 1) * 3);
  int o = (int)(i & 1);
  a[0] = f[0 + o];
  a[1] = f[2 + o];
  a[2] = f[4 + o];
  b[0] = f[6 + o];
  b[1] = f[8 + o];
  b[2] = f[10 + o];
}
__device__ __forceinline__ void pack_state(float4* pk, int64_t i, const double* q,
                                           const double* p, const PackScale& ps) {
  pack_write(pk, i, (float)((q[0] - ps.cx) * ps.s), (float)((q[1] - ps.cy) * ps.s),
             (float)((q[2] - ps.cz) * ps.s), (float)p[0], (float)p[1], (float)p[2]);
}

// ---------------------------------------------------------------- epilogues
// What happens to one point's finished forward sums (F_i and the raw Phi sum
// Sum c g d_s).  Used by the exact and the Barnes-Hut kernels alike.
struct FwdEpi {
  double* q;            // N x 3 state (updated in place when h != 0)
  double* p;            // N x 3 state
  float4* pack_next;    // next step's pack (NULL = none)
  float4* raw_next;     // next step's FP32 raw positions {x,y,z,0} (NULL = none)
  double* F_out;        // N x 3 F (NULL = none)
  double* Phi_out;      // N x 3 Phi (NULL = none)
  double* pf_part;      // per-point p.F for H (NULL = none), N entries
  const double* center; // recentring point (device, 3 doubles)
  double s;             // coordinate scale
  double phi_scale;     // sigma^-2 / s
  double h;             // Euler step (0 = no update)
  bool iterate;         // fixed-point pass of a semi-implicit step: the next pack
                        // gets (q, p + h Phi), the state is not changed
  int64_t N;
};

// Epilogue of point i (state and output rows) whose pack entry is ipk, with
// recentring point `center` (batched subjects have their own packs/centres).
__device__ __forceinline__ void fwd_epilogue_at(int64_t i, int64_t ipk, const double* center,
                                                const double F[3], const double Sraw[3],
                                                const FwdEpi& e) {
  double Phi[3] = {Sraw[0] * e.phi_scale, Sraw[1] * e.phi_scale, Sraw[2] * e.phi_scale};
  double* q = e.q + 3 * i;
  double* p = e.p + 3 * i;
  if (e.F_out) {
    e.F_out[3 * i + 0] = F[0];
    e.F_out[3 * i + 1] = F[1];
    e.F_out[3 * i + 2] = F[2];
  }
  if (e.Phi_out) {
    e.Phi_out[3 * i + 0] = Phi[0];
    e.Phi_out[3 * i + 1] = Phi[1];
    e.Phi_out[3 * i + 2] = Phi[2];
  }
  if (e.pf_part) e.pf_part[i] = p[0] * F[0] + p[1] * F[1] + p[2] * F[2];
  if (e.h != 0.0) {
    double qn[3], pn[3];
    for (int a = 0; a < 3; a++) {
      qn[a] = e.iterate ? q[a] : q[a] + e.h * F[a];
      pn[a] = p[a] + e.h * Phi[a];
    }
    if (!e.iterate)
      for (int a = 0; a < 3; a++) q[a] = qn[a], p[a] = pn[a];
    PackScale ps{center[0], center[1], center[2], e.s};
    if (e.pack_next) pack_state(e.pack_next, ipk, qn, pn, ps);
    if (e.raw_next)
      e.raw_next[ipk] = make_float4((float)qn[0], (float)qn[1], (float)qn[2], 0.f);
  }
}

__device__ __forceinline__ void fwd_epilogue(int64_t i, const double F[3], const double Sraw[3],
                                             const FwdEpi& e) {
  fwd_epilogue_at(i, i, e.center, F, Sraw, e);
}

// Tracer points carried by the velocity field of Eq. 3: with v = Sum_j g p_j
// finished, x += h v (FP64) and the next step's tracer record
// {(x - c) s, 0} is written.
struct TracerEpi {
  double* x;                // M x 3 tracer positions (updated when h != 0)
  float4* xpk_next;         // next step's tracer records (NULL = none)
  float4* xraw_next;        // next step's FP32 tracer positions (NULL = none)
  double* v_out;            // M x 3 velocity (NULL = none)
  const double* center;     // recentring point (the particles')
  double s;                 // coordinate scale
  double h;
  int64_t M;
};

__device__ __forceinline__ void tracer_epilogue(int64_t i, const double v[3], const TracerEpi& e) {
  if (e.v_out)
    for (int a = 0; a < 3; a++) e.v_out[3 * i + a] = v[a];
  if (e.h != 0.0) {
    double xn[3];
    for (int a = 0; a < 3; a++) {
      xn[a] = e.x[3 * i + a] + e.h * v[a];
      e.x[3 * i + a] = xn[a];
    }
    if (e.xpk_next)
      e.xpk_next[i] = make_float4((float)((xn[0] - e.center[0]) * e.s),
                                  (float)((xn[1] - e.center[1]) * e.s),
                                  (float)((xn[2] - e.center[2]) * e.s), 0.f);
    if (e.xraw_next) e.xraw_next[i] = make_float4((float)xn[0], (float)xn[1], (float)xn[2], 0.f);
  }
}

// Adjoint.  With a = alpha^{k+1}, b = beta^{k+1}, w = b_i - b_j and the
// scaled difference d_s, the backward step is alpha += h dA, beta += h dB,
//   dA = sigma^-2 (-A1 / s + A2 - 2 ln2 A3),   dB = B1 + sigma^-2 B2 / s,
// A1 = Sum g (a_i.p_j + a_j.p_i) d_s, A2 = Sum c g w, A3 = Sum c g (w.d_s) d_s,
// B1 = Sum g a_j, B2 = Sum g (w.d_s) p_j.  The FP32 adjoint pack holds beta
// scaled by mu = 2 ln2 s (b' = mu b, so w' = mu w).  Because
// 2 ln2 s^2 = sigma^-2 (s^2 = log2(e) / (2 sigma^2)), the pair kernels then
// accumulate three sums with no constants,
//   A13' = Sum (g (a_i.p_j + a_j.p_i) + c g (w'.d_s)) d_s,   A2' = Sum c g w',
//   B'   = Sum g (a_j + (w'.d_s) p_j),
// and dA = sigma^-2 (A2' / mu - A13' / s), dB = B'.
struct AdjEpi {
  double* al;           // N x 3 alpha (updated in place when h != 0)
  double* be;           // N x 3 beta
  float4* pack_next;    // next (earlier) step's adjoint pack (NULL = none)
  double* dA_out;       // N x 3 (NULL = none)
  double* dB_out;       // N x 3 (NULL = none)
  const double* F0;     // when non-NULL (last backward step): grad = beta + F0
  double* grad;         // N x 3 gradient output
  double* rho;          // N x 3 (NULL = none): receives h dB (semi-implicit adjoint)
  bool pack_rho;        // the next adjoint pack gets (0, rho) instead of (alpha, beta)
  double inv_s2;        // sigma^-2
  double inv_s;         // 1 / s
  double mu;            // beta's scale in the adjoint pack
  double h;
  int64_t N;
};

// Beta's scale in the FP32 adjoint pack for coordinate scale s.
__host__ __device__ __forceinline__ double adj_beta_scale(double s) {
  return 1.3862943611198906 * s;  // 2 ln 2 s
}

__device__ __forceinline__ void adj_epilogue_at(int64_t i, int64_t ipk, const double A13[3],
                                                const double A2[3], const double B[3],
                                                const AdjEpi& e) {
  double dA[3], dB[3];
  for (int a = 0; a < 3; a++) {
    dA[a] = e.inv_s2 * (A2[a] / e.mu - e.inv_s * A13[a]);
    dB[a] = B[a];
  }
  if (e.dA_out)
    for (int a = 0; a < 3; a++) e.dA_out[3 * i + a] = dA[a];
  if (e.dB_out)
    for (int a = 0; a < 3; a++) e.dB_out[3 * i + a] = dB[a];
  if (e.h != 0.0) {
    double an[3], bn[3], hb[3];
    for (int a = 0; a < 3; a++) {
      hb[a] = e.h * dB[a];
      an[a] = e.al[3 * i + a] + e.h * dA[a];
      bn[a] = e.be[3 * i + a] + hb[a];
      e.al[3 * i + a] = an[a];
      e.be[3 * i + a] = bn[a];
    }
    if (e.rho)
      for (int a = 0; a < 3; a++) e.rho[3 * i + a] = hb[a];
    if (e.pack_next && e.pack_rho)
      pack_write(e.pack_next, ipk, 0.f, 0.f, 0.f, (float)(e.mu * hb[0]), (float)(e.mu * hb[1]),
                 (float)(e.mu * hb[2]));
    else if (e.pack_next)
      pack_write(e.pack_next, ipk, (float)an[0], (float)an[1], (float)an[2],
                 (float)(e.mu * bn[0]), (float)(e.mu * bn[1]), (float)(e.mu * bn[2]));
    if (e.F0)
      for (int a = 0; a < 3; a++) e.grad[3 * i + a] = bn[a] + e.F0[3 * i + a];
  }
}

__device__ __forceinline__ void adj_epilogue(int64_t i, const double A13[3], const double A2[3],
                                             const double B[3], const AdjEpi& e) {
  adj_epilogue_at(i, i, A13, A2, B, e);
}

}  // namespace gs
