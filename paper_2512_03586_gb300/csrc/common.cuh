// common.cuh -- shared device definitions of the ES-BGK library (sm_103a).
//
// Layouts (device, all inside the caller's workspace):
//   f  : storage type S, [cell c = j*nx + i][vy][vx]  -- velocity-contiguous,
//        one cell's N_v^2 values are one coalesced run.
//   U  : float64 [4][nc]  (rho, rho u_x, rho u_y, E), structure of arrays.
//   Phi: float64 [stage][4][nc], the Euler divergences of earlier stages.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define ESBGK_DEV __device__ __forceinline__

namespace esbgk {

constexpr int kThreads = 256;            // threads of every per-cell CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMaxStages = 4;
constexpr double kPi = 3.14159265358979323846;

// Geometry of one problem (Sec. 3.2).
struct Geo {
  int nx, ny, nc;      // cells per axis, cells
  int nv, nvv;         // velocity nodes per axis, nv*nv
  int bcx, bcy;        // 0 periodic, 1 outflow
  double dx, dy;       // cell sizes
  double vmax, dv, w;  // velocity bound, step, quadrature weight dv^2
  double v0;           // first node, -vmax + dv/2
  // float copies for the FP32 arithmetic (rounded once on the host)
  float fv0, fdv, fw, fidx, fidy;
};

// Model constants (Sec. 2, 3.1), with float copies for the FP32 arithmetic.
struct Model {
  double beta, tau, eps_w, eta_factor, delta;
  float fbeta, ftau, feps_w;
  int tau_rho;  // relaxation time tau * rho (else tau)
  int comp_moments;  // compensated FP32 moment sums
};

// The double or the float copy of a constant, for arithmetic type R.
template <typename R>
ESBGK_DEV R pick(double d, float f);
template <>
ESBGK_DEV double pick<double>(double d, float) {
  return d;
}
template <>
ESBGK_DEV float pick<float>(double, float f) {
  return f;
}

// Device error word: first error wins.
struct DevErr {
  int code;
  int pad;
  long long cell;
};

enum : int { kErrNone = 0, kErrNonRealizable = 1, kErrTimeout = 2 };

ESBGK_DEV void report_error(DevErr* e, int code, long long cell) {
  if (e && atomicCAS(&e->code, 0, code) == 0) e->cell = cell;
}

// ---------------------------------------------------------------------------
// mbarrier helpers (shared-memory barriers that asynchronous units arrive on).

ESBGK_DEV unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

ESBGK_DEV void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the asynchronous proxy.
ESBGK_DEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

ESBGK_DEV bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete, giving up after a
// bounded number of polls (false: it did not complete).
constexpr unsigned kWaitLimit = 1u << 20;
ESBGK_DEV bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit = kWaitLimit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 32-bit integer hash (the "lowbias32" xorshift-multiply mixer published by
// C. Wellons, 2018): counter-based random bits for stochastic rounding.
ESBGK_DEV uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// float -> bf16 with stochastic rounding: add 16 random bits below the kept
// mantissa and truncate, so that the rounding error has zero mean.
ESBGK_DEV unsigned short bf16_sr_bits(float v, uint32_t r) {
  return (unsigned short)((__float_as_uint(v) + (r & 0xffffu)) >> 16);
}

// Storage <-> arithmetic type mapping.
template <typename S> struct Real;
template <> struct Real<double> { using T = double; };
template <> struct Real<float> { using T = float; };
template <> struct Real<__nv_bfloat16> { using T = float; };

ESBGK_DEV double ld(const double* p) { return __ldg(p); }
ESBGK_DEV float ld(const float* p) { return __ldg(p); }
ESBGK_DEV float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
ESBGK_DEV void st(double* p, double v) { *p = v; }
ESBGK_DEV void st(float* p, float v) { *p = v; }
ESBGK_DEV void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// plain (coherent) loads for arrays written earlier in the same kernel by the
// same thread (accumulators updated in place)
ESBGK_DEV double ldc(const double* p) { return *p; }
ESBGK_DEV float ldc(const float* p) { return *p; }
ESBGK_DEV float ldc(const __nv_bfloat16* p) { return __bfloat162float(*p); }

ESBGK_DEV double fdiv(double a, double b) { return a / b; }
ESBGK_DEV float fdiv(float a, float b) { return __fdividef(a, b); }

// Precision-explicit |x|, sqrt and max: a float argument must never be
// promoted to double (on GB300 the FP64 pipe is narrow).
ESBGK_DEV float rabs(float x) { return fabsf(x); }
ESBGK_DEV double rabs(double x) { return fabs(x); }
ESBGK_DEV float rsqrt_(float x) { return sqrtf(x); }
ESBGK_DEV double rsqrt_(double x) { return sqrt(x); }
ESBGK_DEV float rmax(float a, float b) { return fmaxf(a, b); }
ESBGK_DEV double rmax(double a, double b) { return fmax(a, b); }

// 2^x.  FP32: the hardware approximation (ex2.approx, max rel. error ~2^-22).
ESBGK_DEV float exp2r(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
ESBGK_DEV double exp2r(double x) { return exp2(x); }

// Index of cell i + d along an axis of n cells under boundary condition bc
// (0 periodic, 1 outflow: ghost cells copy the edge cell).
ESBGK_DEV int nb(int i, int n, int bc) {
  if (bc == 0) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// CWENO3 (Levy-Puppo-Russo) value at the face of the middle cell that faces
// `c`, from cell averages a | b | c.  P_L, P_R are the one-sided lines,
// P_0 = (P_opt - P_L/4 - P_R/4)/(1/2); the face value of
// sum_k alpha_k P_k / sum_k alpha_k with alpha_k = d_k/(eps + IS_k)^2 is
// evaluated with a single division by multiplying every alpha through by
// (eps+IS_0)^2 (eps+IS_L)^2 (eps+IS_R)^2.
template <typename R>
ESBGK_DEV R cweno_face(R a, R b, R c, R epsw) {
  const R dl = b - a, dr = c - b, d1 = c - a;
  const R D = dr - dl;
  const R PL = b + R(0.5) * dl;
  const R PR = b + R(0.5) * dr;
  const R P0 = b + D * R(1.0 / 6.0) + R(0.25) * d1;
  const R IS0 = R(13.0 / 3.0) * D * D + R(0.25) * d1 * d1;
  R sL = epsw + dl * dl;
  sL *= sL;
  R sR = epsw + dr * dr;
  sR *= sR;
  R s0 = epsw + IS0;
  s0 *= s0;
  const R a0 = R(0.5) * sL * sR;
  const R aL = R(0.25) * s0 * sR;
  const R aR = R(0.25) * s0 * sL;
  return fdiv(a0 * P0 + aL * PL + aR * PR, a0 + aL + aR);
}

// Compensated summation of FP32 moments.  comp_add: Neumaier's variant of
// Kahan summation (the rounding error of s + x, exact, kept in c; valid in
// either magnitude order).  group_sum_comp: the butterfly over L lanes with
// the error-free two-sum of the partial sums at every level, compensations
// added alongside; the result is s + c, identical in every lane (two-sum's
// error term does not depend on the operand order).
ESBGK_DEV void comp_add(float& s, float& c, float x) {
  const float t = s + x;
  c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}
template <int L>
ESBGK_DEV float group_sum_comp(float s, float c, unsigned mask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) {
    const float so = __shfl_xor_sync(mask, s, o, L), co = __shfl_xor_sync(mask, c, o, L);
    const float t = s + so, bp = t - s;
    c += co + ((s - (t - bp)) + (so - bp));
    s = t;
  }
  return s + c;
}

// The same face value for two independent stencils at once, on the paired
// FP32 instructions of sm_100-family GPUs (two lanes of float arithmetic per
// issued instruction); the divisions stay per component.
ESBGK_DEV float2 splat2(float a) { return make_float2(a, a); }
ESBGK_DEV float2 cweno_face2(float2 a, float2 b, float2 c, float2 epsw) {
  const float2 m1 = splat2(-1.0f);
  const float2 dl = __ffma2_rn(a, m1, b);  // b - a
  const float2 dr = __ffma2_rn(b, m1, c);  // c - b
  const float2 d1 = __ffma2_rn(a, m1, c);  // c - a
  const float2 D = __ffma2_rn(dl, m1, dr);
  const float2 PL = __ffma2_rn(splat2(0.5f), dl, b);
  const float2 PR = __ffma2_rn(splat2(0.5f), dr, b);
  const float2 P0 = __ffma2_rn(splat2(0.25f), d1, __ffma2_rn(D, splat2(1.0f / 6.0f), b));
  const float2 IS0 = __ffma2_rn(__fmul2_rn(splat2(13.0f / 3.0f), D), D, __fmul2_rn(__fmul2_rn(splat2(0.25f), d1), d1));
  float2 sL = __ffma2_rn(dl, dl, epsw);
  sL = __fmul2_rn(sL, sL);
  float2 sR = __ffma2_rn(dr, dr, epsw);
  sR = __fmul2_rn(sR, sR);
  float2 s0 = __fadd2_rn(epsw, IS0);
  s0 = __fmul2_rn(s0, s0);
  const float2 a0 = __fmul2_rn(__fmul2_rn(splat2(0.5f), sL), sR);
  const float2 q = __fmul2_rn(splat2(0.25f), s0);
  const float2 aL = __fmul2_rn(q, sR);
  const float2 aR = __fmul2_rn(q, sL);
  const float2 num = __ffma2_rn(a0, P0, __ffma2_rn(aL, PL, __fmul2_rn(aR, PR)));
  const float2 den = __fadd2_rn(__fadd2_rn(a0, aL), aR);
  return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

// F(b, c, d) - F(a, b, c) for two node pairs: the difference of the upwind
// CWENO3 face values at the two faces of the middle cells b | c, each face
// from the cell behind it and its two neighbours (the same weights as
// cweno_face2).  The three differences d1 = b - a, d2 = c - b, d3 = d - c and
// their squares t = d^2 + eps, s = t^2 serve both faces: with dl, dr the
// differences behind and ahead of a face's upwind cell,
//   F = u + 1/2 [s_l s_r (dl + 5 dr)/6 + (z/2)(s_r dl + s_l dr)] / [s_l s_r + (z/2)(s_l + s_r)],
//   z/2 = (55/(12 sqrt 2) (t_l + t_r) - 49/(6 sqrt 2) dl dr + eps (1 - 55/6)/sqrt 2)^2
// (z = (eps + 13/3 (dr - dl)^2 + 1/4 (dl + dr)^2)^2 rewritten through the
// squares already formed).
ESBGK_DEV float2 cweno_dface2(float2 a, float2 b, float2 c, float2 d, float2 epsw) {
  const float2 m1 = splat2(-1.0f);
  const float2 d1 = __ffma2_rn(a, m1, b), d2 = __ffma2_rn(b, m1, c), d3 = __ffma2_rn(c, m1, d);
  const float2 t1 = __ffma2_rn(d1, d1, epsw), t2 = __ffma2_rn(d2, d2, epsw), t3 = __ffma2_rn(d3, d3, epsw);
  const float2 s1 = __fmul2_rn(t1, t1), s2 = __fmul2_rn(t2, t2), s3 = __fmul2_rn(t3, t3);
  const float2 C1 = splat2((float)(55.0 / 12.0 / 1.4142135623730951));
  const float2 C2 = splat2((float)(-49.0 / 6.0 / 1.4142135623730951));
  const float2 c3 = __fmul2_rn(epsw, splat2((float)((1.0 - 55.0 / 6.0) / 1.4142135623730951)));
  const float2 c16 = splat2(1.0f / 6.0f), c56 = splat2(5.0f / 6.0f);
  auto face = [&](float2 u, float2 dl, float2 dr, float2 tl, float2 tr, float2 sl, float2 sr) {
    const float2 z0 = __ffma2_rn(__fadd2_rn(tl, tr), C1, __ffma2_rn(__fmul2_rn(dl, dr), C2, c3));
    const float2 zh = __fmul2_rn(z0, z0), xy = __fmul2_rn(sl, sr);
    const float2 p = __ffma2_rn(c16, dl, __fmul2_rn(c56, dr));
    const float2 tt = __ffma2_rn(sr, dl, __fmul2_rn(sl, dr));
    const float2 num = __ffma2_rn(xy, p, __fmul2_rn(zh, tt));
    const float2 den = __ffma2_rn(zh, __fadd2_rn(sl, sr), xy);
    float rx, ry;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(den.y));
    return __ffma2_rn(splat2(0.5f), __fmul2_rn(num, make_float2(rx, ry)), u);
  };
  return __ffma2_rn(face(b, d1, d2, t1, t2, s1, s2), m1, face(c, d2, d3, t2, t3, s2, s3));
}

// Case of global work unit u: the largest c with off[c] <= u (off ascending,
// off[0] = 0, n >= 1).
ESBGK_DEV int find_case(const int* off, int n, int u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename R>
ESBGK_DEV R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a group of L lanes (L = 32: the warp; L = 16: a half-warp, mask
// holding that half's lanes).
template <int L, typename R>
ESBGK_DEV R group_sum(R v, unsigned mask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, L);
  return v;
}

// Block-wide sum of N per-thread values (kThreads threads).  Result lands in
// out[0..N) (shared memory, float64) after the call; red is shared scratch of
// kWarps*N doubles.  Warp sums run in the arithmetic type R, the cross-warp
// sum in float64.
template <int N, typename R>
ESBGK_DEV void block_sum(R (&v)[N], double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int n = 0; n < N; ++n) {
    R s = warp_sum(v[n]);
    if (lane == 0) red[warp * N + n] = (double)s;
  }
  __syncthreads();
  if (warp == 0 && lane < N) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w * N + lane];
    out[lane] = s;
  }
  __syncthreads();
}

}  // namespace esbgk
