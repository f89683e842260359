// kernels_impl.cuh -- the per-precision kernels of the ES-BGK library.
//
// Included by one translation unit per storage type S (double, float,
// __nv_bfloat16), each of which instantiates the launchers declared in
// launch.h.  Per-element arithmetic runs in R = Real<S>::T.
//
// Work decomposition: one warp owns one cell.  Its 32 lanes stride over the
// N_v^2 velocities (lane l always handles nodes l, l+32, ...), so every
// velocity reduction is a warp butterfly (no CTA barrier) and the per-cell
// solves run redundantly in all lanes (no broadcast).  A CTA holds
// kCellWarps independent cells; per-warp shared memory keeps f* of the cell
// between the passes.  A persistent grid walks the compacted work
// list: kinetic cells, then buffer cells, then chunks of 32 fluid cells (one
// lane per cell).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "launch.h"


namespace esbgk {

constexpr int kCellWarps = 4;                  // cells (warps) per CTA at most
constexpr int kCellThreads = kCellWarps * 32;  // threads per CTA at most
constexpr double kLog2e = 1.4426950408889634;

// Monomial index of xi_x^p xi_y^q (p + q <= 4) among the 15 projection sums.
__host__ __device__ constexpr int mono(int p, int q) { return (p + q) * (p + q + 1) / 2 + q; }

// Per-cell parameters of the discrete Gaussian, identical in every lane.
template <typename R>
struct CellPar {
  R ux, uy;          // mean velocity
  R qxx, qxy, qyy;   // exponent -log2(e)/2 (v-u)^T Tt^{-1} (v-u) = qxx cx^2 + qxy cx cy + qyy cy^2
  R pref;            // rho / (2 pi sqrt(det Tt))
  R isT;             // 1/sqrt(T), scale of xi = (v-u)/sqrt(T)
  R t[6];            // projection targets (rho, 0, 0, rho Tt/T)
  R a[6];            // projection coefficients
};

// Velocity node iterator of one lane: nodes k = lane, lane+32, ... with
// (kx, ky) = (k mod N_v, k div N_v) and the node velocities
// (vx, vy) = v0 + (kx, ky) dv, advanced without divisions or int->float
// conversions (on GB300 conversions run on the narrow FP64 pipe).  fx, fy
// hold kx, ky as exact small integers in R, so vx, vy are bit-identical to
// v0 + R(kx) dv.
template <typename R>
struct NodeIter {
  int k, kx, dkx, nv, step;
  R fx, fy, fdkx, fdky, fnv, v0, dv;
  // Nodes start, start + step, ... (step = 32 lanes x nodes per lane).
  ESBGK_DEV NodeIter(int start, int nv_, R v0_, R dv_, int step_ = 32)
      : k(start), kx(start % nv_), dkx(step_ % nv_), nv(nv_), step(step_), fx(R(start % nv_)), fy(R(start / nv_)),
        fdkx(R(step_ % nv_)), fdky(R(step_ / nv_)), fnv(R(nv_)), v0(v0_), dv(dv_) {}
  ESBGK_DEV R vx() const { return v0 + fx * dv; }
  ESBGK_DEV R vy() const { return v0 + fy * dv; }
  ESBGK_DEV void next() {
    k += step;
    kx += dkx;
    fx += fdkx;
    fy += fdky;
    if (kx >= nv) {
      kx -= nv;
      fx -= fnv;
      fy += R(1);
    }
  }
};

// Vector loads and stores of W consecutive nodes (16 bytes at most).
template <typename S, int W>
struct VecIO;
template <>
struct VecIO<float, 4> {
  static ESBGK_DEV void ld(const float* p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  }
  static ESBGK_DEV void ldc(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  }
  static ESBGK_DEV void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static ESBGK_DEV void st_sr(float* p, const float (&v)[4], uint32_t) { st(p, v); }
};
template <>
struct VecIO<float, 2> {
  static ESBGK_DEV void ld(const float* p, float (&v)[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x, v[1] = t.y;
  }
  static ESBGK_DEV void ldc(const float* p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
  static ESBGK_DEV void st(float* p, const float (&v)[2]) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
  static ESBGK_DEV void st_sr(float* p, const float (&v)[2], uint32_t) { st(p, v); }
};
template <>
struct VecIO<double, 2> {
  static ESBGK_DEV void ld(const double* p, double (&v)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x, v[1] = t.y;
  }
  static ESBGK_DEV void ldc(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
  static ESBGK_DEV void st(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
  static ESBGK_DEV void st_sr(double* p, const double (&v)[2], uint32_t) { st(p, v); }
};
template <>
struct VecIO<__nv_bfloat16, 4> {
  static ESBGK_DEV void unpack(uint2 t, float (&v)[4]) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.y));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
  static ESBGK_DEV void ld(const __nv_bfloat16* p, float (&v)[4]) {
    unpack(__ldg(reinterpret_cast<const uint2*>(p)), v);
  }
  static ESBGK_DEV void ldc(const __nv_bfloat16* p, float (&v)[4]) {
    unpack(*reinterpret_cast<const uint2*>(p), v);
  }
  static ESBGK_DEV void st(__nv_bfloat16* p, const float (&v)[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&a);
    t.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
  }
  // stochastic rounding; key: a random 32-bit value for the group
  static ESBGK_DEV void st_sr(__nv_bfloat16* p, const float (&v)[4], uint32_t key) {
    const uint32_t r0 = mix32(key), r1 = mix32(key ^ 0x9e3779b9u);
    uint2 t;
    t.x = (uint32_t)bf16_sr_bits(v[0], r0) | ((uint32_t)bf16_sr_bits(v[1], r0 >> 16) << 16);
    t.y = (uint32_t)bf16_sr_bits(v[2], r1) | ((uint32_t)bf16_sr_bits(v[3], r1 >> 16) << 16);
    *reinterpret_cast<uint2*>(p) = t;
  }
};
template <>
struct VecIO<__nv_bfloat16, 2> {
  static ESBGK_DEV void unpack(unsigned t, float (&v)[2]) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t));
    v[0] = a.x, v[1] = a.y;
  }
  static ESBGK_DEV void ld(const __nv_bfloat16* p, float (&v)[2]) {
    unpack(__ldg(reinterpret_cast<const unsigned*>(p)), v);
  }
  static ESBGK_DEV void ldc(const __nv_bfloat16* p, float (&v)[2]) { unpack(*reinterpret_cast<const unsigned*>(p), v); }
  static ESBGK_DEV void st(__nv_bfloat16* p, const float (&v)[2]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    *reinterpret_cast<unsigned*>(p) = *reinterpret_cast<const unsigned*>(&a);
  }
  static ESBGK_DEV void st_sr(__nv_bfloat16* p, const float (&v)[2], uint32_t key) {
    const uint32_t r = mix32(key);
    *reinterpret_cast<unsigned*>(p) = (uint32_t)bf16_sr_bits(v[0], r) | ((uint32_t)bf16_sr_bits(v[1], r >> 16) << 16);
  }
};
// shared-memory copies of f* in the arithmetic type
template <typename R, int W>
struct SmemVec;
template <>
struct SmemVec<float, 4> {
  static ESBGK_DEV void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static ESBGK_DEV void ld(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  }
};
template <>
struct SmemVec<float, 2> {
  static ESBGK_DEV void st(float* p, const float (&v)[2]) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
  static ESBGK_DEV void ld(const float* p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
};
template <>
struct SmemVec<double, 2> {
  static ESBGK_DEV void st(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
  static ESBGK_DEV void ld(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x, v[1] = t.y;
  }
};
// nodes per vector group for storage type S
template <typename S>
struct VecW {
  static constexpr int value = 16 / sizeof(typename Real<S>::T) < 4 ? 16 / sizeof(typename Real<S>::T) : 4;
};

// Temperature tensor from the moments of a cell (hypothesis H3 and Sec. 2).
// m are the raw sums over nodes of f, c f, c (x) c f with c = v - u0 about a
// reference velocity u0 (this keeps Theta = S'/rho - (u-u0)(u-u0) free of
// cancellation); w is the quadrature weight.
//   rho = w m0, u = u0 + w m1/rho, Theta, T = tr(Theta)/2;
//   relax: Theta <- (Theta + k T I)/(1 + k), k = h (1 - beta) -- the exact
//          stress moment of the implicit stage;
//   Tt = (1 - beta) T I + beta Theta; its determinant in float64.
// Returns false for a non-realizable state.
template <typename R>
ESBGK_DEV bool es_params(const R (&m)[6], R u0x, R u0y, R w, R beta, R h, bool relax, CellPar<R>& P) {
  const R rho = w * m[0];
  if (!(rho > R(0))) return false;
  const R ir = R(1) / rho;
  const R dux = w * m[1] * ir, duy = w * m[2] * ir;
  R txx = w * m[3] * ir - dux * dux, txy = w * m[4] * ir - dux * duy, tyy = w * m[5] * ir - duy * duy;
  const R T = R(0.5) * (txx + tyy);
  if (!(T > R(0))) return false;
  if (relax) {
    const R k = h * (R(1) - beta);
    const R inv = R(1) / (R(1) + k);
    txx = (txx + k * T) * inv;
    txy = txy * inv;
    tyy = (tyy + k * T) * inv;
  }
  const R Txx = (R(1) - beta) * T + beta * txx;
  const R Txy = beta * txy;
  const R Tyy = (R(1) - beta) * T + beta * tyy;
  const double det = fma((double)Txx, (double)Tyy, -(double)Txy * (double)Txy);
  if (!(det > 0.0)) return false;
  const R idet = R(1) / R(det);  // det in float64 (cancellation); its inverse in the arithmetic type
  P.ux = u0x + dux;
  P.uy = u0y + duy;
  P.qxx = R(-0.5 * kLog2e) * Tyy * idet;
  P.qxy = R(kLog2e) * Txy * idet;
  P.qyy = R(-0.5 * kLog2e) * Txx * idet;
  P.pref = rho * R(0.5 / kPi) / rsqrt_(R(det));
  P.isT = R(1) / rsqrt_(T);
  const R rT = rho / T;
  P.t[0] = rho;
  P.t[1] = R(0);
  P.t[2] = R(0);
  P.t[3] = rT * Txx;
  P.t[4] = rT * Txy;
  P.t[5] = rT * Tyy;
  return true;
}

// Parameters of the Maxwellian of (rho, u, T): Tt = T I.
template <typename R>
ESBGK_DEV bool maxwell_params(double rho, double ux, double uy, double T, CellPar<R>& P) {
  if (!(rho > 0.0) || !(T > 0.0)) return false;
  const R iT = R(1) / R(T);
  P.ux = R(ux);
  P.uy = R(uy);
  P.qxx = R(-0.5 * kLog2e) * iT;
  P.qxy = R(0);
  P.qyy = P.qxx;
  P.pref = R(rho) * R(0.5 / kPi) * iT;
  P.isT = R(1) / rsqrt_(R(T));
  P.t[0] = R(rho);
  P.t[1] = P.t[2] = R(0);
  P.t[3] = R(rho);
  P.t[4] = R(0);
  P.t[5] = R(rho);
  return true;
}

template <typename R>
ESBGK_DEV R gauss_at(const CellPar<R>& P, R cx, R cy) {
  return P.pref * exp2r(P.qxx * cx * cx + P.qxy * cx * cy + P.qyy * cy * cy);
}

// Projection of the discrete Gaussian onto exact moments (whole warp): the 15
// sums w sum G xi^p eta^q over the nodes, then H a = t - r with
// H_mn = w sum G psi_m psi_n, r_m = w sum G psi_m, psi = (1, x, y, x^2, xy, y^2).
// After this G_hat = G (1 + a . psi) has w sum psi G_hat = t.
// L lanes per cell (32, or 16 for a half-warp; mask: the group's lanes).
template <typename R, int L>
ESBGK_DEV bool project_solve(const R (&s)[15], int lane, CellPar<R>& P, unsigned mask);

template <typename R, int W = 1, int L = 32>
ESBGK_DEV bool project(const Geo& g, int lane, CellPar<R>& P, unsigned mask = 0xffffffffu) {
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  R s[15];
#pragma unroll
  for (int n = 0; n < 15; ++n) s[n] = R(0);
  NodeIter<R> it(lane * W, g.nv, v0, dv, L * W);
  if constexpr (std::is_same<R, float>::value && W % 2 == 0) {
    // Row segments: a lane takes runs of whole node groups of one velocity
    // row (v_y fixed), sums G x^p (p = 0..4) along the run on the paired
    // FP32 instructions and adds them times y^q into the 15 sums once per run.
    // A segment is half a row when the row has an even number of groups and
    // that still leaves every lane a segment, else a whole row.  G is formed
    // from the same operands as in the relaxation pass (cx = (v_x - u_x) +
    // j dv of the group's first node), so both passes see the same G.
    const int gpr = g.nv / W, nrows = g.nv;
    const int segg = (gpr % 2 == 0 && nrows * 2 >= L) ? gpr / 2 : gpr;
    const int nseg = nrows * (gpr / segg);
    const float2 qxx2 = splat2(P.qxx), pref2 = splat2(P.pref), isT2 = splat2(P.isT);
#pragma unroll 1
    for (int sg = lane; sg < nseg; sg += L) {
      const int k0 = sg * segg * W;  // first node of the segment
      const int ky = k0 / g.nv, kx0 = k0 - ky * g.nv;
      const float cy = (v0 + R(ky) * dv) - P.uy, y = cy * P.isT;
      const float2 qy = splat2(P.qyy * cy * cy), qc = splat2(P.qxy * cy);
      float2 R0 = splat2(0.0f), R1 = R0, R2 = R0, R3 = R0, R4 = R0;
#pragma unroll 1
      for (int gg = 0; gg < segg; ++gg) {
        const float cx0 = (v0 + R(kx0 + gg * W) * dv) - P.ux;
#pragma unroll
        for (int j = 0; j < W; j += 2) {
          const float cxa = cx0 + R(j) * dv;
          const float2 cx = make_float2(cxa, cxa + dv);
          const float2 e = __ffma2_rn(qxx2, __fmul2_rn(cx, cx), __ffma2_rn(qc, cx, qy));
          const float2 G = __fmul2_rn(pref2, make_float2(exp2r(e.x), exp2r(e.y)));
          const float2 x = __fmul2_rn(cx, isT2);
          const float2 t1 = __fmul2_rn(G, x), t2 = __fmul2_rn(t1, x), t3 = __fmul2_rn(t2, x);
          R0 = __fadd2_rn(R0, G);
          R1 = __fadd2_rn(R1, t1);
          R2 = __fadd2_rn(R2, t2);
          R3 = __fadd2_rn(R3, t3);
          R4 = __ffma2_rn(t3, x, R4);
        }
      }
      const float rr[5] = {R0.x + R0.y, R1.x + R1.y, R2.x + R2.y, R3.x + R3.y, R4.x + R4.y};
      float yq[5];
      yq[0] = 1.0f;
#pragma unroll
      for (int q = 1; q < 5; ++q) yq[q] = yq[q - 1] * y;
#pragma unroll
      for (int pp = 0; pp < 5; ++pp)
#pragma unroll
        for (int q = 0; q + pp < 5; ++q) s[mono(pp, q)] = fmaf(rr[pp], yq[q], s[mono(pp, q)]);
    }
  } else {
#pragma unroll 1
  for (; it.k < g.nvv; it.next())
#pragma unroll
    for (int j = 0; j < W; ++j) {
    const R cx = it.vx() + R(j) * dv - P.ux, cy = it.vy() - P.uy;
    const R G = gauss_at(P, cx, cy);
    const R x = cx * P.isT, y = cy * P.isT;
    const R Gx = G * x, Gy = G * y;
    const R Gxx = Gx * x, Gxy = Gx * y, Gyy = Gy * y;
    s[0] += G;
    s[1] += Gx;
    s[2] += Gy;
    s[3] += Gxx;
    s[4] += Gxy;
    s[5] += Gyy;
    s[6] += Gxx * x;
    s[7] += Gxx * y;
    s[8] += Gxy * y;
    s[9] += Gyy * y;
    s[10] += Gxx * x * x;
    s[11] += Gxx * x * y;
    s[12] += Gxx * y * y;
    s[13] += Gxy * y * y;
    s[14] += Gyy * y * y;
  }
  }
#pragma unroll
  for (int n = 0; n < 15; ++n) s[n] = group_sum<L>(s[n], mask) * pick<R>(g.w, g.fw);
  return project_solve<R, L>(s, lane, P, mask);
}

// The projection's 6 x 6 system from the 15 weighted sums s (mono order),
// identical in every lane: H a = t - r.
template <typename R, int L>
ESBGK_DEV bool project_solve(const R (&s)[15], int lane, CellPar<R>& P, unsigned mask) {
  // H a = t - r by Gaussian elimination spread over lanes 0..5 (lane m holds
  // row m and its right-hand side; H is symmetric positive definite, so no
  // pivoting), pivot rows broadcast by shuffles.
  constexpr int PP[6] = {0, 1, 0, 2, 1, 0};
  constexpr int PQ[6] = {0, 0, 1, 0, 1, 2};
  const int row = lane < 6 ? lane : 5;
  R h[7];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    R v = R(0);
#pragma unroll
    for (int m = 0; m < 6; ++m)
      if (row == m) v = s[mono(PP[m] + PP[n], PQ[m] + PQ[n])];
    h[n] = v;
  }
  {
    R v = R(0);
#pragma unroll
    for (int m = 0; m < 6; ++m)
      if (row == m) v = P.t[m] - s[mono(PP[m], PQ[m])];
    h[6] = v;
  }
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    R piv[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) piv[n] = __shfl_sync(mask, h[n], p, L);
    ok = ok && piv[p] > R(0);
    const R fct = row > p ? h[p] / piv[p] : R(0);
#pragma unroll
    for (int n = 0; n < 7; ++n) h[n] -= fct * piv[n];
  }
  // back substitution: a_p = (b_p - sum_{n>p} U_pn a_n) / U_pp
#pragma unroll
  for (int p = 5; p >= 0; --p) {
    R acc = h[6];
#pragma unroll
    for (int n = p + 1; n < 6; ++n) acc -= h[n] * P.a[n];
    const R ap = __shfl_sync(mask, acc / h[p], p, L);
    P.a[p] = ap;
  }
  return ok;
}

// G_hat at node (cx, cy) = v - u.
template <typename R>
ESBGK_DEV R ghat(const CellPar<R>& P, R cx, R cy) {
  const R G = gauss_at(P, cx, cy);
  const R x = cx * P.isT, y = cy * P.isT;
  return G * (R(1) + P.a[0] + P.a[1] * x + P.a[2] * y + P.a[3] * x * x + P.a[4] * x * y + P.a[5] * y * y);
}

// G_hat at two nodes of one velocity row on the paired FP32 instructions:
// G_hat = G (c0 + c1 x + a3 x^2), the row's y terms of 1 + a . psi folded into
// c0 and c1, and the exponent's y terms into qy, qc, once per row.
struct GhatRow {
  float2 qy, qc, c0, c1;
};
ESBGK_DEV GhatRow ghat_row(const CellPar<float>& P, float cy) {
  const float y = cy * P.isT;
  return GhatRow{splat2(P.qyy * cy * cy), splat2(P.qxy * cy), splat2(1.0f + P.a[0] + P.a[2] * y + P.a[5] * y * y),
                 splat2(P.a[1] + P.a[4] * y)};
}
ESBGK_DEV float2 ghat_pair(const CellPar<float>& P, const GhatRow& r, float2 cx) {
  const float2 e = __ffma2_rn(splat2(P.qxx), __fmul2_rn(cx, cx), __ffma2_rn(r.qc, cx, r.qy));
  const float2 G = __fmul2_rn(splat2(P.pref), make_float2(exp2r(e.x), exp2r(e.y)));
  const float2 x = __fmul2_rn(cx, splat2(P.isT));
  return __fmul2_rn(G, __ffma2_rn(__ffma2_rn(splat2(P.a[3]), x, r.c1), x, r.c0));
}

// Element offsets of the two-cell cross stencil of cell c (BC mapped):
// o[0..3] = i-2, i-1, i+1, i+2 along x, o[4..7] the same along y.  Offsets
// are 32-bit: the library limits N_c N_v^2 to below 2^31 elements.
ESBGK_DEV void stencil_offsets(const Geo& g, int c, unsigned (&o)[8]) {
  const int i = c % g.nx, j = c / g.nx;
  const int d[4] = {-2, -1, 1, 2};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[q] = (unsigned)(j * g.nx + nb(i + d[q], g.nx, g.bcx)) * (unsigned)g.nvv;
    o[4 + q] = (unsigned)(nb(j + d[q], g.ny, g.bcy) * g.nx + i) * (unsigned)g.nvv;
  }
}

// ---------------------------------------------------------------------------
// Euler part (fluid cells), one lane per cell.

// Physical flux of Eq. Euler_Compact along d (0 = x, 1 = y), gamma = 2, and the
// local wave speed |u_d| + sqrt(gamma P/rho); a reconstructed face state whose
// pressure is not positive has no sound speed (P clipped at 0 in the speed).
template <typename R>
ESBGK_DEV void euler_phys(const R (&U)[4], int d, R (&F)[4], R& a) {
  const R rho = U[0], ux = U[1] / rho, uy = U[2] / rho;
  const R P = (R(2) - R(1)) * (U[3] - R(0.5) * rho * (ux * ux + uy * uy));
  const R un = d == 0 ? ux : uy;
  F[0] = rho * un;
  F[1] = U[1] * un + (d == 0 ? P : R(0));
  F[2] = U[2] * un + (d == 1 ? P : R(0));
  F[3] = un * (U[3] + P);
  a = rabs(un) + rsqrt_(R(2) * rmax(P, R(0)) / rho);
}

// Phi(U)(c): CWENO3 face states per component, local Lax-Friedrichs flux at
// the four faces of the cell, divergence (Eq. semidiscrete Euler).
// ovr/omask: faces whose flux is given (bit 2d: the face -1/2 along axis d,
// bit 2d+1: the face +1/2; ovr[bit][component]).
// WALLS (solid obstacles, View::wsrc): the line's values come from the
// stencil maps; a mirror image across a wall has its normal momentum reversed.
template <typename R, bool WALLS = false>
ESBGK_DEV void euler_phi_cell(const Geo& g, const double* __restrict__ U, int c, R epsw, R (&phi)[4],
                              const R (*ovr)[4] = nullptr, int omask = 0, const View* Vw = nullptr) {
  const int i = c % g.nx, j = c / g.nx;
#pragma unroll
  for (int q = 0; q < 4; ++q) phi[q] = R(0);
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    int cell[5];
    bool refl[5] = {false, false, false, false, false};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      if (WALLS && t != 2) {
        const size_t at = (size_t)(d * 4 + (t < 2 ? t : t - 1)) * g.nc + c;
        cell[t] = Vw->wsrc[at];
        refl[t] = Vw->wrefl[at] != 0;
      } else {
        cell[t] = d == 0 ? j * g.nx + nb(i + t - 2, g.nx, g.bcx) : nb(j + t - 2, g.ny, g.bcy) * g.nx + i;
      }
    }
    R q[5][4];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
#pragma unroll
      for (int m = 0; m < 4; ++m) q[t][m] = (R)U[(size_t)m * g.nc + cell[t]];
      if (WALLS && refl[t]) q[t][1 + d] = -q[t][1 + d];
    }
    R Lm[4], Rm[4], Lp[4], Rp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      Lm[m] = cweno_face(q[0][m], q[1][m], q[2][m], epsw);  // right face of cell -1
      Rm[m] = cweno_face(q[3][m], q[2][m], q[1][m], epsw);  // left face of cell 0
      Lp[m] = cweno_face(q[1][m], q[2][m], q[3][m], epsw);  // right face of cell 0
      Rp[m] = cweno_face(q[4][m], q[3][m], q[2][m], epsw);  // left face of cell +1
    }
    R FLm[4], FRm[4], FLp[4], FRp[4], aLm, aRm, aLp, aRp;
    euler_phys(Lm, d, FLm, aLm);
    euler_phys(Rm, d, FRm, aRm);
    euler_phys(Lp, d, FLp, aLp);
    euler_phys(Rp, d, FRp, aRp);
    const R am = rmax(aLm, aRm), ap = rmax(aLp, aRp);
    const R ih = R(1) / (R)(d == 0 ? g.dx : g.dy);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      R Fm = R(0.5) * (FLm[m] + FRm[m]) - R(0.5) * am * (Rm[m] - Lm[m]);
      R Fp = R(0.5) * (FLp[m] + FRp[m]) - R(0.5) * ap * (Rp[m] - Lp[m]);
      if (omask & (1 << (2 * d))) Fm = ovr[2 * d][m];
      if (omask & (2 << (2 * d))) Fp = ovr[2 * d + 1][m];
      phi[m] += (Fp - Fm) * ih;
    }
  }
}

// U^(i)(c) = U^n(c) - sum_j coef_j Phi_j(c) for a fluid cell, after storing
// Phi_{i-1}(c) when requested (Eqs. RKEuler, RKEuler_2).
template <typename R, bool WALLS = false>
ESBGK_DEV void euler_cell(const StageArgs& A, const View& V, int c, double (&Uc)[4], const R (*ovr)[4] = nullptr,
                          int omask = 0) {
  const size_t nc = V.g.nc;
  if (A.phi_store >= 0) {
    R phi[4];
    euler_phi_cell<R, WALLS>(V.g, A.U_prev, c, pick<R>(V.m.eps_w, V.m.feps_w), phi, ovr, omask, &V);
#pragma unroll
    for (int m = 0; m < 4; ++m) A.Phi[((size_t)A.phi_store * 4 + m) * nc + c] = (double)phi[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double u = A.Un[m * nc + c];
    for (int jj = 0; jj < A.nphi; ++jj) u -= A.phi_coef[jj] * A.Phi[((size_t)jj * 4 + m) * nc + c];
    A.U_out[m * nc + c] = u;
    Uc[m] = u;
  }
}

// Moments w sum F (1, v_x, v_y, |v|^2/2) of the kinetic numerical flux
// through the face between cells a (low side) and b (high side) along axis d
// (am below a, bp above b): F = v_d times the upwind CWENO3 face value, the
// right face of a for v_d > 0 and the left face of b for v_d < 0 -- the same
// face values, from the same arguments, as the kinetic cell's transport.
// Warp-wide, one node per lane and iteration; every lane returns the sums.
template <typename S>
ESBGK_DEV void face_flux_moments(const S* __restrict__ f, const Geo& g, const Model& mdl, int am, int a, int b,
                                 int bp, int d, int lane, typename Real<S>::T (&G)[4]) {
  using R = typename Real<S>::T;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv), epsw = pick<R>(mdl.eps_w, mdl.feps_w);
  const size_t n = g.nvv;
  const S *fam = f + (size_t)am * n, *fa = f + (size_t)a * n, *fb = f + (size_t)b * n, *fbp = f + (size_t)bp * n;
  R s[4] = {R(0), R(0), R(0), R(0)};
  NodeIter<R> it(lane, g.nv, v0, dv);
#pragma unroll 1
  for (; it.k < g.nvv; it.next()) {
    const unsigned k = it.k;
    const R vx = it.vx(), vy = it.vy(), vn = d == 0 ? vx : vy;
    const R q = vn > R(0) ? cweno_face(ld(fam + k), ld(fa + k), ld(fb + k), epsw)
                          : cweno_face(ld(fbp + k), ld(fb + k), ld(fa + k), epsw);
    const R F = vn * q;
    s[0] += F;
    s[1] += F * vx;
    s[2] += F * vy;
    s[3] += F * R(0.5) * (vx * vx + vy * vy);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) G[m] = warp_sum(s[m]) * pick<R>(g.w, g.fw);
}

// Conservative interface of buffer cell c (StageArgs::iface): the kinetic
// flux moments at each face of c shared with a kinetic cell, computed from
// f_src (f of the previous stage; filled in buffer cells, so every stencil
// cell holds f).  Returns the face mask of euler_phi_cell.  Warp-wide.
template <typename S>
ESBGK_DEV int interface_fluxes(const StageArgs& A, const View& V, int c, int lane,
                               typename Real<S>::T (&ovr)[4][4]) {
  const Geo& g = V.g;
  const S* f = (const S*)A.f_src;
  const int i = c % g.nx, j = c / g.nx;
  int mask = 0;
#pragma unroll 1
  for (int face = 0; face < 4; ++face) {
    const int d = face >> 1, up = face & 1;  // axis; the face above (+1/2) or below (-1/2) c
    auto cell = [&](int off) {
      return d == 0 ? j * g.nx + nb(i + off, g.nx, g.bcx) : nb(j + off, g.ny, g.bcy) * g.nx + i;
    };
    const int other = cell(up ? 1 : -1);
    if (other == c || !V.flags[other]) continue;
    // the face between a (low side) and b (high side)
    const int lo = up ? 0 : -1;
    face_flux_moments<S>(f, g, V.m, cell(lo - 1), cell(lo), cell(lo + 1), cell(lo + 2), d, lane, ovr[face]);
    mask |= 1 << face;
  }
  return mask;
}

// Primitive variables of U (Sec. 2): u = m/rho, T = (E - rho |u|^2/2)/rho.
ESBGK_DEV void prim_of(const double (&U)[4], double& rho, double& ux, double& uy, double& T) {
  rho = U[0];
  const double ir = 1.0 / rho;
  ux = U[1] * ir;
  uy = U[2] * ir;
  T = (U[3] - 0.5 * rho * (ux * ux + uy * uy)) * ir;
}

// Reference velocity for the moment sums of cell c: the mean velocity held
// in U (0 when U is not usable).
// Only a centring point for the sums: computed in the arithmetic type.
template <typename R>
ESBGK_DEV void ref_velocity(const double* U, size_t nc, int c, R& u0x, R& u0y) {
  u0x = R(0);
  u0y = R(0);
  if (!U) return;
  const R rho = R(U[c]);
  if (rho > R(0)) {
    const R ir = R(1) / rho;
    u0x = R(U[nc + c]) * ir;
    u0y = R(U[2 * nc + c]) * ir;
  }
}

// Conserved variables (float64) from the raw moment sums about u0.
template <typename R>
ESBGK_DEV void cons_from_sums(const R (&m)[6], R u0x, R u0y, double w, double (&U)[4]) {
  const double m0 = w * (double)m[0], m1 = w * (double)m[1], m2 = w * (double)m[2];
  const double ux = u0x, uy = u0y;
  U[0] = m0;
  U[1] = m1 + ux * m0;
  U[2] = m2 + uy * m0;
  U[3] = 0.5 * w * ((double)m[3] + (double)m[5]) + ux * m1 + uy * m2 + 0.5 * (ux * ux + uy * uy) * m0;
}

// ---------------------------------------------------------------------------
// Kinetic cell of a stage (or of the final combination), one warp.
// Loads of one batch are issued together before any store of the batch:
// the compiler cannot prove that the output arrays do not alias the inputs,
// so without this every store would wait for the previous node's loads.
#ifndef ESBGK_BATCH
#define ESBGK_BATCH 2
#endif
constexpr int kBatch = ESBGK_BATCH;

// The seven values of the transport stencil of node k (centre, then upwind,
// downwind and far-upwind neighbours along x and along y for the sign of v).
template <typename S, typename R>
ESBGK_DEV void stencil_load(const S* __restrict__ f, unsigned o0, const unsigned (&o)[8], unsigned k, bool px,
                            bool py, R (&q)[7]) {
  q[0] = ld(f + o0 + k);
  q[1] = ld(f + (px ? o[1] : o[2]) + k);
  q[2] = ld(f + (px ? o[2] : o[1]) + k);
  q[3] = ld(f + (px ? o[0] : o[3]) + k);
  q[4] = ld(f + (py ? o[5] : o[6]) + k);
  q[5] = ld(f + (py ? o[6] : o[5]) + k);
  q[6] = ld(f + (py ? o[4] : o[7]) + k);
}

// The same with solid obstacles: o[8] and the reflection bits rb come from the
// stencil maps (stencil_walls); a reflected value is read at the mirrored node
// (v_x -> -v_x: kxm, v_y -> -v_y: kym).
template <typename S, typename R>
ESBGK_DEV void stencil_load_walls(const S* __restrict__ f, unsigned o0, const unsigned (&o)[8], unsigned rb,
                                  unsigned k, unsigned kxm, unsigned kym, bool px, bool py, R (&q)[7]) {
  auto val = [&](int e) {
    const unsigned kk = (rb >> e) & 1u ? (e < 4 ? kxm : kym) : k;
    return ld(f + o[e] + kk);
  };
  q[0] = ld(f + o0 + k);
  q[1] = val(px ? 1 : 2);
  q[2] = val(px ? 2 : 1);
  q[3] = val(px ? 0 : 3);
  q[4] = val(py ? 5 : 6);
  q[5] = val(py ? 6 : 5);
  q[6] = val(py ? 4 : 7);
}

// Element offsets and reflection bits of the stencil of cell c with solid
// obstacles (View::wsrc, wrefl; the order of stencil_offsets).
ESBGK_DEV void stencil_walls(const View& V, int c, unsigned (&o)[8], unsigned& rb) {
  rb = 0u;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const size_t at = (size_t)e * V.g.nc + c;
    o[e] = (unsigned)V.wsrc[at] * (unsigned)V.g.nvv;
    rb |= (unsigned)(V.wrefl[at] != 0) << e;
  }
}

// L(f) at a node from its stencil values: upwind (Lax-Friedrichs with |v|)
// flux of CWENO3 face values; L_x = |v_x| (F(face away from the upwind
// neighbour) - F(face toward it)) / dx, the same along y.
template <typename R>
ESBGK_DEV R transport_of(const R (&q)[7], R vx, R vy, R idx, R idy, R epsw) {
  const R Lx = rabs(vx) * (cweno_face(q[1], q[0], q[2], epsw) - cweno_face(q[3], q[1], q[0], epsw)) * idx;
  const R Ly = rabs(vy) * (cweno_face(q[4], q[0], q[5], epsw) - cweno_face(q[6], q[4], q[0], epsw)) * idy;
  return Lx + Ly;
}

// ||f - M_hat[f]||_{L1_v} of the cell whose node values are in sf and whose raw
// moment sums about u0 are m (Eq. eqKintoFluid1), one warp; -1 if the
// moments are not realizable.
template <typename R, int W, int L = 32>
ESBGK_DEV R l1_deviation(const Geo& g, int lane, const R (&m)[6], R u0x, R u0y, const R* sf,
                         unsigned mask = 0xffffffffu) {
  CellPar<R> P;
  if (!es_params<R>(m, u0x, u0y, pick<R>(g.w, g.fw), R(0), R(0), false, P) || !project<R, W, L>(g, lane, P, mask))
    return R(-1);
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  R s = R(0);
  NodeIter<R> it(lane * W, g.nv, v0, dv, L * W);
  if constexpr (std::is_same<R, float>::value && W % 2 == 0) {
    for (; it.k < g.nvv; it.next()) {
      const GhatRow row = ghat_row(P, it.vy() - P.uy);
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float cxa = it.vx() + R(j) * dv - P.ux;
        const float2 d = __ffma2_rn(ghat_pair(P, row, make_float2(cxa, cxa + dv)), splat2(-1.0f),
                                    *reinterpret_cast<const float2*>(sf + it.k + j));
        s += rabs(d.x) + rabs(d.y);
      }
    }
  } else {
    for (; it.k < g.nvv; it.next())
#pragma unroll
      for (int j = 0; j < W; ++j) s += rabs(sf[it.k + j] - ghat(P, it.vx() + R(j) * dv - P.ux, it.vy() - P.uy));
  }
  return group_sum<L>(s, mask) * pick<R>(g.w, g.fw);
}

// Flag values of each compile-time stage shape (StageMode).
template <int M>
struct ModeT {  // kGeneric: unused values
  static constexpr bool relax = false, base_src = false, acc_src = false;
  static constexpr int nacc = 0;
};
template <>
struct ModeT<kFirstRelax2> {
  static constexpr bool relax = true, base_src = true, acc_src = true;
  static constexpr int nacc = 2;
};
template <>
struct ModeT<kLoadedRelax1> {
  static constexpr bool relax = true, base_src = false, acc_src = false;
  static constexpr int nacc = 1;
};
template <>
struct ModeT<kFinal> {
  static constexpr bool relax = false, base_src = false, acc_src = false;
  static constexpr int nacc = 0;
};
template <>
struct ModeT<kFirstRelax0> {
  static constexpr bool relax = true, base_src = true, acc_src = false;
  static constexpr int nacc = 0;
};


// Kinetic cell of a stage (or of the final combination), one warp.
// Pass 1 forms f* = star_base + star_cL L(f_src) and its moments, keeps f* in
// the warp's shared memory and writes the partial accumulators
// acc_in + acc_cL L to the accumulator outputs; pass 3 adds acc_cQ Q to them
// (a re-read that stays in L2) and writes f.  Without a collision term
// (the final combination) everything is written in pass 1.
template <typename S, int M, bool WALLS = false>
ESBGK_DEV void kinetic_cell(const StageArgs& A, const View& V, int c, int lane, typename Real<S>::T* sfs) {
  using R = typename Real<S>::T;
  constexpr bool GEN = M == kGeneric;
  const Geo& g = V.g;
  const unsigned o0 = (unsigned)c * (unsigned)g.nvv;
  unsigned o[8], rb = 0u;
  if (WALLS)
    stencil_walls(V, c, o, rb);
  else
    stencil_offsets(g, c, o);
  const S* fsrc = (const S*)A.f_src;
  const S* sbase = (const S*)A.star_base;
  const bool has_src = GEN ? fsrc != nullptr : true;
  const bool base_is_src = GEN ? A.star_base == A.f_src : ModeT<M>::base_src;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  const R idx = pick<R>(1.0 / g.dx, g.fidx), idy = pick<R>(1.0 / g.dy, g.fidy);
  const R epsw = pick<R>(V.m.eps_w, V.m.feps_w), cL = pick<R>(A.star_cL, A.f_star_cL);
  const bool relax = GEN ? A.h_coef > 0.0 : ModeT<M>::relax;
  const bool proj = GEN ? (relax || A.need_q) : ModeT<M>::relax;
  S* fout = (S*)A.f_out;
  const bool has_out = GEN ? fout != nullptr : true;
  const int nacc = GEN ? A.nacc : ModeT<M>::nacc;
  const S* ain[3];
  S* aout[3];
  bool asrc[3];
  R aL[3], aQ[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    ain[t] = t < nacc ? (const S*)A.acc_in[t] : nullptr;
    aout[t] = t < nacc ? (S*)A.acc_out[t] : nullptr;
    asrc[t] = t < nacc && (GEN ? ain[t] == fsrc : ModeT<M>::acc_src);
    aL[t] = t < nacc ? pick<R>(A.acc_cL[t], A.f_acc_cL[t]) : R(0);
    aQ[t] = t < nacc ? pick<R>(A.acc_cQ[t], A.f_acc_cQ[t]) : R(0);
  }
  R u0x, u0y;
  ref_velocity(A.U_prev, g.nc, c, u0x, u0y);

  // pass 1: transport of the previous stage, f*, moments of f*
  R m[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) m[n] = R(0);
  NodeIter<R> it(lane, g.nv, v0, dv);
  while (it.k < g.nvv) {
    int kk[kBatch];
    bool val[kBatch];
    R vx[kBatch], vy[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      kk[u] = it.k;
      val[u] = it.k < g.nvv;
      vx[u] = it.vx();
      vy[u] = it.vy();
      it.next();
    }
    R q[kBatch][7], bs[kBatch], ai[kBatch][3];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (!val[u]) continue;
      const int k = kk[u];
      if (has_src) {
        if (WALLS) {
          const unsigned ky = (unsigned)k / (unsigned)g.nv, kx = (unsigned)k - ky * (unsigned)g.nv;
          const unsigned kxm = k + g.nv - 1u - 2u * kx, kym = k + (g.nv - 1u - 2u * ky) * (unsigned)g.nv;
          stencil_load_walls<S, R>(fsrc, o0, o, rb, k, kxm, kym, vx[u] > R(0), vy[u] > R(0), q[u]);
        } else {
          stencil_load<S, R>(fsrc, o0, o, k, vx[u] > R(0), vy[u] > R(0), q[u]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 7; ++e) q[u][e] = R(0);
      }
      bs[u] = base_is_src ? q[u][0] : ld(sbase + o0 + k);
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t < nacc) ai[u][t] = asrc[t] ? q[u][0] : ld(ain[t] + o0 + k);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (!val[u]) continue;
      const int k = kk[u];
      const R L = has_src ? transport_of(q[u], vx[u], vy[u], idx, idy, epsw) : R(0);
      const R fs = bs[u] + cL * L;
      if (proj) {
        sfs[k] = fs;
      } else {
        // no collision term: f = f*, Q = 0
        if (has_out) st(fout + o0 + k, fs);
        if (A.l1_out) sfs[k] = fs;
      }
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t < nacc) st(aout[t] + o0 + k, ai[u][t] + aL[t] * L);
      const R cx = vx[u] - u0x, cy = vy[u] - u0y;
      m[0] += fs;
      m[1] += cx * fs;
      m[2] += cy * fs;
      m[3] += cx * cx * fs;
      m[4] += cx * cy * fs;
      m[5] += cy * cy * fs;
    }
  }
#pragma unroll
  for (int n = 0; n < 6; ++n) m[n] = warp_sum(m[n]);
  if (lane == 0) {  // U of the cell (float64), written by one lane
    double Uc[4];
    cons_from_sums(m, u0x, u0y, g.w, Uc);
    const size_t nc = g.nc;
#pragma unroll
    for (int q = 0; q < 4; ++q) A.U_out[q * nc + c] = A.kin_u_moments ? Uc[q] : A.Un[q * nc + c];
  }
  if (!proj) {
    if (A.l1_out) {
      __syncwarp();
      const R l1 = l1_deviation<R, 1>(g, lane, m, u0x, u0y, sfs);
      if (lane == 0) {
        if (l1 < R(0)) report_error(V.err, kErrNonRealizable, c);
        A.l1_out[c] = (double)l1;
      }
    }
    return;
  }

  // collision rate nu = tau / eps (tau * rho with the density model, rho of
  // f*) and h = dt a_ii nu in the arithmetic type
  const R tau = pick<R>(V.m.tau, V.m.ftau) * (V.m.tau_rho ? pick<R>(g.w, g.fw) * m[0] : R(1));
  const R nu = tau / R(V.eps[c]), h = pick<R>(A.h_coef, A.f_h_coef) * nu;
  CellPar<R> P;
  bool ok = es_params<R>(m, u0x, u0y, pick<R>(g.w, g.fw), pick<R>(V.m.beta, V.m.fbeta), h, relax, P);
  if (ok) ok = project<R>(g, lane, P);
  if (!ok && lane == 0) report_error(V.err, kErrNonRealizable, c);

  // pass 3: G_hat, implicit relaxation, Q, accumulators, outputs
  const R inv1h = R(1) / (R(1) + h);
  NodeIter<R> jt(lane, g.nv, v0, dv);
  while (jt.k < g.nvv) {
    int kk[kBatch];
    bool val[kBatch];
    R vx[kBatch], vy[kBatch], pa[kBatch][3], fs[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      kk[u] = jt.k;
      val[u] = jt.k < g.nvv;
      vx[u] = jt.vx();
      vy[u] = jt.vy();
      jt.next();
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (!val[u]) continue;
      fs[u] = sfs[kk[u]];
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t < nacc) pa[u][t] = ldc(aout[t] + o0 + kk[u]);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (!val[u]) continue;
      const int k = kk[u];
      R fnew = fs[u], Q = R(0);
      if (ok) {
        const R Gh = ghat(P, vx[u] - P.ux, vy[u] - P.uy);
        // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f) = nu (G_hat - f*)/(1 + h)
        if (relax) fnew = (fs[u] + h * Gh) * inv1h;
        Q = nu * (Gh - fs[u]) * inv1h;
      }
      if (has_out) st(fout + o0 + k, fnew);
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (t < nacc) st(aout[t] + o0 + k, pa[u][t] + aQ[t] * Q);
    }
  }
}

// Moment sums of the paired FP32 vector forms: compensation compiled out, or
// chosen at run time by Model::comp_moments.
enum : int { kSumsPlain = 0, kSumsRunTime = 1 };

// Vector form of kinetic_cell for a specialised launch mode: each lane takes W
// consecutive nodes of one velocity row per iteration (one vector load per
// stencil array instead of W), which needs N_v divisible by W (a group never
// straddles a row end) and 16-byte aligned arrays.  SX (N_v/2 not a multiple
// of W): the group holding v_x = 0 has nodes moving either way; it loads the
// fourth x-neighbour too and takes each node's upwind stencil.
// L lanes per cell: 32 (the warp) or 16 (a half-warp; mask: its lanes; lane:
// the index within the half) -- two cells per warp for small velocity grids.
// WALLS: solid obstacles (the stencil maps of View; no group straddles v_x = 0).
// SUMS: how the paired FP32 forms sum the moments -- kSumsPlain compiles the
// compensation out (no compensation state live in the node loop),
// kSumsRunTime follows Model::comp_moments.
template <typename S, int M, int W, int L = 32, bool SX = false, bool WALLS = false, int SUMS = kSumsRunTime>
ESBGK_DEV void kinetic_cell_vec(const StageArgs& A, const View& V, int c, int lane, typename Real<S>::T* sfs,
                                unsigned mask = 0xffffffffu) {
  static_assert(!(WALLS && SX), "the wall form has no straddling group");
  using R = typename Real<S>::T;
  using IO = VecIO<S, W>;
  using SM = SmemVec<R, W>;
  using MT = ModeT<M>;
  const Geo& g = V.g;
  const unsigned o0 = (unsigned)c * (unsigned)g.nvv;
  unsigned o[8];
  unsigned rb = 0u;  // reflection bits of the stencil positions (solid obstacles)
  if constexpr (WALLS)
    stencil_walls(V, c, o, rb);
  else
    stencil_offsets(g, c, o);
  const S* fsrc = (const S*)A.f_src;
  const S* sbase = (const S*)A.star_base;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  const R idx = pick<R>(1.0 / g.dx, g.fidx), idy = pick<R>(1.0 / g.dy, g.fidy);
  const R epsw = pick<R>(V.m.eps_w, V.m.feps_w), cL = pick<R>(A.star_cL, A.f_star_cL);
  constexpr bool relax = MT::relax;
  constexpr int nacc = MT::nacc;
  // f* and every accumulator start from f_src (the first relaxed stage): the
  // partial accumulators f_src + aL L are not written in pass 1; pass 3
  // rebuilds them from f* = f_src + cL L as f_src + (aL / cL)(f* - f_src)
  // (the same value up to the rounding of f*; cL != 0 by the host's choice
  // of this mode)
  constexpr bool kRebuild = relax && MT::base_src && MT::acc_src && nacc > 0;
  S* fout = (S*)A.f_out;
  const S* ain[nacc > 0 ? nacc : 1];
  S* aout[nacc > 0 ? nacc : 1];
  R aL[nacc > 0 ? nacc : 1], aQ[nacc > 0 ? nacc : 1];
#pragma unroll
  for (int t = 0; t < nacc; ++t) {
    ain[t] = (const S*)A.acc_in[t];
    aout[t] = (S*)A.acc_out[t];
    aL[t] = pick<R>(A.acc_cL[t], A.f_acc_cL[t]);
    aQ[t] = pick<R>(A.acc_cQ[t], A.f_acc_cQ[t]);
  }
  R u0x, u0y;
  ref_velocity(A.U_prev, g.nc, c, u0x, u0y);
  // random key of this launch for the stochastic rounding of bf16 stores
  const uint32_t s0 = A.seed ? mix32(*A.seed * 0x632be5abu + A.sid) : 0u;

  // column of the group that straddles v_x = 0 (none: -1)
  const int half_nv = g.nv >> 1, kz = SX ? half_nv - half_nv % W : -1;

  // pass 1: transport of the previous stage, f*, moments of f*
  // (FP32 arithmetic with an even group: pairs of nodes on paired instructions)
  // FP32 moments: paired partial sums per lane (short runs), a butterfly over
  // the lanes.  With compensated sums (Model::comp_moments) the paired sums
  // go every kFlush groups into a Neumaier-compensated accumulator per lane
  // (m, mc) and the lanes are added with error-free two-sums.
  constexpr bool kPacked = std::is_same<R, float>::value && W % 2 == 0;
  const bool kComp = kPacked && SUMS == kSumsRunTime && V.m.comp_moments;
  constexpr int kFlush = 4;
  R m[6];
  float2 m2[6];
  float mc[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    m[n] = R(0);
    m2[n] = splat2(0.0f);
    mc[n] = 0.0f;
  }
  int blk = 0;
  NodeIter<R> it(lane * W, g.nv, v0, dv, L * W);
#pragma unroll 1
  for (; it.k < g.nvv; it.next()) {
    const unsigned k = it.k;
    const R vx0 = it.vx(), vy = it.vy();
    const bool px = vx0 > R(0), py = vy > R(0);
    R q0[W], ux[W], dx[W], fx[W], uy[W], dy[W], fy[W], bs[W], ai[nacc > 0 ? nacc : 1][W];
    // the group's values at stencil position e; a mirror image across a wall
    // face (reflection bit set) is read at the mirrored nodes: along x the
    // node order reversed within the row (the mirrored group starts at
    // N_v - W - k_x, aligned because W divides N_v), along y the mirrored row
    // (oe: the position's cell offset, re: its reflection bit, xa: along x)
    auto ldn = [&](unsigned oe, bool re, bool xa, R (&v)[W]) {
      if constexpr (WALLS) {
        if (re) {
          const unsigned kxg = (unsigned)it.kx, kyg = (unsigned)it.fy, nvu = (unsigned)g.nv;
          if (xa) {
            R t[W];
            IO::ld(fsrc + oe + kyg * nvu + (nvu - (unsigned)W - kxg), t);
#pragma unroll
            for (int j = 0; j < W; ++j) v[j] = t[W - 1 - j];
          } else {
            IO::ld(fsrc + oe + (nvu - 1u - kyg) * nvu + kxg, v);
          }
          return;
        }
      }
      IO::ld(fsrc + oe + k, v);
    };
    auto bit = [&](int e) { return WALLS && ((rb >> e) & 1u); };
    IO::ld(fsrc + o0 + k, q0);
    ldn(px ? o[1] : o[2], px ? bit(1) : bit(2), true, ux);
    ldn(px ? o[2] : o[1], px ? bit(2) : bit(1), true, dx);
    ldn(px ? o[0] : o[3], px ? bit(0) : bit(3), true, fx);
    if (SX && it.kx == kz) {
      // first node v_x < 0 (loaded above), the last ones v_x > 0: upwind is
      // the left neighbour, downwind the right one, far side two to the left
      R l2[W];
      IO::ld(fsrc + o[0] + k, l2);
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (vx0 + R(j) * dv > R(0)) {
          const R t = ux[j];
          ux[j] = dx[j];
          dx[j] = t;
          fx[j] = l2[j];
        }
    }
    ldn(py ? o[5] : o[6], py ? bit(5) : bit(6), false, uy);
    ldn(py ? o[6] : o[5], py ? bit(6) : bit(5), false, dy);
    ldn(py ? o[4] : o[7], py ? bit(4) : bit(7), false, fy);
    if (MT::base_src) {
#pragma unroll
      for (int j = 0; j < W; ++j) bs[j] = q0[j];
    } else {
      IO::ld(sbase + o0 + k, bs);
    }
#pragma unroll
    for (int t = 0; t < nacc; ++t) {
      if (MT::acc_src) {
#pragma unroll
        for (int j = 0; j < W; ++j) ai[t][j] = q0[j];
      } else {
        IO::ld(ain[t] + o0 + k, ai[t]);
      }
    }
    R fs[W], pa[nacc > 0 ? nacc : 1][W];
    const R ay = rabs(vy) * idy;
    if constexpr (kPacked) {
      // nodes j, j + 1 together on the paired FP32 instructions
      const float2 e2 = splat2(epsw), m1 = splat2(-1.0f);
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float2 Q = make_float2(q0[j], q0[j + 1]);
        const float2 Ux = make_float2(ux[j], ux[j + 1]), Uy = make_float2(uy[j], uy[j + 1]);
        const float2 dFx = cweno_dface2(make_float2(fx[j], fx[j + 1]), Ux, Q, make_float2(dx[j], dx[j + 1]), e2);
        const float2 dFy = cweno_dface2(make_float2(fy[j], fy[j + 1]), Uy, Q, make_float2(dy[j], dy[j + 1]), e2);
        const float vxa = vx0 + R(j) * dv, vxb = vxa + dv;
        const float2 Lf = __ffma2_rn(make_float2(rabs(vxa) * idx, rabs(vxb) * idx), dFx, __fmul2_rn(splat2(ay), dFy));
        const float2 F = __ffma2_rn(splat2(cL), Lf, make_float2(bs[j], bs[j + 1]));
        fs[j] = F.x;
        fs[j + 1] = F.y;
#pragma unroll
        for (int t = 0; t < (kRebuild ? 0 : nacc); ++t) {
          const float2 Pa = __ffma2_rn(splat2(aL[t]), Lf, make_float2(ai[t][j], ai[t][j + 1]));
          pa[t][j] = Pa.x;
          pa[t][j + 1] = Pa.y;
        }
        const float2 cx = make_float2(vxa - u0x, vxb - u0x), cy = splat2(vy - u0y);
        const float2 xf = __fmul2_rn(cx, F), yf = __fmul2_rn(cy, F);
        m2[0] = __fadd2_rn(m2[0], F);
        m2[1] = __fadd2_rn(m2[1], xf);
        m2[2] = __fadd2_rn(m2[2], yf);
        m2[3] = __ffma2_rn(cx, xf, m2[3]);
        m2[4] = __ffma2_rn(cy, xf, m2[4]);
        m2[5] = __ffma2_rn(cy, yf, m2[5]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const R vx = vx0 + R(j) * dv;
        const R Lx = rabs(vx) * idx * (cweno_face(ux[j], q0[j], dx[j], epsw) - cweno_face(fx[j], ux[j], q0[j], epsw));
        const R Ly = ay * (cweno_face(uy[j], q0[j], dy[j], epsw) - cweno_face(fy[j], uy[j], q0[j], epsw));
        const R Lf = Lx + Ly;
        fs[j] = bs[j] + cL * Lf;
#pragma unroll
        for (int t = 0; t < (kRebuild ? 0 : nacc); ++t) pa[t][j] = ai[t][j] + aL[t] * Lf;
        const R cx = vx - u0x, cy = vy - u0y;
        m[0] += fs[j];
        m[1] += cx * fs[j];
        m[2] += cy * fs[j];
        m[3] += cx * cx * fs[j];
        m[4] += cx * cy * fs[j];
        m[5] += cy * cy * fs[j];
      }
    }
    const uint32_t kb = s0 + ((o0 + k) << 3);  // distinct per group and stored array
    if (relax) {
      SM::st(sfs + k, fs);
    } else {
      IO::st_sr(fout + o0 + k, fs, kb);
      if (A.l1_out) SM::st(sfs + k, fs);
    }
#pragma unroll
    for (int t = 0; t < (kRebuild ? 0 : nacc); ++t) IO::st_sr(aout[t] + o0 + k, pa[t], kb + 1 + t);
    if constexpr (kPacked) {
      if (kComp && ++blk == kFlush) {
        blk = 0;
#pragma unroll
        for (int n = 0; n < 6; ++n) {
          comp_add(m[n], mc[n], m2[n].x + m2[n].y);
          m2[n] = splat2(0.0f);
        }
      }
    }
  }
  if constexpr (kPacked) {
    if (kComp) {
#pragma unroll
      for (int n = 0; n < 6; ++n) {
        comp_add(m[n], mc[n], m2[n].x + m2[n].y);
        m[n] = group_sum_comp<L>(m[n], mc[n], mask);
      }
    } else {
#pragma unroll
      for (int n = 0; n < 6; ++n) m[n] = group_sum<L>(m2[n].x + m2[n].y, mask);
    }
  } else {
#pragma unroll
    for (int n = 0; n < 6; ++n) m[n] = group_sum<L>(m[n], mask);
  }
  if (lane == 0) {  // U of the cell (float64), written by one lane
    double Uc[4];
    cons_from_sums(m, u0x, u0y, g.w, Uc);
    const size_t nc = g.nc;
#pragma unroll
    for (int q = 0; q < 4; ++q) A.U_out[q * nc + c] = A.kin_u_moments ? Uc[q] : A.Un[q * nc + c];
  }
  if (!relax) {
    if (A.l1_out) {
      __syncwarp(mask);
      const R l1 = l1_deviation<R, W, L>(g, lane, m, u0x, u0y, sfs, mask);
      if (lane == 0) {
        if (l1 < R(0)) report_error(V.err, kErrNonRealizable, c);
        A.l1_out[c] = (double)l1;
      }
    }
    return;
  }

  // collision rate nu = tau / eps (tau * rho with the density model, rho of
  // f*) and h = dt a_ii nu in the arithmetic type
  const R tau = pick<R>(V.m.tau, V.m.ftau) * (V.m.tau_rho ? pick<R>(g.w, g.fw) * m[0] : R(1));
  const R nu = tau / R(V.eps[c]), h = pick<R>(A.h_coef, A.f_h_coef) * nu;
  CellPar<R> P;
  bool ok = es_params<R>(m, u0x, u0y, pick<R>(g.w, g.fw), pick<R>(V.m.beta, V.m.fbeta), h, true, P);
  if (ok) ok = project<R, W, L>(g, lane, P, mask);
  if (!ok && lane == 0) report_error(V.err, kErrNonRealizable, c);

  // pass 3: G_hat, implicit relaxation, Q, accumulators, outputs
  const R inv1h = R(1) / (R(1) + h);
  R rL[nacc > 0 ? nacc : 1];  // aL / cL of the rebuilt accumulators
#pragma unroll
  for (int t = 0; t < nacc; ++t) rL[t] = kRebuild ? aL[t] / cL : R(0);
  NodeIter<R> jt(lane * W, g.nv, v0, dv, L * W);
#pragma unroll 1
  for (; jt.k < g.nvv; jt.next()) {
    const unsigned k = jt.k;
    R fs[W], pa[nacc > 0 ? nacc : 1][W], fn[W];
    SM::ld(sfs + k, fs);
    if constexpr (kRebuild) {
      R q[W];  // f_src, read in pass 1 and still in L2
      IO::ld(fsrc + o0 + k, q);
      if constexpr (kPacked) {
#pragma unroll
        for (int j = 0; j < W; j += 2) {
          const float2 Q0 = make_float2(q[j], q[j + 1]);
          const float2 D = __ffma2_rn(Q0, splat2(-1.0f), make_float2(fs[j], fs[j + 1]));
#pragma unroll
          for (int t = 0; t < nacc; ++t) {
            const float2 Pa = __ffma2_rn(splat2(rL[t]), D, Q0);
            pa[t][j] = Pa.x;
            pa[t][j + 1] = Pa.y;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < nacc; ++t)
#pragma unroll
          for (int j = 0; j < W; ++j) pa[t][j] = q[j] + rL[t] * (fs[j] - q[j]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < nacc; ++t) IO::ldc(aout[t] + o0 + k, pa[t]);
    }
    const R cy = jt.vy() - P.uy, cx0 = jt.vx() - P.ux;
    if constexpr (kPacked) {
      // pairs of nodes on the paired FP32 instructions
      const GhatRow row = ghat_row(P, cy);
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float2 F = make_float2(fs[j], fs[j + 1]);
        float2 Fn = F, Q = splat2(0.0f);
        if (ok) {
          const float cxa = cx0 + R(j) * dv;
          const float2 Gh = ghat_pair(P, row, make_float2(cxa, cxa + dv));
          // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f) = nu (G_hat - f*)/(1 + h)
          Fn = __fmul2_rn(__ffma2_rn(splat2(h), Gh, F), splat2(inv1h));
          Q = __fmul2_rn(splat2(nu * inv1h), __ffma2_rn(F, splat2(-1.0f), Gh));
        }
        fn[j] = Fn.x;
        fn[j + 1] = Fn.y;
#pragma unroll
        for (int t = 0; t < nacc; ++t) {
          const float2 Pa = __ffma2_rn(splat2(aQ[t]), Q, make_float2(pa[t][j], pa[t][j + 1]));
          pa[t][j] = Pa.x;
          pa[t][j + 1] = Pa.y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < W; ++j) {
        R Q = R(0);
        fn[j] = fs[j];
        if (ok) {
          const R Gh = ghat(P, cx0 + R(j) * dv, cy);
          // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f) = nu (G_hat - f*)/(1 + h)
          fn[j] = (fs[j] + h * Gh) * inv1h;
          Q = nu * (Gh - fs[j]) * inv1h;
        }
#pragma unroll
        for (int t = 0; t < nacc; ++t) pa[t][j] += aQ[t] * Q;
      }
    }
    const uint32_t kb = s0 + ((o0 + k) << 3);
    IO::st_sr(fout + o0 + k, fn, kb);
#pragma unroll
    for (int t = 0; t < nacc; ++t) IO::st_sr(aout[t] + o0 + k, pa[t], kb + 4 + t);
  }
}

// Writes f := M_hat[U] (the discrete Maxwellian, Eq. Coupling_FluKin) into
// cell c of f, one warp.  Returns false for a non-realizable U.
// W > 1: groups of W consecutive nodes of a row (N_v divisible by W, f 16-byte
// aligned), one vector store per group.
template <typename S, int W = 1>
ESBGK_DEV bool fill_maxwell(S* f, const Geo& g, int c, int lane, const double (&U)[4], uint32_t key = 0u) {
  using R = typename Real<S>::T;
  double rho, ux, uy, T;
  prim_of(U, rho, ux, uy, T);
  CellPar<R> P;
  if (!maxwell_params<R>(rho, ux, uy, T, P) || !project<R, W>(g, lane, P)) return false;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  const size_t o0 = (size_t)c * g.nvv;
  NodeIter<R> it(lane * W, g.nv, v0, dv, 32 * W);
#pragma unroll 1
  for (; it.k < g.nvv; it.next()) {
    if constexpr (W > 1) {
      R v[W];
      const R cy = it.vy() - P.uy, cx0 = it.vx() - P.ux;
      if constexpr (std::is_same<R, float>::value && W % 2 == 0) {
        const GhatRow row = ghat_row(P, cy);
#pragma unroll
        for (int j = 0; j < W; j += 2) {
          const float cxa = cx0 + R(j) * dv;
          const float2 Gh = ghat_pair(P, row, make_float2(cxa, cxa + dv));
          v[j] = Gh.x;
          v[j + 1] = Gh.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = ghat(P, cx0 + R(j) * dv, cy);
      }
      VecIO<S, W>::st_sr(f + o0 + it.k, v, key + (uint32_t)((o0 + it.k) << 3));
    } else {
      st(f + o0 + it.k, ghat(P, it.vx() - P.ux, it.vy() - P.uy));
    }
  }
  return true;
}

// Second half of a buffer cell: f := M_hat[U] over the velocities (when
// filling is on) from the Euler result Uc held by lane 0.
template <typename S, int W = 1>
ESBGK_DEV void buffer_fill(const StageArgs& A, const View& V, int c, int lane, double (&Uc)[4]) {
  if (!A.fill) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) Uc[q] = __shfl_sync(0xffffffffu, Uc[q], 0);
  if (!A.hoc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) Uc[q] = A.Un[(size_t)q * V.g.nc + c];
  }
  const uint32_t key = A.seed ? mix32(*A.seed * 0x632be5abu + A.sid + 0x51u) : 0u;
  if (!fill_maxwell<S, W>((S*)A.f_out, V.g, c, lane, Uc, key) && lane == 0) report_error(V.err, kErrNonRealizable, c);
}


// Buffer cell of a stage: Euler update (lane 0), then f := M_hat[U] over the
// velocities when filling is on.
template <typename S, int W = 1>
ESBGK_DEV void buffer_cell(const StageArgs& A, const View& V, int c, int lane) {
  using R = typename Real<S>::T;
  double Uc[4] = {0, 0, 0, 0};
  R ovr[4][4];
  const int omask = (A.iface && A.f_src && A.phi_store >= 0) ? interface_fluxes<S>(A, V, c, lane, ovr) : 0;
  if (lane == 0) euler_cell<R>(A, V, c, Uc, ovr, omask);
  buffer_fill<S, W>(A, V, c, lane, Uc);
}

#ifndef ESBGK_STAGE_MIN_BLOCKS
#define ESBGK_STAGE_MIN_BLOCKS 4  // resident CTAs per SM the register budget is sized for
#endif

// PAIR (vector form, small velocity grids): a kinetic unit is two cells, one
// per half-warp, so that twice as many cells are in flight when a cell has
// only a few node groups per lane.
// WALLS: solid obstacles (View::wsrc): the generic scalar form and the wide
// vector form are compiled with them.
// SUMS: the moment sums of the vector forms (kinetic_cell_vec).
template <typename S, int M, int W, bool PAIR = false, bool SX = false, bool WALLS = false, int SUMS = kSumsPlain>
__global__ void __launch_bounds__(kCellThreads, ESBGK_STAGE_MIN_BLOCKS) stage_kernel(StageArgs A, View V) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool proj = A.h_coef > 0.0 || A.need_q || A.l1_out;
  constexpr int kPer = PAIR ? 2 : 1;  // cells per kinetic unit
  const int half = PAIR ? lane >> 4 : 0;
  R* sfs = reinterpret_cast<R*>(dsm) + (proj ? (size_t)(warp * kPer + half) * V.g.nvv : 0);
  const int nK = V.counts[0], nB = V.counts[1], nF = V.counts[2];
  const int nKu = (nK + kPer - 1) / kPer;
  const int nFc = (nF + 31) / 32;
  const int total = nKu + nB + nFc;
  long long mine = 0, fills = 0;
  // first wave round-robin; later units claimed from the launch's counter, so
  // a warp that drew a long unit (kinetic cell) does not also own a fixed
  // share of the short ones (units are ordered kinetic, buffer, fluid)
  const int first = gridDim.x * nwarps;
  int u = blockIdx.x * nwarps + warp;
  while (u < total) {
    if (u < nKu) {
      if constexpr (PAIR) {
        const int ci = 2 * u + half;  // this half's cell
        if (ci < nK) {
          kinetic_cell_vec<S, M, W, 16, SX, false, SUMS>(A, V, V.klist[ci], lane & 15, sfs,
                                                         half ? 0xffff0000u : 0x0000ffffu);
          ++mine;
        }
      } else if constexpr (W > 1) {
        kinetic_cell_vec<S, M, W, 32, SX, WALLS, SUMS>(A, V, V.klist[u], lane, sfs);
        ++mine;
      } else {
        kinetic_cell<S, M, WALLS>(A, V, V.klist[u], lane, sfs);
        ++mine;
      }
      __syncwarp();
    } else {
      // a buffer cell (Euler update on lane 0, then the fill) or a chunk of
      // 32 fluid cells (one per lane): one call site of the Euler update
      const bool buf = u < nKu + nB;
      const int q = (u - nKu - nB) * 32 + lane;
      const int ec = buf ? (lane == 0 ? V.blist[u - nKu] : -1) : (q < nF ? V.flist[q] : -1);
      double Uc[4] = {0, 0, 0, 0};
      R ovr[4][4];
      const int omask =
          (buf && A.iface && A.f_src && A.phi_store >= 0) ? interface_fluxes<S>(A, V, V.blist[u - nKu], lane, ovr) : 0;
      if (ec >= 0) euler_cell<R, WALLS>(A, V, ec, Uc, ovr, omask);
      if (buf) {
        buffer_fill<S, W>(A, V, V.blist[u - nKu], lane, Uc);
        fills += A.fill ? 1 : 0;
      }
    }
    if (A.wq) {
      int v = 0;
      if (lane == 0) v = atomicAdd(A.wq, 1);
      u = first + __shfl_sync(0xffffffffu, v, 0);
    } else {
      u += first;
    }
  }
  if ((lane & (32 / kPer - 1)) == 0 && A.ctr && mine && A.f_src)  // one lane per cell group
    atomicAdd((unsigned long long*)A.ctr, (unsigned long long)mine);
  if (lane == 0 && A.ctr && fills) atomicAdd((unsigned long long*)A.ctr + 1, (unsigned long long)fills);
}

// ---------------------------------------------------------------------------
// Fill f := M_hat[U] in the cells of two lists and copy U^n -> U^(1) in all
// cells (start of a step), and remember the regime map.
template <typename S>
__global__ void __launch_bounds__(kCellThreads) prep_kernel(PrepArgs P, View V) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const Geo& g = V.g;
  const int n1 = P.count1 ? *P.count1 : 0, n2 = P.count2 ? *P.count2 : 0;
  const int nCopy = P.copy_to ? (g.nc + 31) / 32 : 0;
  const int total = n1 + n2 + nCopy;
  S* f = (S*)P.f;
  if (blockIdx.x == 0 && (int)threadIdx.x < P.wq_n) P.wq_zero[threadIdx.x] = 0;
  // stochastic-rounding key of this step's fills (the counter is advanced by a
  // launch of its own before this one)
  const uint32_t key = P.seed ? mix32(*P.seed * 0x632be5abu + 0x7fu) : 0u;
  constexpr int kW = VecW<S>::value;
  const bool vec = g.nv % kW == 0 && ((uintptr_t)f & 15u) == 0;
  for (int u = blockIdx.x * nwarps + warp; u < total; u += gridDim.x * nwarps) {
    if (u < n1 + n2) {
      const int c = u < n1 ? P.list1[u] : P.list2[u - n1];
      double Uc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) Uc[q] = P.U[(size_t)q * g.nc + c];
      const bool ok = vec ? fill_maxwell<S, kW>(f, g, c, lane, Uc, key) : fill_maxwell<S>(f, g, c, lane, Uc);
      if (!ok && lane == 0) report_error(V.err, kErrNonRealizable, c);
    } else {
      const int c = (u - n1 - n2) * 32 + lane;
      if (c < g.nc) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P.copy_to[(size_t)q * g.nc + c] = P.U[(size_t)q * g.nc + c];
        if (P.flags_prev) P.flags_prev[c] = V.flags[c];
      }
    }
  }
}

// Moments of cell c of f into sf (when given) and m (raw sums about u0).
template <typename S>
ESBGK_DEV void load_moments(const S* f, const Geo& g, int c, int lane, typename Real<S>::T u0x,
                            typename Real<S>::T u0y, typename Real<S>::T* sf, typename Real<S>::T (&m)[6]) {
  using R = typename Real<S>::T;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  const size_t o0 = (size_t)c * g.nvv;
#pragma unroll
  for (int n = 0; n < 6; ++n) m[n] = R(0);
  NodeIter<R> it(lane, g.nv, v0, dv);
#pragma unroll 1
  for (; it.k < g.nvv; it.next()) {
    const R x = ld(f + o0 + it.k);
    if (sf) sf[it.k] = x;
    const R cx = it.vx() - u0x, cy = it.vy() - u0y;
    m[0] += x;
    m[1] += cx * x;
    m[2] += cy * x;
    m[3] += cx * cx * x;
    m[4] += cx * cy * x;
    m[5] += cy * cy * x;
  }
#pragma unroll
  for (int n = 0; n < 6; ++n) m[n] = warp_sum(m[n]);
}

// ---------------------------------------------------------------------------
// L1 deviation ||f - M_hat[f]||_{L1_v} of the kinetic cells (Eq. eqKintoFluid1).
template <typename S>
__global__ void __launch_bounds__(kCellThreads) l1_kernel(const void* fptr, const double* U, double* L1, View V) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const Geo& g = V.g;
  R* sf = reinterpret_cast<R*>(dsm) + (size_t)warp * g.nvv;
  const S* f = (const S*)fptr;
  const int nK = V.counts[0];
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  for (int u = blockIdx.x * nwarps + warp; u < nK; u += gridDim.x * nwarps) {
    const int c = V.klist[u];
    R u0x, u0y, m[6];
    ref_velocity(U, g.nc, c, u0x, u0y);
    load_moments<S>(f, g, c, lane, u0x, u0y, sf, m);
    // Maxwellian of f's own moments: the ES tensor with beta = 0
    CellPar<R> P;
    bool ok = es_params<R>(m, u0x, u0y, pick<R>(g.w, g.fw), R(0), R(0), false, P);
    if (ok) ok = project<R>(g, lane, P);
    if (!ok) {
      if (lane == 0) report_error(V.err, kErrNonRealizable, c);
      continue;
    }
    R s = R(0);
    NodeIter<R> it(lane, g.nv, v0, dv);
#pragma unroll 1
    for (; it.k < g.nvv; it.next()) s += rabs(sf[it.k] - ghat(P, it.vx() - P.ux, it.vy() - P.uy));
    s = warp_sum(s);
    if (lane == 0) L1[c] = g.w * (double)s;
  }
}

// ---------------------------------------------------------------------------
// Relaxation of independent cells (entry point esbgk_relax_cells).
template <typename S>
__global__ void __launch_bounds__(kCellThreads) relax_cells_kernel(const S* fstar, const double* h, int n, Geo g,
                                                                    double beta, S* fout, S* gout) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  R* sf = reinterpret_cast<R*>(dsm) + (size_t)warp * g.nvv;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  for (int c = blockIdx.x * nwarps + warp; c < n; c += gridDim.x * nwarps) {
    const size_t o0 = (size_t)c * g.nvv;
    R m[6];
    load_moments<S>(fstar, g, c, lane, R(0), R(0), sf, m);
    const R hh = (R)h[c];
    CellPar<R> P;
    bool ok = es_params<R>(m, R(0), R(0), pick<R>(g.w, g.fw), (R)beta, hh, true, P);
    if (ok) ok = project<R>(g, lane, P);
    const R nan = R(__int_as_float(0x7fc00000));
    const R inv1h = R(1) / (R(1) + hh);
    NodeIter<R> it(lane, g.nv, v0, dv);
    for (; it.k < g.nvv; it.next()) {
      if (ok) {
        const R Gh = ghat(P, it.vx() - P.ux, it.vy() - P.uy);
        st(fout + o0 + it.k, (sf[it.k] + hh * Gh) * inv1h);
        st(gout + o0 + it.k, Gh);
      } else {
        st(fout + o0 + it.k, nan);
        st(gout + o0 + it.k, nan);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// U := moments(f) in the kinetic cells (Eq. Coupling_KinFlu).
template <typename S>
__global__ void __launch_bounds__(kCellThreads) moments_kernel(const void* fptr, double* U, View V) {
  using R = typename Real<S>::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const Geo& g = V.g;
  const S* f = (const S*)fptr;
  for (int u = blockIdx.x * nwarps + warp; u < V.counts[0]; u += gridDim.x * nwarps) {
    const int c = V.klist[u];
    R m[6];
    load_moments<S>(f, g, c, lane, R(0), R(0), nullptr, m);
    double Uc[4];
    cons_from_sums(m, R(0), R(0), g.w, Uc);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) U[(size_t)q * g.nc + c] = Uc[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Batched form.  A warp copies the descriptor of its unit's case into shared
// memory and runs the same per-cell code as the single-case kernels.

// Copy a descriptor of `bytes` (multiple of 4) with the 32 lanes of a warp.
ESBGK_DEV void warp_copy(void* dst, const void* src, int bytes, int lane) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int w = lane; w < bytes / 4; w += 32) d[w] = s[w];
  __syncwarp();
}

static_assert(kCellWarps * sizeof(CaseStage) <= kBatchStaticSmem && sizeof(CaseStage) % 4 == 0, "descriptor copies");
static_assert(kCellWarps * sizeof(CaseRegime) <= kBatchStaticSmem && sizeof(CaseRegime) % 4 == 0, "descriptor copies");
static_assert(kCellWarps * sizeof(CasePrep) <= kBatchStaticSmem && sizeof(CasePrep) % 4 == 0, "descriptor copies");

// One variant of the per-cell code (W, PAIR, SX as in stage_kernel); `off` is the
// unit prefix of this variant, in which cases of other variants are empty.
template <typename S, int M, int W, bool PAIR, bool SX, int SUMS = kSumsPlain>
__global__ void __launch_bounds__(kCellThreads, ESBGK_STAGE_MIN_BLOCKS)
    batch_stage_kernel(const CaseStage* __restrict__ cases, const int* __restrict__ off, int n, int max_nvv) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) CaseStage cs[kCellWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int kPer = PAIR ? 2 : 1;  // cells per kinetic unit
  const int half = PAIR ? lane >> 4 : 0;
  R* sfs = reinterpret_cast<R*>(dsm) + (size_t)warp * max_nvv;
  const int total = off[n];
  for (int u = blockIdx.x * nwarps + warp; u < total; u += gridDim.x * nwarps) {
    const int c = find_case(off, n, u);
    __syncwarp();
    warp_copy(&cs[warp], &cases[c], sizeof(CaseStage), lane);
    const View& V = cs[warp].V;
    const StageArgs& A = cs[warp].A;
    const int local = u - off[c];
    const int nK = V.counts[0], nB = V.counts[1], nF = V.counts[2];
    const int nKu = (nK + kPer - 1) / kPer;
    if (local < nKu) {
      if constexpr (PAIR) {
        // two cells, one per half-warp, each with its own f* array
        const int ci = 2 * local + half;
        if (ci < nK) {
          kinetic_cell_vec<S, M, W, 16, SX, false, SUMS>(A, V, V.klist[ci], lane & 15, sfs + half * V.g.nvv,
                                                         half ? 0xffff0000u : 0x0000ffffu);
          if ((lane & 15) == 0 && A.ctr && A.f_src) atomicAdd((unsigned long long*)A.ctr, 1ull);
        }
        __syncwarp();
      } else {
        if constexpr (W > 1)
          kinetic_cell_vec<S, M, W, 32, SX, false, SUMS>(A, V, V.klist[local], lane, sfs);
        else
          kinetic_cell<S, M>(A, V, V.klist[local], lane, sfs);
        if (lane == 0 && A.ctr && A.f_src) atomicAdd((unsigned long long*)A.ctr, 1ull);
      }
    } else if (local < nKu + nB) {
      buffer_cell<S, W>(A, V, V.blist[local - nKu], lane);
      if (lane == 0 && A.ctr && A.fill) atomicAdd((unsigned long long*)A.ctr + 1, 1ull);
    } else {
      const int q = (local - nKu - nB) * 32 + lane;
      if (q < nF) {
        double Uc[4];
        euler_cell<R>(A, V, V.flist[q], Uc);
      }
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(kCellThreads) batch_prep_kernel(const CasePrep* __restrict__ cases,
                                                                   const int* __restrict__ off, int n) {
  __shared__ __align__(16) CasePrep cp[kCellWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int total = off[n];
  for (int u = blockIdx.x * nwarps + warp; u < total; u += gridDim.x * nwarps) {
    const int c = find_case(off, n, u);
    __syncwarp();
    warp_copy(&cp[warp], &cases[c], sizeof(CasePrep), lane);
    const View& V = cp[warp].V;
    const PrepArgs& P = cp[warp].P;
    const Geo& g = V.g;
    const int local = u - off[c];
    const int n1 = P.count1 ? *P.count1 : 0, n2 = P.count2 ? *P.count2 : 0;
    if (local < n1 + n2) {
      const int cell = local < n1 ? P.list1[local] : P.list2[local - n1];
      double Uc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) Uc[q] = P.U[(size_t)q * g.nc + cell];
      constexpr int kW = VecW<S>::value;
      const bool vec = g.nv % kW == 0 && ((uintptr_t)P.f & 15u) == 0;
      const uint32_t key = P.seed ? mix32(*P.seed * 0x632be5abu + 0x7fu) : 0u;
      const bool ok = vec ? fill_maxwell<S, kW>((S*)P.f, g, cell, lane, Uc, key) : fill_maxwell<S>((S*)P.f, g, cell, lane, Uc);
      if (!ok && lane == 0) report_error(V.err, kErrNonRealizable, cell);
    } else {
      const int cell = (local - n1 - n2) * 32 + lane;
      if (cell < g.nc && P.copy_to) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P.copy_to[(size_t)q * g.nc + cell] = P.U[(size_t)q * g.nc + cell];
        if (P.flags_prev) P.flags_prev[cell] = V.flags[cell];
      }
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(kCellThreads) batch_l1_kernel(const CaseRegime* __restrict__ cases,
                                                                 const int* __restrict__ off, int n, int max_nvv) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) CaseRegime cr[kCellWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  R* sf = reinterpret_cast<R*>(dsm) + (size_t)warp * max_nvv;
  const int total = off[n];
  for (int u = blockIdx.x * nwarps + warp; u < total; u += gridDim.x * nwarps) {
    const int c = find_case(off, n, u);
    __syncwarp();
    warp_copy(&cr[warp], &cases[c], sizeof(CaseRegime), lane);
    const CaseRegime& Rg = cr[warp];
    const Geo& g = Rg.V.g;
    const int cell = Rg.klist[u - off[c]];
    R u0x, u0y, m[6];
    ref_velocity(Rg.Un, g.nc, cell, u0x, u0y);
    load_moments<S>((const S*)Rg.f, g, cell, lane, u0x, u0y, sf, m);
    __syncwarp();
    const R l1 = l1_deviation<R, 1>(g, lane, m, u0x, u0y, sf);
    if (lane == 0) {
      if (l1 < R(0)) report_error(Rg.V.err, kErrNonRealizable, cell);
      Rg.L1[cell] = (double)l1;
    }
  }
}

}  // namespace esbgk

#include "tile_impl.cuh"

namespace esbgk {

// ---------------------------------------------------------------------------
// Host-side launchers for storage type S.
// The stage kernels with run-time moment sums (compensated sums requested;
// FP32 arithmetic only), compiled in translation units of their own
// (kernels_f32_sums.cu, kernels_bf16_sums.cu) so that the main ones build in
// parallel with them.  The first argument selects the storage type.
using StageFnT = void (*)(StageArgs, View);
using BatchFnT = void (*)(const CaseStage*, const int*, int, int);
StageFnT stage_fn_runtime_sums(const float*, int m, int var);
StageFnT stage_fn_runtime_sums(const __nv_bfloat16*, int m, int var);
BatchFnT batch_fn_runtime_sums(const float*, int m, int var);
BatchFnT batch_fn_runtime_sums(const __nv_bfloat16*, int m, int var);

template <typename S>
struct Launch {
  using R = typename Real<S>::T;
  // Warps per CTA so that `arrays` shared arrays of N_v^2 values per warp fit
  // the device's opt-in shared memory per block (fewer warps for large FP64
  // velocity grids).
  static int max_smem() {
    static int v = 0;
    if (!v) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (v <= 0) v = 48 * 1024;
    }
    return v;
  }
  static int warps_for(const Geo& g, int arrays) {
    const size_t per = (size_t)arrays * g.nvv * sizeof(R);
    int w = kCellWarps;
    while (w > 1 && per * w > (size_t)max_smem()) --w;
    return w;
  }
  static size_t smem_for(const Geo& g, int arrays) {
    return (size_t)warps_for(g, arrays) * arrays * g.nvv * sizeof(R);
  }
  // Occupancy (blocks per SM), memoised: the launchers call it on every launch.
  static int occ(const void* fn, int threads, size_t smem) {
    struct Entry {
      const void* fn;
      int threads;
      size_t smem;
      int nb;
    };
    static Entry cache[32];
    static int used = 0;
    for (int q = 0; q < used; ++q)
      if (cache[q].fn == fn && cache[q].threads == threads && cache[q].smem == smem) return cache[q].nb;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
    nb = nb < 1 ? 1 : nb;
    if (used < 32) cache[used++] = {fn, threads, smem, nb};
    return nb;
  }

  using StageFn = StageFnT;
  static constexpr int kW = VecW<S>::value;
  // node groups of the variants: kW, or 2 (fewer nodes per group than kW
  // when N_v is not a multiple of kW)
  static constexpr int narrow_w() { return kW > 2 ? 2 : kW; }
  template <int M, int SUMS>
  static StageFn stage_variant(int var) {
    switch (var) {
      case kVarWide: return stage_kernel<S, M, kW, false, false, false, SUMS>;
      case kVarWidePair: return stage_kernel<S, M, kW, true, false, false, SUMS>;
      case kVarWideSx: return stage_kernel<S, M, kW, false, true, false, SUMS>;
      case kVarWideSxPair: return stage_kernel<S, M, kW, true, true, false, SUMS>;
      case kVarNarrowSx: return stage_kernel<S, M, narrow_w(), false, true, false, SUMS>;
      case kVarNarrowSxPair: return stage_kernel<S, M, narrow_w(), true, true, false, SUMS>;
      default: return stage_kernel<S, M, 1>;  // the scalar form sums plainly
    }
  }
  template <int SUMS>
  static StageFn stage_fn_sums(int m, int var) {
    switch (m) {
      case kFirstRelax2: return stage_variant<kFirstRelax2, SUMS>(var);
      case kLoadedRelax1: return stage_variant<kLoadedRelax1, SUMS>(var);
      case kFinal: return stage_variant<kFinal, SUMS>(var);
      case kFirstRelax0: return stage_variant<kFirstRelax0, SUMS>(var);
      default: return stage_kernel<S, kGeneric, 1>;
    }
  }
  // comp: compensated moment sums requested (only the FP32-arithmetic vector
  // forms have them; the others always sum plainly)
  static StageFn stage_fn(int m, int var = kVarScalar, bool comp = false) {
    if constexpr (std::is_same<R, float>::value)
      if (comp) return stage_fn_runtime_sums((const S*)nullptr, m, var);
    return stage_fn_sums<kSumsPlain>(m, var);
  }
  // With solid obstacles: the wide vector form with the wall stencils (one
  // cell per warp) where the specialised modes would take a wide form, else
  // the generic scalar form.
  static StageFn wall_fn(int m, int var) {
    if (var == kVarWide || var == kVarWidePair) {
      switch (m) {
        case kFirstRelax2: return stage_kernel<S, kFirstRelax2, kW, false, false, true, kSumsRunTime>;
        case kLoadedRelax1: return stage_kernel<S, kLoadedRelax1, kW, false, false, true, kSumsRunTime>;
        case kFinal: return stage_kernel<S, kFinal, kW, false, false, true, kSumsRunTime>;
        case kFirstRelax0: return stage_kernel<S, kFirstRelax0, kW, false, false, true, kSumsRunTime>;
        default: break;
      }
    }
    return stage_kernel<S, kGeneric, 1, false, false, true>;
  }
  static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
  // Per-cell code of a stage launch: the vector form (specialised modes,
  // every f-sized array 16-byte aligned, N_v divisible by the group size)
  // with groups of kW nodes, else of 2, else the scalar form; two cells per
  // warp when a cell has at most kPairMaxNodes nodes (few node groups per
  // lane: per-cell latency dominates).
  static int variant(const StageArgs& A, const Geo& g, int mode) {
    if (mode == kGeneric) return kVarScalar;
    if (!aligned16(A.f_src) || !aligned16(A.star_base) || !aligned16(A.f_out)) return kVarScalar;
    for (int t = 0; t < A.nacc; ++t)
      if (!aligned16(A.acc_in[t]) || !aligned16(A.acc_out[t])) return kVarScalar;
    const int pair = g.nvv <= kPairMaxNodes ? 1 : 0;
    if (g.nv % (2 * kW) == 0) return kVarWide + pair;
    if (kW > 2 && g.nv % kW == 0) return kVarWideSx + pair;
    if (g.nv % 2 == 0) return kVarNarrowSx + pair;  // N_v/2 odd when kW = 2
    return kVarScalar;
  }
  using BatchFn = BatchFnT;
  template <int M, int SUMS>
  static BatchFn batch_variant(int var) {
    switch (var) {
      case kVarWide: return batch_stage_kernel<S, M, kW, false, false, SUMS>;
      case kVarWidePair: return batch_stage_kernel<S, M, kW, true, false, SUMS>;
      case kVarWideSx: return batch_stage_kernel<S, M, kW, false, true, SUMS>;
      case kVarWideSxPair: return batch_stage_kernel<S, M, kW, true, true, SUMS>;
      case kVarNarrowSx: return batch_stage_kernel<S, M, narrow_w(), false, true, SUMS>;
      case kVarNarrowSxPair: return batch_stage_kernel<S, M, narrow_w(), true, true, SUMS>;
      default: return batch_stage_kernel<S, M, 1, false, false>;  // the scalar form sums plainly
    }
  }
  template <int SUMS>
  static BatchFn batch_fn_sums(int m, int var) {
    switch (m) {
      case kFirstRelax2: return batch_variant<kFirstRelax2, SUMS>(var);
      case kLoadedRelax1: return batch_variant<kLoadedRelax1, SUMS>(var);
      case kFinal: return batch_variant<kFinal, SUMS>(var);
      case kFirstRelax0: return batch_variant<kFirstRelax0, SUMS>(var);
      default: return batch_stage_kernel<S, kGeneric, 1, false, false>;
    }
  }
  // comp: some case of the launch asks for compensated moment sums
  static BatchFn batch_fn(int m, int var, bool comp) {
    if constexpr (std::is_same<R, float>::value)
      if (comp) return batch_fn_runtime_sums((const S*)nullptr, m, var);
    return batch_fn_sums<kSumsPlain>(m, var);
  }
  // Tiled stage kernel (every cell kinetic, regime frozen): the specialised
  // modes, an even N_v, the per-pair arrays aligned, no fused L1 deviation,
  // and f* of a whole tile in shared memory.
  using TileFn = void (*)(StageArgs, View);
  template <int M, int E>
  static TileFn tile_variant(bool sx, bool comp) {
    if (comp) return sx ? tile_stage_kernel<S, M, true, true, E> : tile_stage_kernel<S, M, false, true, E>;
    return sx ? tile_stage_kernel<S, M, true, false, E> : tile_stage_kernel<S, M, false, false, E>;
  }
  template <int E>
  static TileFn tile_edge_fn(int m, bool sx, bool comp) {
    switch (m) {
      case kFirstRelax2: return tile_variant<kFirstRelax2, E>(sx, comp);
      case kLoadedRelax1: return tile_variant<kLoadedRelax1, E>(sx, comp);
      case kFinal: return tile_variant<kFinal, E>(sx, comp);
      case kFirstRelax0: return tile_variant<kFirstRelax0, E>(sx, comp);
      default: return nullptr;
    }
  }
  // compensated sums only change the float arithmetic
  static TileFn tile_fn(int m, bool sx, bool comp) {
    comp = comp && std::is_same<R, float>::value;
    return tile_edge_fn<kTileEdge>(m, sx, comp);
  }
  static bool aligned_pair(const void* p) { return ((uintptr_t)p % (2 * sizeof(S))) == 0; }
  static int tile_ok(const StageArgs& A, const Geo& g) {
    const int mode = stage_mode(A);
    if (mode == kGeneric || g.nv % 2 != 0 || A.l1_out || A.iface) return 0;
    if (TileSmem<R, kTileEdge>::bytes(g) > (size_t)max_smem()) return 0;
    if (!aligned_pair(A.f_src) || !aligned_pair(A.star_base) || !aligned_pair(A.f_out)) return 0;
    for (int t = 0; t < A.nacc; ++t)
      if (!aligned_pair(A.acc_in[t]) || !aligned_pair(A.acc_out[t])) return 0;
    return 1;
  }
  static void stage_tile(const StageArgs& A, const View& V, int grid, cudaStream_t s) {
    const Geo& g = V.g;
    const TileFn fn = tile_fn(stage_mode(A), (g.nv / 2) % 2 != 0, V.m.comp_moments != 0);
    const size_t smem = TileSmem<R, kTileEdge>::bytes(g);
    constexpr int E = kTileEdge, threads = TileShape<E>::kThreads;
    const int ntiles = ((g.nx + E - 1) / E) * ((g.ny + E - 1) / E);
    int gr = rescale(g, grid, (const void*)fn, threads, smem);
    if (gr > ntiles) gr = ntiles;
    fn<<<gr, threads, smem, s>>>(A, V);
  }
  static cudaError_t setup(const Geo& g) {
    if ((size_t)g.nvv * sizeof(R) > (size_t)max_smem()) return cudaErrorInvalidValue;
    cudaError_t e;
    const int mx = max_smem();
    for (int m = 0; m < kNumModes; ++m)
      for (int v = 0; v < 4; ++v) {
        const TileFn fn = tile_fn(m, v & 1, v & 2);
        if (fn && (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
          return e;
      }
    for (int m = 0; m < kNumModes; ++m)
      for (int v = 0; v < 2 * kNumVariants; ++v)
        if ((e = cudaFuncSetAttribute(stage_fn(m, v % kNumVariants, v >= kNumVariants),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
          return e;
    if ((e = cudaFuncSetAttribute(l1_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
      return e;
    for (int m = 0; m < kNumModes; ++m)
      if ((e = cudaFuncSetAttribute(wall_fn(m, kVarWide), cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
          cudaSuccess)
        return e;
    // batched kernels: set here so that their launches can be graph-captured
    const int mb = mx - kBatchStaticSmem;
    for (int m = 0; m < kNumModes; ++m)
      for (int v = 0; v < 2 * kNumVariants; ++v)
        if ((e = cudaFuncSetAttribute(batch_fn(m, v % kNumVariants, v >= kNumVariants),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, mb)) != cudaSuccess)
          return e;
    if ((e = cudaFuncSetAttribute(batch_l1_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mb)) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(relax_cells_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  }
  static int blocks_per_sm(const Geo& g) {
    return occ((const void*)stage_fn(kGeneric), kCellThreads, smem_for(g, 1));
  }
  // `grid` is the SM count times blocks_per_sm(); each launch rescales it to
  // its own footprint.
  static int rescale(const Geo& g, int grid, const void* fn, int threads, size_t smem) {
    const int nsm = grid / blocks_per_sm(g);
    const int g2 = (nsm > 0 ? nsm : 1) * occ(fn, threads, smem);
    return g2 > 0 ? g2 : grid;
  }
  static void stage(const StageArgs& A, const View& V, int grid, cudaStream_t s) {
    const bool proj = A.h_coef > 0.0 || A.need_q || A.l1_out;
    const int mode = stage_mode(A), var = variant(A, V.g, mode);
    const int arrays = V.wsrc || !variant_pairs(var) ? 1 : 2;  // f* arrays per warp
    const int threads = 32 * warps_for(V.g, arrays);
    const size_t smem = proj ? smem_for(V.g, arrays) : 0;
    // solid obstacles: the forms with the wall stencils
    const StageFn fn = V.wsrc ? wall_fn(mode, var) : stage_fn(mode, var, V.m.comp_moments != 0);
    fn<<<rescale(V.g, grid, (const void*)fn, threads, smem), threads, smem, s>>>(A, V);
  }
  static void prep(const PrepArgs& P, const View& V, int grid, cudaStream_t s) {
    prep_kernel<S><<<rescale(V.g, grid, (const void*)prep_kernel<S>, kCellThreads, 0), kCellThreads, 0, s>>>(P, V);
  }
  static void l1(const void* f, const double* U, double* L1, const View& V, int grid, cudaStream_t s) {
    const int threads = 32 * warps_for(V.g, 1);
    const size_t smem = smem_for(V.g, 1);
    l1_kernel<S><<<rescale(V.g, grid, (const void*)l1_kernel<S>, threads, smem), threads, smem, s>>>(f, U, L1, V);
  }
  static void relax_cells(const void* fs, const double* h, int n, const Geo& g, double beta, void* fo, void* go,
                          int grid, cudaStream_t s) {
    const int threads = 32 * warps_for(g, 1);
    relax_cells_kernel<S><<<grid, threads, smem_for(g, 1), s>>>((const S*)fs, h, n, g, beta, (S*)fo, (S*)go);
  }
  static size_t batch_smem(int max_nvv, int threads) { return (size_t)(threads / 32) * max_nvv * sizeof(R); }
  static int batch_stage_occupancy(int mode, int var, bool comp, int max_nvv, int threads) {
    return occ((const void*)batch_fn(mode, var, comp), threads, batch_smem(max_nvv, threads));
  }
  static void batch_stage(const CaseStage* cases, const int* off, int n, int mode, int var, bool comp, int max_nvv,
                          int threads, int grid, cudaStream_t s) {
    const BatchFn fn = batch_fn(mode, var, comp);
    fn<<<grid, threads, batch_smem(max_nvv, threads), s>>>(cases, off, n, max_nvv);
  }
  static void batch_prep(const CasePrep* cases, const int* off, int n, int grid, cudaStream_t s) {
    batch_prep_kernel<S><<<grid, kCellThreads, 0, s>>>(cases, off, n);
  }
  static void batch_l1(const CaseRegime* cases, const int* off, int n, int max_nvv, int grid, cudaStream_t s) {
    batch_l1_kernel<S><<<grid, kCellThreads, kCellWarps * (size_t)max_nvv * sizeof(R), s>>>(cases, off, n, max_nvv);
  }
  static int variant_public(const StageArgs& A, const Geo& g) { return variant(A, g, stage_mode(A)); }
  static void moments(const void* f, double* U, const View& V, int grid, cudaStream_t s) {
    moments_kernel<S><<<rescale(V.g, grid, (const void*)moments_kernel<S>, kCellThreads, 0), kCellThreads, 0, s>>>(
        f, U, V);
  }
};

#define ESBGK_INSTANTIATE(S, NAME)                                                                            \
  const Launchers NAME = {sizeof(S),                          &Launch<S>::setup,        &Launch<S>::blocks_per_sm, \
                          &Launch<S>::stage,                  &Launch<S>::prep,         &Launch<S>::l1,            \
                          &Launch<S>::relax_cells,            &Launch<S>::moments,      &Launch<S>::batch_stage,   \
                          &Launch<S>::batch_prep,             &Launch<S>::batch_l1,                               \
                          &Launch<S>::batch_stage_occupancy, &Launch<S>::variant_public, VecW<S>::value,       \
                          &Launch<S>::tile_ok,                &Launch<S>::stage_tile};

}  // namespace esbgk
