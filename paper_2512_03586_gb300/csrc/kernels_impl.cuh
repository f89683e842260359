// kernels_impl.cuh -- the per-precision kernels of the ES-BGK library.
//
// Included by one translation unit per storage type S (double, float,
// __nv_bfloat16), each of which instantiates the launchers declared in
// launch.h.  All per-element arithmetic runs in R = Real<S>::T; per-cell tensor
// solves and U run in float64.
#pragma once

#include "common.cuh"
#include "launch.h"

namespace esbgk {

// ---------------------------------------------------------------------------
// Per-CTA shared state of one cell.
struct CellShared {
  double red[kWarps * 15];
  double tot[16];
  double rho, ux, uy, T;          // moments of the cell
  double ixx, ixy, iyy;           // inverse temperature tensor
  double pref, isT;               // rho/(2 pi sqrt det Tt), 1/sqrt(T)
  double h, nu;                   // implicit coefficient dt a_ii nu, nu = tau/eps
  double a[6];                    // moment-projection coefficients
  double U[4];                    // conserved variables (fluid/buffer cells)
  int ok;
};

// Monomial index of xi_x^p xi_y^q (p + q <= 4) in the 15 projection sums.
__host__ __device__ constexpr int mono(int p, int q) { return (p + q) * (p + q + 1) / 2 + q; }

// Exponents of the quadratic basis psi = (1, x, y, x^2, xy, y^2).
static __device__ __constant__ int kPsiP[6] = {0, 1, 0, 2, 1, 0};
static __device__ __constant__ int kPsiQ[6] = {0, 0, 1, 0, 1, 2};

// Per-cell temperature tensor and Gaussian parameters (thread 0 only).
// From the moments m = (rho, m_x, m_y, S_xx, S_xy, S_yy) (already multiplied by
// w): u = m/rho, Theta = S/rho - u u, T = tr(Theta)/2 (hypothesis H3, Sec. 2).
// If relax: Theta <- (Theta + k T I)/(1 + k), k = h (1 - beta), the exact
// stress moment of the implicit stage.  Tt = (1 - beta) T I + beta Theta.
// Returns false for a non-realizable state.
static __device__ bool cell_tensor(CellShared& sh, const double* m, double beta, double h, bool relax) {
  const double rho = m[0];
  if (!(rho > 0.0)) return false;
  const double ux = m[1] / rho, uy = m[2] / rho;
  double txx = m[3] / rho - ux * ux, txy = m[4] / rho - ux * uy, tyy = m[5] / rho - uy * uy;
  const double T = 0.5 * (txx + tyy);
  if (!(T > 0.0)) return false;
  if (relax) {
    const double k = h * (1.0 - beta);
    const double inv = 1.0 / (1.0 + k);
    txx = (txx + k * T) * inv;
    txy = txy * inv;
    tyy = (tyy + k * T) * inv;
  }
  const double Txx = (1.0 - beta) * T + beta * txx;
  const double Txy = beta * txy;
  const double Tyy = (1.0 - beta) * T + beta * tyy;
  const double det = Txx * Tyy - Txy * Txy;
  if (!(det > 0.0)) return false;
  sh.rho = rho;
  sh.ux = ux;
  sh.uy = uy;
  sh.T = T;
  sh.ixx = Tyy / det;
  sh.ixy = -Txy / det;
  sh.iyy = Txx / det;
  sh.pref = rho / (2.0 * kPi * sqrt(det));
  sh.isT = 1.0 / sqrt(T);
  // targets t of the projection (density, zero mean in xi, stress Tt/T)
  sh.a[0] = rho;
  sh.a[1] = 0.0;
  sh.a[2] = 0.0;
  sh.a[3] = rho * Txx / T;
  sh.a[4] = rho * Txy / T;
  sh.a[5] = rho * Tyy / T;
  return true;
}

// Same parameters for the Maxwellian of (rho, u, T): Tt = T I.
static __device__ bool cell_maxwell(CellShared& sh, double rho, double ux, double uy, double T) {
  if (!(rho > 0.0) || !(T > 0.0)) return false;
  sh.rho = rho;
  sh.ux = ux;
  sh.uy = uy;
  sh.T = T;
  sh.ixx = 1.0 / T;
  sh.ixy = 0.0;
  sh.iyy = 1.0 / T;
  sh.pref = rho / (2.0 * kPi * T);
  sh.isT = 1.0 / sqrt(T);
  sh.a[0] = rho;
  sh.a[1] = 0.0;
  sh.a[2] = 0.0;
  sh.a[3] = rho;
  sh.a[4] = 0.0;
  sh.a[5] = rho;
  return true;
}

// 6x6 symmetric positive definite solve by Cholesky, in place on b.
static __device__ bool chol6(double (&H)[6][6], double (&b)[6]) {
  double L[6][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double s = H[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) return false;
    const double d = sqrt(s);
    L[j][j] = d;
    const double id = 1.0 / d;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      double t = H[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t * id;
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * b[k];
    b[i] = t / L[i][i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    double t = b[i];
#pragma unroll
    for (int k = i + 1; k < 6; ++k) t -= L[k][i] * b[k];
    b[i] = t / L[i][i];
  }
  return true;
}

// Discrete Gaussian with exact moments (the projected ES Gaussian): evaluate
// G_k = pref exp(-(v_k-u)^T Tt^{-1} (v_k-u)/2) into Gs[k], reduce the 15
// moments w sum G xi^p eta^q (xi = (v-u)/sqrt T), and solve H a = t - r for the
// coefficients of G_hat = G (1 + a . psi).  Needs sh filled by cell_tensor or
// cell_maxwell (sh.a holds the targets t on entry).  Sets sh.ok = 0 on a
// singular system.  All threads of the CTA must call it.
template <typename R>
__device__ void gauss_project(const Geo& g, CellShared& sh, R* Gs) {
  const R L2E = R(1.4426950408889634);
  const R ux = (R)sh.ux, uy = (R)sh.uy;
  const R qxx = (R)(-0.5 * sh.ixx) * L2E, qxy = (R)(-sh.ixy) * L2E, qyy = (R)(-0.5 * sh.iyy) * L2E;
  const R pref = (R)sh.pref, isT = (R)sh.isT;
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv;
  R s[15];
#pragma unroll
  for (int n = 0; n < 15; ++n) s[n] = R(0);
  for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
    const int kx = k % g.nv, ky = k / g.nv;
    const R cx = v0 + R(kx) * dv - ux, cy = v0 + R(ky) * dv - uy;
    const R G = pref * exp2r(qxx * cx * cx + qxy * cx * cy + qyy * cy * cy);
    Gs[k] = G;
    const R x = cx * isT, y = cy * isT;
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
  block_sum<15>(s, sh.red, sh.tot);
  if (threadIdx.x == 0) {
    const double w = g.w;
    double H[6][6], rhs[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
#pragma unroll
      for (int n = 0; n < 6; ++n) H[m][n] = w * sh.tot[mono(kPsiP[m] + kPsiP[n], kPsiQ[m] + kPsiQ[n])];
      rhs[m] = sh.a[m] - w * sh.tot[mono(kPsiP[m], kPsiQ[m])];
    }
    const bool ok = chol6(H, rhs);
#pragma unroll
    for (int m = 0; m < 6; ++m) sh.a[m] = ok ? rhs[m] : 0.0;
    sh.ok = ok ? sh.ok : 0;
  }
  __syncthreads();
}

// G_hat at node k from the stored G_k.
template <typename R>
ESBGK_DEV R ghat_at(const Geo& g, const CellShared& sh, const R* a, R G, int k) {
  const int kx = k % g.nv, ky = k / g.nv;
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv, isT = (R)sh.isT;
  const R x = (v0 + R(kx) * dv - (R)sh.ux) * isT, y = (v0 + R(ky) * dv - (R)sh.uy) * isT;
  return G * (R(1) + a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y);
}

// Element offsets of the two-cell cross stencil of cell c (BC mapped):
// o[0..3] = i-2, i-1, i+1, i+2 along x, o[4..7] the same along y.
ESBGK_DEV void stencil_offsets(const Geo& g, int c, size_t (&o)[8]) {
  const int i = c % g.nx, j = c / g.nx;
  const int d[4] = {-2, -1, 1, 2};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[q] = ((size_t)j * g.nx + nb(i + d[q], g.nx, g.bcx)) * g.nvv;
    o[4 + q] = ((size_t)nb(j + d[q], g.ny, g.bcy) * g.nx + i) * g.nvv;
  }
}

// L(f) at node k of cell c: upwind (Lax-Friedrichs with |v_k|) flux of CWENO3
// face values along x and y.  up/dn/far are the upwind, downwind and far
// upwind neighbours for the sign of v, so no branch diverges within a warp;
// L_x = |v_x| (F(face away from upwind) - F(face toward upwind)) / dx.
template <typename S, typename R>
ESBGK_DEV R transport_at(const S* __restrict__ f, size_t o0, const size_t (&o)[8], int k, R vx, R vy,
                         R idx, R idy, R epsw, R& q0) {
  q0 = ld(f + o0 + k);
  const bool px = vx > R(0), py = vy > R(0);
  const R ux = ld(f + (px ? o[1] : o[2]) + k);
  const R dx = ld(f + (px ? o[2] : o[1]) + k);
  const R fx = ld(f + (px ? o[0] : o[3]) + k);
  const R uy = ld(f + (py ? o[5] : o[6]) + k);
  const R dy = ld(f + (py ? o[6] : o[5]) + k);
  const R fy = ld(f + (py ? o[4] : o[7]) + k);
  const R Lx = fabs(vx) * (cweno_face(ux, q0, dx, epsw) - cweno_face(fx, ux, q0, epsw)) * idx;
  const R Ly = fabs(vy) * (cweno_face(uy, q0, dy, epsw) - cweno_face(fy, uy, q0, epsw)) * idy;
  return Lx + Ly;
}

// ---------------------------------------------------------------------------
// Euler part (fluid cells), one thread per cell.

// Physical flux of Eq. Euler_Compact along d (0 = x, 1 = y), gamma = 2, and the
// local wave speed |u_d| + sqrt(gamma P/rho).
template <typename R>
ESBGK_DEV void euler_phys(const R (&U)[4], int d, R (&F)[4], R& a) {
  const R rho = U[0], ux = U[1] / rho, uy = U[2] / rho;
  const R P = (R(2) - R(1)) * (U[3] - R(0.5) * rho * (ux * ux + uy * uy));
  const R un = d == 0 ? ux : uy;
  F[0] = rho * un;
  F[1] = U[1] * un + (d == 0 ? P : R(0));
  F[2] = U[2] * un + (d == 1 ? P : R(0));
  F[3] = un * (U[3] + P);
  a = fabs(un) + sqrt(R(2) * P / rho);
}

// Phi(U)(c): CWENO3 face states per component, local Lax-Friedrichs flux at
// the four faces of the cell, divergence (Eq. semidiscrete Euler).
template <typename R>
__device__ void euler_phi_cell(const Geo& g, const double* __restrict__ U, int c, R epsw, R (&phi)[4]) {
  const int i = c % g.nx, j = c / g.nx;
#pragma unroll
  for (int q = 0; q < 4; ++q) phi[q] = R(0);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    int cell[5];
#pragma unroll
    for (int t = 0; t < 5; ++t)
      cell[t] = d == 0 ? j * g.nx + nb(i + t - 2, g.nx, g.bcx) : nb(j + t - 2, g.ny, g.bcy) * g.nx + i;
    R q[5][4];
#pragma unroll
    for (int t = 0; t < 5; ++t)
#pragma unroll
      for (int m = 0; m < 4; ++m) q[t][m] = (R)U[(size_t)m * g.nc + cell[t]];
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
    const R am = fmax(aLm, aRm), ap = fmax(aLp, aRp);
    const R ih = R(1) / (R)(d == 0 ? g.dx : g.dy);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const R Fm = R(0.5) * (FLm[m] + FRm[m]) - R(0.5) * am * (Rm[m] - Lm[m]);
      const R Fp = R(0.5) * (FLp[m] + FRp[m]) - R(0.5) * ap * (Rp[m] - Lp[m]);
      phi[m] += (Fp - Fm) * ih;
    }
  }
}

// U^(i)(c) = U^n(c) - sum_j coef_j Phi_j(c) for a fluid cell, after storing
// Phi_{i-1}(c) when requested (Eqs. RKEuler, RKEuler_2).
template <typename R>
__device__ void euler_cell(const StageArgs& A, const View& V, int c, double (&Uc)[4]) {
  const size_t nc = V.g.nc;
  if (A.phi_store >= 0) {
    R phi[4];
    euler_phi_cell<R>(V.g, A.U_prev, c, (R)V.m.eps_w, phi);
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

// Primitive variables of U (Sec. 2): u = m/rho, T = (E - rho |u|^2/2)/rho.
ESBGK_DEV void prim_of(const double (&U)[4], double& rho, double& ux, double& uy, double& T) {
  rho = U[0];
  ux = U[1] / rho;
  uy = U[2] / rho;
  T = (U[3] - 0.5 * rho * (ux * ux + uy * uy)) / rho;
}

// ---------------------------------------------------------------------------
// Kinetic cell of a stage (or of the final combination).
template <typename S>
__device__ void kinetic_cell(const StageArgs& A, const View& V, int c, CellShared& sh,
                             typename Real<S>::T* sm) {
  using R = typename Real<S>::T;
  const Geo& g = V.g;
  R* sfs = sm;
  R* sL = sm + g.nvv;
  R* sG = sm + 2 * g.nvv;
  R* sc0 = sm + 3 * g.nvv;
  const size_t o0 = (size_t)c * g.nvv;
  size_t o[8];
  stencil_offsets(g, c, o);
  const S* fsrc = (const S*)A.f_src;
  const S* sbase = (const S*)A.star_base;
  const bool base_is_src = A.star_base == A.f_src;
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv;
  const R idx = (R)(1.0 / g.dx), idy = (R)(1.0 / g.dy), epsw = (R)V.m.eps_w, cL = (R)A.star_cL;

  // pass 1: transport of the previous stage, f*, moments of f*
  R m[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) m[n] = R(0);
  for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
    const int kx = k % g.nv, ky = k / g.nv;
    const R vx = v0 + R(kx) * dv, vy = v0 + R(ky) * dv;
    R L = R(0), q0 = R(0);
    if (fsrc) L = transport_at<S, R>(fsrc, o0, o, k, vx, vy, idx, idy, epsw, q0);
    const R base = base_is_src ? q0 : ld(sbase + o0 + k);
    const R fs = base + cL * L;
    sfs[k] = fs;
    sL[k] = L;
    sc0[k] = q0;
    m[0] += fs;
    m[1] += vx * fs;
    m[2] += vy * fs;
    m[3] += vx * vx * fs;
    m[4] += vx * vy * fs;
    m[5] += vy * vy * fs;
  }
  block_sum<6>(m, sh.red, sh.tot);

  const bool relax = A.h_coef > 0.0;
  const bool proj = relax || A.need_q;
  if (threadIdx.x == 0) {
    double mom[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) mom[n] = g.w * sh.tot[n];
    const double nu = V.m.tau / V.eps[c];
    sh.nu = nu;
    sh.h = A.h_coef * nu;
    int ok = 1;
    if (proj) ok = cell_tensor(sh, mom, V.m.beta, sh.h, relax) ? 1 : 0;
    sh.ok = ok;
    // conserved variables of f* = those of f^(i) (the relaxation conserves them)
    sh.U[0] = mom[0];
    sh.U[1] = mom[1];
    sh.U[2] = mom[2];
    sh.U[3] = 0.5 * (mom[3] + mom[5]);
  }
  __syncthreads();
  if (proj && sh.ok) gauss_project<R>(g, sh, sG);
  if (proj && threadIdx.x == 0 && !sh.ok) report_error(V.err, kErrNonRealizable, c);

  // pass 3: G_hat, implicit relaxation, Q, accumulators, outputs
  const bool doproj = proj && sh.ok;
  R a[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) a[n] = (R)sh.a[n];
  const R h = (R)sh.h, inv1h = R(1) / (R(1) + h), nu = (R)sh.nu;
  S* fout = (S*)A.f_out;
  for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
    const R fs = sfs[k], L = sL[k];
    R fnew = fs, Q = R(0);
    if (doproj) {
      const R Gh = ghat_at<R>(g, sh, a, sG[k], k);
      // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f) = nu (G_hat - f*)/(1 + h)
      if (relax) fnew = (fs + h * Gh) * inv1h;
      Q = nu * (Gh - fs) * inv1h;
    }
    if (fout) st(fout + o0 + k, fnew);
    for (int t = 0; t < A.nacc; ++t) {
      const S* ai = (const S*)A.acc_in[t];
      const R base = ai == fsrc ? sc0[k] : ldc(ai + o0 + k);
      st((S*)A.acc_out[t] + o0 + k, base + (R)A.acc_cL[t] * L + (R)A.acc_cQ[t] * Q);
    }
  }
  if (threadIdx.x == 0) {
    const size_t nc = g.nc;
#pragma unroll
    for (int q = 0; q < 4; ++q) A.U_out[q * nc + c] = A.kin_u_moments ? sh.U[q] : A.Un[q * nc + c];
  }
}

// Buffer cell of a stage: Euler update (thread 0), then f := M_hat[U]
// (Eq. Coupling_FluKin) over the velocities when filling is on.
template <typename S>
__device__ void buffer_cell(const StageArgs& A, const View& V, int c, CellShared& sh,
                            typename Real<S>::T* sm) {
  using R = typename Real<S>::T;
  const Geo& g = V.g;
  if (threadIdx.x == 0) {
    double Uc[4];
    euler_cell<R>(A, V, c, Uc);
    if (!A.hoc) {
#pragma unroll
      for (int q = 0; q < 4; ++q) Uc[q] = A.Un[(size_t)q * g.nc + c];
    }
    double rho, ux, uy, T;
    prim_of(Uc, rho, ux, uy, T);
    sh.ok = A.fill ? (cell_maxwell(sh, rho, ux, uy, T) ? 1 : 0) : 1;
  }
  __syncthreads();
  if (!A.fill) return;
  if (!sh.ok) {
    if (threadIdx.x == 0) report_error(V.err, kErrNonRealizable, c);
    return;
  }
  R* sG = sm;
  gauss_project<R>(g, sh, sG);
  R a[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) a[n] = (R)sh.a[n];
  S* fout = (S*)A.f_out;
  const size_t o0 = (size_t)c * g.nvv;
  for (int k = threadIdx.x; k < g.nvv; k += kThreads) st(fout + o0 + k, ghat_at<R>(g, sh, a, sG[k], k));
}

template <typename S>
__global__ void __launch_bounds__(kThreads) stage_kernel(StageArgs A, View V) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ CellShared sh;
  R* sm = reinterpret_cast<R*>(dsm);
  const int nK = V.counts[0], nB = V.counts[1], nF = V.counts[2];
  const int nFc = (nF + kThreads - 1) / kThreads;
  const int total = nK + nB + nFc;
  long long mine = 0, fills = 0;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    if (u < nK) {
      kinetic_cell<S>(A, V, V.klist[u], sh, sm);
      ++mine;
    } else if (u < nK + nB) {
      buffer_cell<S>(A, V, V.blist[u - nK], sh, sm);
      fills += A.fill ? 1 : 0;
    } else {
      const int q = (u - nK - nB) * kThreads + threadIdx.x;
      if (q < nF) {
        double Uc[4];
        euler_cell<R>(A, V, V.flist[q], Uc);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && A.ctr) {
    if (mine && A.f_src) atomicAdd((unsigned long long*)A.ctr, (unsigned long long)mine);
    if (fills) atomicAdd((unsigned long long*)A.ctr + 1, (unsigned long long)fills);
  }
}

// ---------------------------------------------------------------------------
// Fill f := M_hat[U] in the cells of two lists and copy U^n -> U^(1) in all
// cells (start of a step), and remember the regime map.
template <typename S>
__global__ void __launch_bounds__(kThreads) prep_kernel(PrepArgs P, View V) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ CellShared sh;
  R* sG = reinterpret_cast<R*>(dsm);
  const Geo& g = V.g;
  const int n1 = P.count1 ? *P.count1 : 0, n2 = P.count2 ? *P.count2 : 0;
  const int nCopy = P.copy_to ? (g.nc + kThreads - 1) / kThreads : 0;
  const int total = n1 + n2 + nCopy;
  S* f = (S*)P.f;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    if (u < n1 + n2) {
      const int c = u < n1 ? P.list1[u] : P.list2[u - n1];
      if (threadIdx.x == 0) {
        double Uc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) Uc[q] = P.U[(size_t)q * g.nc + c];
        double rho, ux, uy, T;
        prim_of(Uc, rho, ux, uy, T);
        sh.ok = cell_maxwell(sh, rho, ux, uy, T) ? 1 : 0;
        if (!sh.ok) report_error(V.err, kErrNonRealizable, c);
      }
      __syncthreads();
      if (sh.ok) {
        gauss_project<R>(g, sh, sG);
        R a[6];
#pragma unroll
        for (int n = 0; n < 6; ++n) a[n] = (R)sh.a[n];
        const size_t o0 = (size_t)c * g.nvv;
        for (int k = threadIdx.x; k < g.nvv; k += kThreads) st(f + o0 + k, ghat_at<R>(g, sh, a, sG[k], k));
      }
    } else {
      const int c = (u - n1 - n2) * kThreads + threadIdx.x;
      if (c < g.nc) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P.copy_to[(size_t)q * g.nc + c] = P.U[(size_t)q * g.nc + c];
        if (P.flags_prev) P.flags_prev[c] = V.flags[c];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// L1 deviation ||f - M_hat[f]||_{L1_v} of the kinetic cells (Eq. eqKintoFluid1).
template <typename S>
__global__ void __launch_bounds__(kThreads) l1_kernel(const void* fptr, double* L1, View V) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ CellShared sh;
  R* sf = reinterpret_cast<R*>(dsm);
  R* sG = sf + V.g.nvv;
  const Geo& g = V.g;
  const S* f = (const S*)fptr;
  const int nK = V.counts[0];
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv;
  for (int u = blockIdx.x; u < nK; u += gridDim.x) {
    const int c = V.klist[u];
    const size_t o0 = (size_t)c * g.nvv;
    R m[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) m[n] = R(0);
    for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
      const R vx = v0 + R(k % g.nv) * dv, vy = v0 + R(k / g.nv) * dv;
      const R x = ld(f + o0 + k);
      sf[k] = x;
      m[0] += x;
      m[1] += vx * x;
      m[2] += vy * x;
      m[3] += vx * vx * x;
      m[4] += vx * vy * x;
      m[5] += vy * vy * x;
    }
    block_sum<6>(m, sh.red, sh.tot);
    if (threadIdx.x == 0) {
      double mom[6];
#pragma unroll
      for (int n = 0; n < 6; ++n) mom[n] = g.w * sh.tot[n];
      // Maxwellian of f's own moments: the ES tensor with beta = 0
      sh.ok = cell_tensor(sh, mom, 0.0, 0.0, false) ? 1 : 0;
      if (!sh.ok) report_error(V.err, kErrNonRealizable, c);
    }
    __syncthreads();
    if (sh.ok) {
      gauss_project<R>(g, sh, sG);
      R a[6];
#pragma unroll
      for (int n = 0; n < 6; ++n) a[n] = (R)sh.a[n];
      R s[1] = {R(0)};
      for (int k = threadIdx.x; k < g.nvv; k += kThreads) s[0] += fabs(sf[k] - ghat_at<R>(g, sh, a, sG[k], k));
      block_sum<1>(s, sh.red, sh.tot);
      if (threadIdx.x == 0) L1[c] = g.w * sh.tot[0];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Relaxation of independent cells (entry point esbgk_relax_cells).
template <typename S>
__global__ void __launch_bounds__(kThreads) relax_cells_kernel(const S* fstar, const double* h, int n, Geo g,
                                                                double beta, S* fout, S* gout) {
  using R = typename Real<S>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ CellShared sh;
  R* sf = reinterpret_cast<R*>(dsm);
  R* sG = sf + g.nvv;
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv;
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const size_t o0 = (size_t)c * g.nvv;
    R m[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) m[q] = R(0);
    for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
      const R vx = v0 + R(k % g.nv) * dv, vy = v0 + R(k / g.nv) * dv;
      const R x = ld(fstar + o0 + k);
      sf[k] = x;
      m[0] += x;
      m[1] += vx * x;
      m[2] += vy * x;
      m[3] += vx * vx * x;
      m[4] += vx * vy * x;
      m[5] += vy * vy * x;
    }
    block_sum<6>(m, sh.red, sh.tot);
    if (threadIdx.x == 0) {
      double mom[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) mom[q] = g.w * sh.tot[q];
      sh.h = h[c];
      sh.ok = cell_tensor(sh, mom, beta, sh.h, true) ? 1 : 0;
    }
    __syncthreads();
    if (sh.ok) gauss_project<R>(g, sh, sG);
    const R nan = R(__int_as_float(0x7fc00000));
    R a[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) a[q] = (R)sh.a[q];
    const R hh = (R)sh.h, inv1h = R(1) / (R(1) + hh);
    for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
      if (sh.ok) {
        const R Gh = ghat_at<R>(g, sh, a, sG[k], k);
        st(fout + o0 + k, (sf[k] + hh * Gh) * inv1h);
        st(gout + o0 + k, Gh);
      } else {
        st(fout + o0 + k, nan);
        st(gout + o0 + k, nan);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// U := moments(f) in the kinetic cells (Eq. Coupling_KinFlu).
template <typename S>
__global__ void __launch_bounds__(kThreads) moments_kernel(const void* fptr, double* U, View V) {
  using R = typename Real<S>::T;
  __shared__ CellShared sh;
  const Geo& g = V.g;
  const S* f = (const S*)fptr;
  const R v0 = (R)(-g.vmax + 0.5 * g.dv), dv = (R)g.dv;
  for (int u = blockIdx.x; u < V.counts[0]; u += gridDim.x) {
    const int c = V.klist[u];
    const size_t o0 = (size_t)c * g.nvv;
    R m[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) m[n] = R(0);
    for (int k = threadIdx.x; k < g.nvv; k += kThreads) {
      const R vx = v0 + R(k % g.nv) * dv, vy = v0 + R(k / g.nv) * dv;
      const R x = ld(f + o0 + k);
      m[0] += x;
      m[1] += vx * x;
      m[2] += vy * x;
      m[3] += vx * vx * x;
      m[4] += vx * vy * x;
      m[5] += vy * vy * x;
    }
    block_sum<6>(m, sh.red, sh.tot);
    if (threadIdx.x == 0) {
      U[c] = g.w * sh.tot[0];
      U[g.nc + c] = g.w * sh.tot[1];
      U[2 * (size_t)g.nc + c] = g.w * sh.tot[2];
      U[3 * (size_t)g.nc + c] = 0.5 * g.w * (sh.tot[3] + sh.tot[5]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers for storage type S.
template <typename S>
struct Launch {
  using R = typename Real<S>::T;
  static size_t smem_stage(const Geo& g) { return 4 * (size_t)g.nvv * sizeof(R); }
  static size_t smem_two(const Geo& g) { return 2 * (size_t)g.nvv * sizeof(R); }

  static cudaError_t setup(const Geo& g) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(stage_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_stage(g))) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(prep_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_two(g))) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(l1_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_two(g))) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(relax_cells_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_two(g));
  }
  static int blocks_per_sm(const Geo& g) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<S>, kThreads, smem_stage(g));
    return nb < 1 ? 1 : nb;
  }
  static void stage(const StageArgs& A, const View& V, int grid, cudaStream_t s) {
    stage_kernel<S><<<grid, kThreads, smem_stage(V.g), s>>>(A, V);
  }
  static void prep(const PrepArgs& P, const View& V, int grid, cudaStream_t s) {
    prep_kernel<S><<<grid, kThreads, smem_two(V.g), s>>>(P, V);
  }
  static void l1(const void* f, double* L1, const View& V, int grid, cudaStream_t s) {
    l1_kernel<S><<<grid, kThreads, smem_two(V.g), s>>>(f, L1, V);
  }
  static void relax_cells(const void* fs, const double* h, int n, const Geo& g, double beta, void* fo, void* go,
                          int grid, cudaStream_t s) {
    relax_cells_kernel<S><<<grid, kThreads, smem_two(g), s>>>((const S*)fs, h, n, g, beta, (S*)fo, (S*)go);
  }
  static void moments(const void* f, double* U, const View& V, int grid, cudaStream_t s) {
    moments_kernel<S><<<grid, kThreads, 0, s>>>(f, U, V);
  }
};

#define ESBGK_INSTANTIATE(S, NAME)                                                  \
  const Launchers NAME = {sizeof(S),          &Launch<S>::setup,  &Launch<S>::blocks_per_sm, \
                          &Launch<S>::stage,  &Launch<S>::prep,   &Launch<S>::l1,            \
                          &Launch<S>::relax_cells, &Launch<S>::moments};

}  // namespace esbgk
