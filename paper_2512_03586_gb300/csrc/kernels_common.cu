// kernels_common.cu -- precision-independent kernels: state set-up, regime
// criteria, compaction of the regime map, macroscopic read-out and totals.
#include "launch.h"

namespace esbgk {

// U = (rho, rho u, 1/2 rho |u|^2 + rho T) from (rho, u, T) (Sec. 2, d_v = 2).
__global__ void init_state_kernel(const double* __restrict__ prim, const uint8_t* __restrict__ kin_in,
                                  double* Un, double* eps, uint8_t* flags, uint8_t* flags_prev, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double rho = prim[c], ux = prim[nc + c], uy = prim[2 * (size_t)nc + c], T = prim[3 * (size_t)nc + c];
  Un[c] = rho;
  Un[nc + c] = rho * ux;
  Un[2 * (size_t)nc + c] = rho * uy;
  Un[3 * (size_t)nc + c] = 0.5 * rho * (ux * ux + uy * uy) + rho * T;
  eps[c] = prim[4 * (size_t)nc + c];
  const uint8_t k = kin_in ? (kin_in[c] ? 1 : 0) : 1;
  flags[c] = k;
  flags_prev[c] = k;
}

__global__ void clear_solid_kernel(uint8_t* flags, uint8_t* flags_prev, const uint8_t* __restrict__ solid, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && solid[c]) flags[c] = flags_prev[c] = 0;
}

void launch_clear_solid(uint8_t* flags, uint8_t* flags_prev, const uint8_t* solid, int nc, cudaStream_t s) {
  clear_solid_kernel<<<(nc + 255) / 256, 256, 0, s>>>(flags, flags_prev, solid, nc);
}

void launch_init_state(const double* prim, const uint8_t* kin_in, double* Un, double* eps, uint8_t* flags,
                       uint8_t* flags_prev, int nc, cudaStream_t s) {
  init_state_kernel<<<(nc + 255) / 256, 256, 0, s>>>(prim, kin_in, Un, eps, flags, flags_prev, nc);
}

// Reciprocal and square root in the criterion's arithmetic type.
// In float64 these are the correctly rounded IEEE operations: the criterion
// meets arguments far outside float's range (lambda_A^2 ~ 1e-52 where the
// flow is uniform), where a float seed refined by Newton steps would start at
// 0 or infinity.  One cell's criterion costs a few of them per step.
__device__ __forceinline__ double crit_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float crit_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double crit_sqrt(double x) { return x > 0.0 ? sqrt(x) : 0.0; }
__device__ __forceinline__ float crit_sqrt(float x) { return x > 0.0f ? sqrtf(x) : 0.0f; }

// Regime criteria of Sec. 3.1.2 for one cell.  X = I - S_1 with
//   S_1 = I - eps D(u) mu/(rho T) - 2/3 (eps kappa/(rho T^{3/2}))^2 grad T grad T^T,
//   mu/(rho T) = 1/(tau (1-beta)),  kappa/(rho T^{3/2}) = 5/2 /(tau sqrt T),
//   D = grad u + grad u^T - 2/3 div u I;
// lambda_A = max |eig X| = |tr X|/2 + sqrt(((X_xx - X_yy)/2)^2 + X_xy^2).
// Gradients: central differences of cell-centre u and T, ghost cells by BC.
// New flag (Eqs. crit:CompEuler, eqKintoFluid1):
//   lambda_A > eta   or   (kinetic and ||f - M||_1 > delta).
// R: float64 for FP64 storage, float32 for FP32/BF16 storage (the decision is
// then taken in the storage's working precision; GB300's FP64 pipe is narrow).
template <typename R>
__device__ __forceinline__ void prim_cell(const double* __restrict__ Un, size_t nc, int cc, R& rho, R& ux, R& uy,
                                          R& T) {
  rho = (R)Un[cc];
  const R mx = (R)Un[nc + cc], my = (R)Un[2 * nc + cc], E = (R)Un[3 * nc + cc];
  const R ir = crit_rcp(rho);
  ux = mx * ir;
  uy = my * ir;
  T = (E - R(0.5) * rho * (ux * ux + uy * uy)) * ir;
}

// The criterion of cell c from the primitive variables of the cell (0) and
// of its east, west, north and south neighbours.
template <typename R>
struct Prims {
  R rho, ux, uy, T;
};
template <typename R>
__device__ __forceinline__ void flags_from_prims(const View& V, const double* __restrict__ L1in, double* L1out,
                                                 double* lamA, uint8_t* flags_out, int c, bool plain,
                                                 const Prims<R>& P0, const Prims<R>& PE, const Prims<R>& PW,
                                                 const Prims<R>& PN, const Prims<R>& PS) {
  const Geo& g = V.g;
  const R i2dx = R(0.5 / g.dx), i2dy = R(0.5 / g.dy);
  const R dudx = (PE.ux - PW.ux) * i2dx, dudy = (PN.ux - PS.ux) * i2dy;
  const R dvdx = (PE.uy - PW.uy) * i2dx, dvdy = (PN.uy - PS.uy) * i2dy;
  const R dTdx = (PE.T - PW.T) * i2dx, dTdy = (PN.T - PS.T) * i2dy;
  const R div = dudx + dvdy;
  const R Dxx = R(2) * dudx - R(2.0 / 3.0) * div;
  const R Dyy = R(2) * dvdy - R(2.0 / 3.0) * div;
  const R Dxy = dudy + dvdx;
  const R eps = (R)V.eps[c];
  const R tau = V.m.tau_rho ? R(V.m.tau) * P0.rho : R(V.m.tau);  // tau * rho with the density model
  const R c1 = eps / (tau * (R(1) - R(V.m.beta)));
  const R kk = R(2.5) * eps * crit_rcp(tau * crit_sqrt(P0.T));
  const R c2 = R(2.0 / 3.0) * kk * kk;
  const R Xxx = c1 * Dxx + c2 * dTdx * dTdx;
  const R Xxy = c1 * Dxy + c2 * dTdx * dTdy;
  const R Xyy = c1 * Dyy + c2 * dTdy * dTdy;
  const R mean = R(0.5) * (Xxx + Xyy), half = R(0.5) * (Xxx - Xyy);
  const R lam = rabs(mean) + crit_sqrt(half * half + Xxy * Xxy);
  const uint8_t kin = V.flags[c];
  const double l1 = kin ? L1in[c] : 0.0;
  lamA[c] = (double)lam;
  L1out[c] = l1;
  if (plain) flags_out[c] = (lam > R(V.m.eta_factor) * eps) || (kin && l1 > V.m.delta) ? 1 : 0;
}

template <typename R>
__device__ void flags_cell(const View& V, const double* __restrict__ Un, const double* __restrict__ L1in,
                           double* L1out, double* lamA, uint8_t* flags_out, int c, bool plain) {
  const Geo& g = V.g;
  const int i = c % g.nx, j = c / g.nx;
  Prims<R> P0, PE, PW, PN, PS;
  prim_cell(Un, g.nc, j * g.nx + nb(i + 1, g.nx, g.bcx), PE.rho, PE.ux, PE.uy, PE.T);
  prim_cell(Un, g.nc, j * g.nx + nb(i - 1, g.nx, g.bcx), PW.rho, PW.ux, PW.uy, PW.T);
  prim_cell(Un, g.nc, nb(j + 1, g.ny, g.bcy) * g.nx + i, PN.rho, PN.ux, PN.uy, PN.T);
  prim_cell(Un, g.nc, nb(j - 1, g.ny, g.bcy) * g.nx + i, PS.rho, PS.ux, PS.uy, PS.T);
  prim_cell(Un, g.nc, c, P0.rho, P0.ux, P0.uy, P0.T);
  flags_from_prims(V, L1in, L1out, lamA, flags_out, c, plain, P0, PE, PW, PN, PS);
}

// Tiled form: a CTA owns FX x FY cells and computes the primitive variables
// of the tile and its one-cell halo once, in shared memory.
constexpr int kFX = 16, kFY = 8;
template <typename R>
__global__ void __launch_bounds__(kFX* kFY) flags_tile_kernel(View V, const double* __restrict__ Un,
                                                              const double* __restrict__ L1in, double* L1out,
                                                              double* lamA, uint8_t* flags_out) {
  constexpr int HX = kFX + 2, HY = kFY + 2;
  __shared__ Prims<R> sp[HX * HY];
  const Geo& g = V.g;
  const int i0 = blockIdx.x * kFX - 1, j0 = blockIdx.y * kFY - 1;
  const int t = threadIdx.y * kFX + threadIdx.x;
  for (int h = t; h < HX * HY; h += kFX * kFY) {
    const int ci = nb(i0 + h % HX, g.nx, g.bcx), cj = nb(j0 + h / HX, g.ny, g.bcy);
    prim_cell(Un, g.nc, cj * g.nx + ci, sp[h].rho, sp[h].ux, sp[h].uy, sp[h].T);
  }
  __syncthreads();
  const int i = blockIdx.x * kFX + threadIdx.x, j = blockIdx.y * kFY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int h0 = (threadIdx.y + 1) * HX + threadIdx.x + 1;
  flags_from_prims(V, L1in, L1out, lamA, flags_out, j * g.nx + i, true, sp[h0], sp[h0 + 1], sp[h0 - 1], sp[h0 + HX],
                   sp[h0 - HX]);
}

// The criterion with solid obstacles: a neighbour across a wall is the
// mirror state of the cell's own side (the stencil maps of View, normal
// velocity reversed); solid cells are never kinetic.
template <typename R>
__global__ void flags_walls_kernel(View V, const double* __restrict__ Un, const double* __restrict__ L1in,
                                   double* L1out, double* lamA, uint8_t* flags_out) {
  const Geo& g = V.g;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.nc) return;
  if (V.solid[c]) {
    lamA[c] = 0.0;
    L1out[c] = 0.0;
    flags_out[c] = 0;
    return;
  }
  Prims<R> P0, Pn[4];  // east, west, north, south: offsets +1, -1 along x, then y
  prim_cell(Un, g.nc, c, P0.rho, P0.ux, P0.uy, P0.T);
  const int slot[4] = {2, 1, 2, 1};  // offset index of +1 and -1 in (-2, -1, +1, +2)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int axis = q / 2, at = (axis * 4 + slot[q]) * g.nc + c;
    Prims<R>& P = Pn[q];
    prim_cell(Un, g.nc, V.wsrc[at], P.rho, P.ux, P.uy, P.T);
    if (V.wrefl[at]) {
      if (axis == 0)
        P.ux = -P.ux;
      else
        P.uy = -P.uy;
    }
  }
  flags_from_prims(V, L1in, L1out, lamA, flags_out, c, true, P0, Pn[0], Pn[1], Pn[2], Pn[3]);
}

void launch_flags(const View& V, const double* Un, const double* L1in, double* L1out, double* lamA,
                  uint8_t* flags_out, bool fp32, cudaStream_t s) {
  const dim3 grid((V.g.nx + kFX - 1) / kFX, (V.g.ny + kFY - 1) / kFY);
  if (V.wsrc) {
    const int nb = (V.g.nc + 255) / 256;
    if (fp32)
      flags_walls_kernel<float><<<nb, 256, 0, s>>>(V, Un, L1in, L1out, lamA, flags_out);
    else
      flags_walls_kernel<double><<<nb, 256, 0, s>>>(V, Un, L1in, L1out, lamA, flags_out);
    return;
  }
  if (fp32)
    flags_tile_kernel<float><<<grid, dim3(kFX, kFY), 0, s>>>(V, Un, L1in, L1out, lamA, flags_out);
  else
    flags_tile_kernel<double><<<grid, dim3(kFX, kFY), 0, s>>>(V, Un, L1in, L1out, lamA, flags_out);
}

// Category of each cell: 0 kinetic, 1 buffer (fluid cell inside the two-cell
// cross stencil of a kinetic cell, Remark rem_coupling), 2 other fluid; bit 2
// (value 4) marks a kinetic cell that was fluid in the previous step.
__device__ int category_of(const Geo& g, const uint8_t* __restrict__ flags, const uint8_t* __restrict__ prev, int c,
                           const uint8_t* __restrict__ solid = nullptr) {
  if (solid && solid[c]) return 3;  // solid: in no list
  if (flags[c]) return prev[c] ? 0 : 4;
  const int i = c % g.nx, j = c / g.nx;
  bool hit = false;
  const int d[4] = {-2, -1, 1, 2};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    hit |= flags[j * g.nx + nb(i + d[q], g.nx, g.bcx)] != 0;
    hit |= flags[nb(j + d[q], g.ny, g.bcy) * g.nx + i] != 0;
  }
  return hit ? 1 : 2;
}

__device__ void categorize_cell(const Geo& g, const uint8_t* __restrict__ flags, const uint8_t* __restrict__ prev,
                                uint8_t* cat, int c) {
  cat[c] = (uint8_t)category_of(g, flags, prev, c);
}

__global__ void categorize_kernel(Geo g, const uint8_t* __restrict__ flags, const uint8_t* __restrict__ prev,
                                  uint8_t* cat, const uint8_t* __restrict__ solid) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.nc) cat[c] = (uint8_t)category_of(g, flags, prev, c, solid);
}

void launch_categorize(const View& V, const uint8_t* flags, const uint8_t* flags_prev, uint8_t* cat,
                       cudaStream_t s) {
  categorize_kernel<<<(V.g.nc + 255) / 256, 256, 0, s>>>(V.g, flags, flags_prev, cat, V.solid);
}

// Deterministic stream compaction of the categories into the lists of
// kinetic, buffer, fluid and converted cells (ascending cell order), one CTA.
constexpr int kScanThreads = 1024;

__device__ int block_exclusive_scan(int v, int* sm, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kScanThreads / 32 ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sm[32 + lane] = w;
  }
  __syncthreads();
  total = sm[32 + 31];
  const int before = warp > 0 ? sm[32 + warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// Each thread owns a run of `chunk` categories (a multiple of 16, so the run
// is read with 16-byte loads); two passes: count, scan, emit.
__device__ __forceinline__ void count_cats(uint32_t w, int base, int nc, int (&n)[4]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int t = (w >> (8 * b)) & 0xff;
    const bool in = base + b < nc;
    n[0] += in && (t & 3) == 0;
    n[1] += in && t == 1;
    n[2] += in && t == 2;
    n[3] += in && t == 4;
  }
}

__device__ void compact_block(const uint8_t* __restrict__ cat, int nc, int* klist, int* blist, int* flist,
                              int* clist, int* counts) {
  __shared__ int sm[64];
  const int chunk = ((nc + kScanThreads - 1) / kScanThreads + 15) / 16 * 16;
  const int lo = threadIdx.x * chunk;
  const int hi = min(nc, lo + chunk);
  const uint4* v = reinterpret_cast<const uint4*>(cat);
  int n[4] = {0, 0, 0, 0};
#pragma unroll 4
  for (int c = lo; c < hi; c += 16) {
    const uint4 x = v[c / 16];
    count_cats(x.x, c, nc, n);
    count_cats(x.y, c + 4, nc, n);
    count_cats(x.z, c + 8, nc, n);
    count_cats(x.w, c + 12, nc, n);
  }
  int off[4], tot[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) off[q] = block_exclusive_scan(n[q], sm, tot[q]);
  for (int c = lo; c < hi; c += 16) {
    const uint4 x = v[c / 16];
    const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      const int cc = c + b;
      if (cc >= nc) break;
      const int t = (w4[b / 4] >> (8 * (b % 4))) & 0xff;
      if ((t & 3) == 0) klist[off[0]++] = cc;
      if (t == 1) blist[off[1]++] = cc;
      if (t == 2) flist[off[2]++] = cc;
      if (t == 4) clist[off[3]++] = cc;
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) counts[q] = tot[q];
  }
}

__global__ void __launch_bounds__(kScanThreads) compact_kernel(const uint8_t* __restrict__ cat, int nc, int* klist,
                                                               int* blist, int* flist, int* clist, int* counts) {
  compact_block(cat, nc, klist, blist, flist, clist, counts);
}

void launch_compact(const uint8_t* cat, int nc, int* klist, int* blist, int* flist, int* clist, int* counts,
                    cudaStream_t s) {
  compact_kernel<<<1, kScanThreads, 0, s>>>(cat, nc, klist, blist, flist, clist, counts);
}

// Categories and lists in two launches, in ascending cell order: kernel 1
// writes each cell's category and the per-block counts of the four lists;
// kernel 2 gives every block its offsets (sum of the counts of the blocks
// before it), scans its cells and writes them.  Block b covers cells
// [b * kCatBlock, (b + 1) * kCatBlock).
constexpr int kCatBlock = 1024;

__global__ void __launch_bounds__(kCatBlock) categorize_count_kernel(Geo g, const uint8_t* __restrict__ flags,
                                                                     const uint8_t* __restrict__ prev, uint8_t* cat,
                                                                     int* block_counts,
                                                                     const uint8_t* __restrict__ solid) {
  __shared__ int sc[4];
  if (threadIdx.x < 4) sc[threadIdx.x] = 0;
  __syncthreads();
  const int c = blockIdx.x * kCatBlock + threadIdx.x;
  const int t = c < g.nc ? category_of(g, flags, prev, c, solid) : -1;
  if (c < g.nc) cat[c] = (uint8_t)t;
  const unsigned full = 0xffffffffu;
  const unsigned m[4] = {__ballot_sync(full, t == 0 || t == 4), __ballot_sync(full, t == 1),
                         __ballot_sync(full, t == 2), __ballot_sync(full, t == 4)};
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (m[q]) atomicAdd(&sc[q], __popc(m[q]));
  __syncthreads();
  if (threadIdx.x < 4) block_counts[blockIdx.x * 4 + threadIdx.x] = sc[threadIdx.x];
}

__global__ void __launch_bounds__(kCatBlock) emit_lists_kernel(int nc, const uint8_t* __restrict__ cat,
                                                               const int* __restrict__ block_counts, int nblocks,
                                                               int* klist, int* blist, int* flist, int* clist,
                                                               int* counts) {
  __shared__ int base[4], tot[4];
  __shared__ int sm[64];
  if (threadIdx.x < 4) {
    int s = 0, all = 0;
    for (int b = 0; b < nblocks; ++b) {
      const int v = block_counts[b * 4 + threadIdx.x];
      if (b < (int)blockIdx.x) s += v;
      all += v;
    }
    base[threadIdx.x] = s;
    tot[threadIdx.x] = all;
  }
  __syncthreads();
  const int c = blockIdx.x * kCatBlock + threadIdx.x;
  const int t = c < nc ? cat[c] : -1;
  int* lists[4] = {klist, blist, flist, clist};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int in = q == 0 ? (t == 0 || t == 4) : (q == 1 ? t == 1 : (q == 2 ? t == 2 : t == 4));
    int total;
    const int off = block_exclusive_scan(in, sm, total);
    if (in) lists[q][base[q] + off] = c;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) counts[threadIdx.x] = tot[threadIdx.x];
}

void launch_categorize_compact(const View& V, const uint8_t* flags, const uint8_t* flags_prev, uint8_t* cat,
                               int* block_counts, int* klist, int* blist, int* flist, int* clist, int* counts,
                               cudaStream_t s) {
  const int nb = (V.g.nc + kCatBlock - 1) / kCatBlock;
  categorize_count_kernel<<<nb, kCatBlock, 0, s>>>(V.g, flags, flags_prev, cat, block_counts, V.solid);
  emit_lists_kernel<<<nb, kCatBlock, 0, s>>>(V.g.nc, cat, block_counts, nb, klist, blist, flist, clist, counts);
}

int categorize_blocks(int nc) { return (nc + kCatBlock - 1) / kCatBlock; }

__global__ void seed_advance_kernel(unsigned* seed) { *seed += 1u; }

void launch_seed_advance(unsigned* seed, cudaStream_t s) { seed_advance_kernel<<<1, 1, 0, s>>>(seed); }

// (rho, u_x, u_y, T) from U.
__global__ void prim_kernel(const double* __restrict__ Un, double* out, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double rho = Un[c], ux = Un[nc + c] / rho, uy = Un[2 * (size_t)nc + c] / rho;
  out[c] = rho;
  out[nc + c] = ux;
  out[2 * (size_t)nc + c] = uy;
  out[3 * (size_t)nc + c] = (Un[3 * (size_t)nc + c] - 0.5 * rho * (ux * ux + uy * uy)) / rho;
}

void launch_prim(const double* Un, double* out, int nc, cudaStream_t s) {
  prim_kernel<<<(nc + 255) / 256, 256, 0, s>>>(Un, out, nc);
}

// Global totals: fixed-order two-level sum of U over cells, times dx dy.
__global__ void totals_partial_kernel(const double* __restrict__ Un, const uint8_t* __restrict__ solid, int nc,
                                      double* partial) {
  __shared__ double red[4][256];
  double s[4] = {0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    if (solid && solid[c]) continue;  // solid cells hold no state
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += Un[(size_t)q * nc + c];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) partial[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void totals_final_kernel(const double* __restrict__ partial, int nb, double* out, double dxdy) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b * 4 + threadIdx.x];
    out[threadIdx.x] = s * dxdy;
  }
}

void launch_totals(const double* Un, const uint8_t* solid, int nc, double* partial, double* out, double dxdy,
                   int grid, cudaStream_t s) {
  totals_partial_kernel<<<grid, 256, 0, s>>>(Un, solid, nc, partial);
  totals_final_kernel<<<1, 32, 0, s>>>(partial, grid, out, dxdy);
}

// ---------------------------------------------------------------------------
// Batched regime update.

// L1 units: the kinetic cells of plain-switch cases whose L1 is not fresh.
__global__ void batch_l1_offsets_kernel(BatchTabs T) {
  if (threadIdx.x != 0) return;
  int acc = 0;
  for (int c = 0; c < T.n; ++c) {
    T.off_l1[c] = acc;
    const CaseRegime& R = T.reg[c];
    acc += (R.plain && !*R.l1_fresh) ? R.counts[0] : 0;
  }
  T.off_l1[T.n] = acc;
}

void launch_batch_l1_offsets(const BatchTabs& T, cudaStream_t s) { batch_l1_offsets_kernel<<<1, 32, 0, s>>>(T); }

template <typename R>
__global__ void batch_flags_kernel(BatchTabs T) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= T.total_cells) return;
  const int c = find_case(T.cell_off, T.n, u);
  const CaseRegime& C = T.reg[c];
  flags_cell<R>(C.V, C.Un, C.L1, C.L1, C.lamA, C.flags, u - T.cell_off[c], C.plain != 0);
}

void launch_batch_flags(const BatchTabs& T, cudaStream_t s) {
  if (T.fp32)
    batch_flags_kernel<float><<<(T.total_cells + 127) / 128, 128, 0, s>>>(T);
  else
    batch_flags_kernel<double><<<(T.total_cells + 127) / 128, 128, 0, s>>>(T);
}

__global__ void batch_categorize_kernel(BatchTabs T) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= T.total_cells) return;
  const int c = find_case(T.cell_off, T.n, u);
  const CaseRegime& R = T.reg[c];
  categorize_cell(R.V.g, R.flags, R.flags_prev, R.cat, u - T.cell_off[c]);
}

void launch_batch_categorize(const BatchTabs& T, cudaStream_t s) {
  batch_categorize_kernel<<<(T.total_cells + 255) / 256, 256, 0, s>>>(T);
}

__global__ void __launch_bounds__(kScanThreads) batch_compact_kernel(BatchTabs T) {
  const CaseRegime& R = T.reg[blockIdx.x];
  compact_block(R.cat, R.V.g.nc, R.klist, R.blist, R.flist, R.clist, R.counts);
}

void launch_batch_compact(const BatchTabs& T, cudaStream_t s) { batch_compact_kernel<<<T.n, kScanThreads, 0, s>>>(T); }

// Stage units (kinetic cells or pairs of them, buffer cells, chunks of 32
// fluid cells) and start-of-step units per case; marks L1 fresh where this
// step's final combination computes it.
__global__ void batch_offsets_kernel(BatchTabs T) {
  if (threadIdx.x != 0) return;
  int as[kNumVariants] = {}, ap = 0;
  for (int c = 0; c < T.n; ++c) {
    const CaseRegime& R = T.reg[c];
    const int* k = R.counts;
    for (int v = 0; v < kNumVariants; ++v) T.off_stage[v * (T.n + 1) + c] = as[v];
    T.off_prep[c] = ap;
    as[R.variant] += (variant_pairs(R.variant) ? (k[0] + 1) / 2 : k[0]) + k[1] + (k[2] + 31) / 32;
    ap += k[1] + (R.conv ? k[3] : 0) + (R.prep_copy ? (R.V.g.nc + 31) / 32 : 0);
    *R.l1_fresh = R.l1_next;
  }
  for (int v = 0; v < kNumVariants; ++v) T.off_stage[v * (T.n + 1) + T.n] = as[v];
  T.off_prep[T.n] = ap;
}

void launch_batch_offsets(const BatchTabs& T, cudaStream_t s) { batch_offsets_kernel<<<1, 32, 0, s>>>(T); }

__global__ void batch_seed_kernel(const CasePrep* cases, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (cases[i].P.seed) *cases[i].P.seed += 1u;
}

void launch_batch_seed_advance(const CasePrep* cases, int n, cudaStream_t s) {
  batch_seed_kernel<<<1, 128, 0, s>>>(cases, n);
}

// ---------------------------------------------------------------------------
// Probe of the bounded device waits: one CTA waits on a shared-memory barrier
// with the library's bounded wait; arrive = 0 leaves the barrier without its
// arrival, so the wait runs out and records kErrTimeout in the word.
__device__ int g_wait_probe_err;

__global__ void wait_probe_kernel(int arrive, unsigned limit) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    g_wait_probe_err = 0;
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    if (!mbar_wait(&bar, 0, limit)) g_wait_probe_err = kErrTimeout;
  }
}

cudaError_t launch_wait_probe(int arrive, unsigned limit, int* err_out, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(arrive, limit);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(err_out, g_wait_probe_err, sizeof(int));
  return e;
}

}  // namespace esbgk
