// tile_impl.cuh -- the tiled stage kernel for regions where every cell is kinetic.
//
// Included by kernels_impl.cuh.  A CTA owns a tile of E x E cells (E = 2 or
// 4), one warp per cell (as in stage_kernel), and walks the velocity nodes in
// chunks of 16 E node pairs.  Per chunk:
//
//   walk phase   -- the transport of Sec. 3.2 computed per face, not per cell:
//                   a thread takes one node pair and one tile row (x walk) or
//                   column (y walk), loads the E + 3 upwind-relevant values
//                   of the line (two ghost cells each side), forms the E + 1
//                   CWENO3 face values of its E cells once each, and writes
//                   v (F_{i+1/2} - F_{i-1/2}) / dx of its E cells to shared
//                   memory.  A cell's 4 faces are shared with its neighbours,
//                   so the tile computes 2 (E + 1) / E faces per cell and node
//                   instead of 4; neighbouring faces also share one
//                   difference and its smoothness term.
//   cell phase   -- the warp of each cell adds its x and y parts, forms
//                   f* = base + c_L L and the partial accumulators, keeps f*
//                   in shared memory and sums the moments of f* (Eq. RKEI1).
//
// After the last chunk each warp finishes its own cell exactly as
// kinetic_cell_vec does: moments -> ES parameters -> projection -> implicit
// relaxation, Q and accumulators (Sec. 2, 3.3, Eq. RKEI1-RKEI2).
//
// The face value uses the same CWENO3 weights as cweno_face, rearranged so
// that the upwind direction is a per-thread coefficient instead of a branch:
// with dl = b - a, dr = c - b, x = (eps+dl^2)^2, y = (eps+dr^2)^2,
// z = (eps + 13/3 (dr-dl)^2 + 1/4 (dl+dr)^2)^2,
//   face = b + 1/2 [x y (5 dr + dl)/3 + z (y dl + x dr)] / [2 x y + z (x + y)]
//        = b + 1/2 [x y (5 dr + dl)/6 + (z/2) (y dl + x dr)] / [x y + (z/2) (x + y)],
// and the face of the mirrored stencil (c, b, a) -- the other upwind
// direction -- is the same expression with 5 dr + dl replaced by 5 dl + dr and
// the sign of the correction flipped.  With t = d^2 + eps of the two
// differences, 13/3 (dr-dl)^2 + 1/4 (dl+dr)^2 + eps
//   = 55/12 (t_l + t_r) - 49/6 dl dr + eps (1 - 55/6),
// so the squares already formed for x and y give z.  Paired FP32 instructions
// take register pairs only, so every constant factor sits in a scalar
// multiply-add or in a per-thread coefficient pair.
#pragma once

namespace esbgk {

// A tile of E x E cells, one warp per cell.  A chunk holds 16 E node pairs,
// so that the 2 E lines (E rows, E columns) of a chunk give every thread one
// walk, and every lane of the cell phase E / 2 pairs.  E = 4: one CTA of 16
// warps per SM, 2.5 faces per cell and node.  E = 2 (four CTAs of 4 warps per
// SM, whose load and compute phases interleave, 3 faces per cell and node)
// took 4.38 ms per step of the 256^2 x 48^2 all-kinetic run against 3.24 ms
// for E = 4: twice the chunks per cell and 5 instead of 3.5 line loads per
// value; the library builds E = 4 only.
template <int E>
struct TileShape {
  static constexpr int kCells = E * E;
  static constexpr int kThreads = 32 * kCells;
  static constexpr int kPairs = 16 * E;
  static constexpr int kHalves = kPairs / 32;
  static constexpr int kMinBlocks = E == 4 ? 1 : 4;
  static_assert(2 * E * kPairs == kThreads && kPairs % 32 == 0, "one walk per thread and chunk");
};
constexpr int kTileEdge = 4;

// Two lanes of arithmetic: paired FP32 instructions for float, component-wise
// for double.
template <typename R> struct PairT;
template <> struct PairT<float> { using T = float2; };
template <> struct PairT<double> { using T = double2; };

ESBGK_DEV float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
ESBGK_DEV float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
ESBGK_DEV float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
ESBGK_DEV float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
ESBGK_DEV float2 pdiv(float2 a, float2 b) { return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y)); }
ESBGK_DEV float2 psplat(float a) { return make_float2(a, a); }
ESBGK_DEV double2 pfma(double2 a, double2 b, double2 c) { return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)); }
ESBGK_DEV double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
ESBGK_DEV double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
ESBGK_DEV double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
ESBGK_DEV double2 pdiv(double2 a, double2 b) { return make_double2(a.x / b.x, a.y / b.y); }
ESBGK_DEV double2 psplat(double a) { return make_double2(a, a); }
ESBGK_DEV float2 mk2(float a, float b) { return make_float2(a, b); }
ESBGK_DEV double2 mk2(double a, double b) { return make_double2(a, b); }

// G_hat at the two nodes of a pair of one velocity row (cx: v_x - u_x of
// both, cy: v_y - u_y): the per-row terms once, then both nodes.
ESBGK_DEV GhatRow ghat_row2(const CellPar<float>& P, float cy) { return ghat_row(P, cy); }
ESBGK_DEV float2 ghat2(const CellPar<float>& P, const GhatRow& r, float2 cx) { return ghat_pair(P, r, cx); }
struct GhatRowD {
  double cy;
};
ESBGK_DEV GhatRowD ghat_row2(const CellPar<double>&, double cy) { return GhatRowD{cy}; }
ESBGK_DEV double2 ghat2(const CellPar<double>& P, const GhatRowD& r, double2 cx) {
  return make_double2(ghat(P, cx.x, r.cy), ghat(P, cx.y, r.cy));
}

// A node pair (two consecutive nodes of one velocity row) of storage type S,
// in the arithmetic type.
template <typename S> struct PairIO;
template <>
struct PairIO<float> {
  static ESBGK_DEV float2 ld(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
  static ESBGK_DEV float2 ldc(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static ESBGK_DEV void st(float* p, float2 v, uint32_t) { *reinterpret_cast<float2*>(p) = v; }
};
template <>
struct PairIO<double> {
  static ESBGK_DEV double2 ld(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
  static ESBGK_DEV double2 ldc(const double* p) { return *reinterpret_cast<const double2*>(p); }
  static ESBGK_DEV void st(double* p, double2 v, uint32_t) { *reinterpret_cast<double2*>(p) = v; }
};
template <>
struct PairIO<__nv_bfloat16> {
  static ESBGK_DEV float2 unpack(unsigned t) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t));
  }
  static ESBGK_DEV float2 ld(const __nv_bfloat16* p) { return unpack(__ldg(reinterpret_cast<const unsigned*>(p))); }
  static ESBGK_DEV float2 ldc(const __nv_bfloat16* p) { return unpack(*reinterpret_cast<const unsigned*>(p)); }
  // stochastic rounding (key: random bits for the pair)
  static ESBGK_DEV void st(__nv_bfloat16* p, float2 v, uint32_t key) {
    const uint32_t r = mix32(key);
    *reinterpret_cast<unsigned*>(p) = (uint32_t)bf16_sr_bits(v.x, r) | ((uint32_t)bf16_sr_bits(v.y, r >> 16) << 16);
  }
};

// Reciprocal: the hardware approximation for float (rcp.approx, at most
// 1 ulp), an IEEE division for double.
ESBGK_DEV float rcp_(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
ESBGK_DEV double rcp_(double x) { return 1.0 / x; }

// Constant pairs of walk_line (register pairs, formed once per kernel):
// m1 = (-1, -1), eps2 = eps_w, C1 = 55/(12 sqrt 2), C2 = -49/(6 sqrt 2),
// c3 = eps_w (1 - 55/6)/sqrt 2.
template <typename P>
struct WalkConst {
  P m1, eps2, C1, C2, c3;
};
template <typename P, typename R>
ESBGK_DEV WalkConst<P> walk_const(R epsw) {
  return WalkConst<P>{psplat(R(-1)), psplat(epsw), psplat(R(55.0 / 12.0 / 1.4142135623730951)),
                      psplat(R(-49.0 / 6.0 / 1.4142135623730951)),
                      psplat(epsw * R((1.0 - 55.0 / 6.0) / 1.4142135623730951))};
}

// Upwind CWENO3 faces along one line of the tile and the transport of its NL
// cells.  u[0..NL+2]: the pair's values in NL+3 consecutive cells, shifted so
// that u[q+1] is the upwind cell of face q, the face between tile cells q-1
// and q (q = 0..NL): cells -2..NL of the line for velocities toward
// increasing cell index, -1..NL+1 otherwise.  Per node of the pair: (cA, cB) = (1/6, 5/6) toward
// increasing index, (5/6, 1/6) the other way, sgnh = +1/2 / -1/2; K the
// constant pairs (walk_const); vs = v / h.  Writes
// v (face_{q+1} - face_q) / h of tile cell q to out[q * stride].  The faces
// are formed in order, each from the difference behind and the difference
// ahead of its upwind cell, so only two differences are live at a time.
template <typename P, typename R, int NL>
ESBGK_DEV void walk_line(const P (&u)[NL + 3], const WalkConst<P>& K, P cA, P cB, P sgnh, P vs, P* out, int stride) {
  P dl = pfma(u[0], K.m1, u[1]);
  P tl = pfma(dl, dl, K.eps2);
  P sl = pmul(tl, tl);
  P prev = psplat(R(0));
#pragma unroll
  for (int q = 0; q <= NL; ++q) {
    const P dr = pfma(u[q + 1], K.m1, u[q + 2]);
    const P tr = pfma(dr, dr, K.eps2);
    const P sr = pmul(tr, tr);
    const P T = padd(tl, tr), Pd = pmul(dl, dr);
    // sqrt(z/2), then z/2
    const P z0 = pfma(T, K.C1, pfma(Pd, K.C2, K.c3));
    const P zh = pmul(z0, z0);
    const P xy = pmul(sl, sr);
    const P p = pfma(cA, dl, pmul(cB, dr));         // (5 d_r + d_l)/6, upwind orientation
    const P tt = pfma(sr, dl, pmul(sl, dr));         // y d_l + x d_r, either orientation
    const P num = pfma(xy, p, pmul(zh, tt));
    const P den = pfma(zh, padd(sl, sr), xy);
    const P face = pfma(sgnh, pmul(num, mk2(rcp_(den.x), rcp_(den.y))), u[q + 1]);
    if (q > 0) out[(q - 1) * stride] = pmul(vs, pfma(prev, K.m1, face));
    prev = face;
    dl = dr;
    tl = tr;
    sl = sr;
  }
}

// The discrete Gaussian of a cell at node pairs, for the projection sums and
// the relaxation pass of the tiled kernel (float arithmetic).  Both passes
// must see the same G at every node, or the projected Gaussian's moments miss
// their targets by rounding each stage, so both evaluate it through these
// functions, from the same per-cell pairs and the same velocity-table entries.
// The per-cell parameters are splatted into register pairs once per cell
// (paired instructions take register pairs only).
struct Gauss2 {
  float2 qxx, qxy, qyy, pref, isT, u;  // u = (u_x, u_y)
};
ESBGK_DEV Gauss2 gauss2(const CellPar<float>& P) {
  return Gauss2{splat2(P.qxx), splat2(P.qxy), splat2(P.qyy), splat2(P.pref), splat2(P.isT), make_float2(P.ux, P.uy)};
}
// Row terms of a group of 4 nodes whose first node has velocity v = (v_x, v_y)
// (a velocity-table entry): c0 = v_x - u_x of the group's pairs (nodes 0, 1)
// and c1 (nodes 2, 3), cyy = (v_y - u_y, v_y - u_y), and the exponent's
// row parts qy = qyy cy^2, qc = qxy cy.  m1 = (-1, -1), off = (0, dv),
// two = (2 dv, 2 dv).
struct Row2 {
  float2 c0, c1, cyy, qy, qc;
};
ESBGK_DEV Row2 row2(const Gauss2& Q, float2 v, float2 m1, float2 off, float2 two) {
  const float2 cg = __ffma2_rn(Q.u, m1, v);
  Row2 r;
  r.c0 = __fadd2_rn(splat2(cg.x), off);
  r.c1 = __fadd2_rn(r.c0, two);
  r.cyy = splat2(cg.y);
  r.qy = __fmul2_rn(Q.qyy, __fmul2_rn(r.cyy, r.cyy));
  r.qc = __fmul2_rn(Q.qxy, r.cyy);
  return r;
}
// G and x = (v_x - u_x)/sqrt(T) at the pair cx of a row.
ESBGK_DEV void gauss_pair(const Gauss2& Q, const Row2& r, float2 cx, float2& G, float2& x) {
  const float2 e = __ffma2_rn(Q.qxx, __fmul2_rn(cx, cx), __ffma2_rn(r.qc, cx, r.qy));
  G = __fmul2_rn(Q.pref, make_float2(exp2r(e.x), exp2r(e.y)));
  x = __fmul2_rn(cx, Q.isT);
}

// Projection sums of the discrete Gaussian (the 15 sums of project), factored
// by velocity rows: along a row segment v_y is fixed, so the lane sums G x^p
// (p = 0..4) over the segment's node pairs and then adds them times y^q into
// the 15 sums once per segment.  A segment is a run of whole groups of 4
// nodes (the relaxation pass's groups): a half row when N_v/2 is a multiple
// of 4, else a whole row (N_v a multiple of 4).  The sums are then solved as
// in project.
ESBGK_DEV bool project_rows(const Geo& g, int lane, CellPar<float>& P, const float2* vt) {
  const int seg = (g.nv / 2) % 4 == 0 ? g.nv / 2 : g.nv, nseg = g.nvv / seg;
  const Gauss2 Q = gauss2(P);
  const float2 m1 = splat2(-1.0f), off = make_float2(0.0f, g.fdv), two = splat2(2.0f * g.fdv);
  float s[15];
#pragma unroll
  for (int n = 0; n < 15; ++n) s[n] = 0.0f;
#pragma unroll 1
  for (int sg = lane; sg < nseg; sg += 32) {
    const int k0 = sg * seg;  // first node of the segment (segments tile the rows in order)
    float2 R0 = splat2(0.0f), R1 = R0, R2 = R0, R3 = R0, R4 = R0;
    float cy = 0.0f;
#pragma unroll 2
    for (int m = 0; m < seg; m += 4) {
      const Row2 r = row2(Q, vt[(k0 + m) >> 1], m1, off, two);
      cy = r.cyy.x;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 G, x;
        gauss_pair(Q, r, h ? r.c1 : r.c0, G, x);
        const float2 t1 = __fmul2_rn(G, x), t2 = __fmul2_rn(t1, x), t3 = __fmul2_rn(t2, x);
        R0 = __fadd2_rn(R0, G);
        R1 = __fadd2_rn(R1, t1);
        R2 = __fadd2_rn(R2, t2);
        R3 = __fadd2_rn(R3, t3);
        R4 = __ffma2_rn(t3, x, R4);
      }
    }
    const float y = cy * P.isT;
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
#pragma unroll
  for (int n = 0; n < 15; ++n) s[n] = warp_sum(s[n]) * g.fw;
  return project_solve<float, 32>(s, lane, P, 0xffffffffu);
}

// Shared-memory layout of the tiled kernel (dynamic): f* of each cell, the
// x and y transport parts of two chunks, and the per-pair velocities.
template <typename R, int E>
struct TileSmem {
  static size_t bytes(const Geo& g) {
    using P = typename PairT<R>::T;
    using T = TileShape<E>;
    return (size_t)T::kCells * g.nvv * sizeof(R) + 2 * 2 * T::kCells * T::kPairs * sizeof(P) +
           (size_t)(g.nvv / 2) * sizeof(P);
  }
};

// Tile t of the grid (tiles of E x E cells): its first cell (i0, j0).
template <int E>
ESBGK_DEV void tile_origin(const Geo& g, int t, int& i0, int& j0) {
  const int tx = (g.nx + E - 1) / E;
  i0 = (t % tx) * E;
  j0 = (t / tx) * E;
}

// SX: some node pair straddles v_x = 0 (N_v/2 odd): its two nodes take
// opposite upwind directions in the x walk.  Otherwise N_v is a multiple of 4
// and the per-cell passes take groups of 4 nodes (two pairs of one row).
// COMP: compensated moment sums (Model::comp_moments, float arithmetic).
//
// Latency: the walk's line values are loaded one chunk ahead into the other
// of two register sets, so they are in flight while the previous chunk
// computes; the cell phase's base and accumulator values are loaded at the
// start of their chunk, before its walk.
template <typename S, int M, bool SX, bool COMP, int E>
__global__ void __launch_bounds__(TileShape<E>::kThreads, TileShape<E>::kMinBlocks)
    tile_stage_kernel(StageArgs A, View V) {
  using TS = TileShape<E>;
  constexpr int kTileCells = TS::kCells, kTileThreads = TS::kThreads, kTilePairs = TS::kPairs;
  constexpr int NH = TS::kHalves;
  using R = typename Real<S>::T;
  using P = typename PairT<R>::T;
  using IO = PairIO<S>;
  using MT = ModeT<M>;
  constexpr bool relax = MT::relax;
  constexpr int nacc = MT::nacc;
  constexpr int NW = SX ? E + 4 : E + 3;            // line values a walk loads
  constexpr int NB = 1 + (MT::acc_src ? 0 : nacc);  // base and accumulator inputs of a cell pair
  constexpr bool F32 = std::is_same<R, float>::value;
  extern __shared__ __align__(16) unsigned char dsm[];
  const Geo& g = V.g;
  const int nvv = g.nvv, npairs = nvv / 2;
  R* fs_all = reinterpret_cast<R*>(dsm);
  P* Lb = reinterpret_cast<P*>(dsm + (size_t)kTileCells * nvv * sizeof(R));  // [2][2][cells][pairs]
  P* vt = Lb + 2 * 2 * kTileCells * kTilePairs;                              // [npairs] (v_x of the first node, v_y)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const R v0 = pick<R>(g.v0, g.fv0), dv = pick<R>(g.dv, g.fdv);
  for (int p = tid; p < npairs; p += kTileThreads) {
    const int k = 2 * p, ky = k / g.nv;
    P v;
    v.x = v0 + R(k - ky * g.nv) * dv;
    v.y = v0 + R(ky) * dv;
    vt[p] = v;
  }
  __syncthreads();

  const S* fsrc = (const S*)A.f_src;
  const S* bsrc = MT::base_src ? fsrc : (const S*)A.star_base;
  S* fout = (S*)A.f_out;
  const R idx = pick<R>(1.0 / g.dx, g.fidx), idy = pick<R>(1.0 / g.dy, g.fidy);
  const P cL2 = psplat(pick<R>(A.star_cL, A.f_star_cL));
  const WalkConst<P> WK = walk_const<P, R>(pick<R>(V.m.eps_w, V.m.feps_w));
  const S* ain[nacc > 0 ? nacc : 1];
  S* aout[nacc > 0 ? nacc : 1];
  P aL2[nacc > 0 ? nacc : 1];
  R aQ[nacc > 0 ? nacc : 1];
#pragma unroll
  for (int t = 0; t < nacc; ++t) {
    ain[t] = (const S*)A.acc_in[t];
    aout[t] = (S*)A.acc_out[t];
    aL2[t] = psplat(pick<R>(A.acc_cL[t], A.f_acc_cL[t]));
    aQ[t] = pick<R>(A.acc_cQ[t], A.f_acc_cQ[t]);
  }
  const uint32_t s0 = A.seed ? mix32(*A.seed * 0x632be5abu + A.sid) : 0u;

  // walk of this thread: x walks (one per tile row) then y walks (one per column)
  const bool xwalk = tid < E * kTilePairs;
  const int wline = xwalk ? tid / kTilePairs : (tid - E * kTilePairs) / kTilePairs;
  const int wpair = tid % kTilePairs;
  const R wscale = xwalk ? idx : idy;
  const int wstride = xwalk ? kTilePairs : E * kTilePairs;
  const int wout = xwalk ? (wline * E) * kTilePairs + wpair : wline * kTilePairs + wpair;
  // cell of this warp in the cell phase
  const int ci = warp % E, cj = warp / E;
  R* fs = fs_all + (size_t)warp * nvv;

  constexpr int W3 = SX ? 2 : 4;  // nodes per group of the per-cell passes
  const int ntiles = ((g.nx + E - 1) / E) * ((g.ny + E - 1) / E);
  const int nchunks = (npairs + kTilePairs - 1) / kTilePairs;
  long long mine = 0;
  // chunks walked so far: the parity picks the transport buffer, so a buffer
  // is rewritten only after the barrier of the chunk that follows its readers
  int gch = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int i0, j0;
    tile_origin<E>(g, tile, i0, j0);
    // the walk's line: cells -2..E+1 of it (boundary conditions applied)
    const bool wvalid = xwalk ? (j0 + wline < g.ny) : (i0 + wline < g.nx);
    unsigned wb[E + 4];
#pragma unroll
    for (int q = 0; q < E + 4; ++q) {
      const int c = xwalk ? (j0 + wline) * g.nx + nb(i0 - 2 + q, g.nx, g.bcx)
                          : nb(j0 - 2 + q, g.ny, g.bcy) * g.nx + (i0 + wline);
      wb[q] = wvalid ? (unsigned)c * (unsigned)nvv : 0u;
    }
    // this warp's cell
    const int ccell = (j0 + cj) * g.nx + (i0 + ci);
    const bool cvalid = (i0 + ci < g.nx) && (j0 + cj < g.ny);
    const unsigned o0 = cvalid ? (unsigned)ccell * (unsigned)nvv : 0u;
    R u0x = R(0), u0y = R(0);
    if (cvalid) ref_velocity(A.U_prev, g.nc, ccell, u0x, u0y);
    const P u0p = mk2(u0x, u0y), offp = mk2(R(0), dv);
    P m2[6];
    R mc_s[COMP ? 6 : 1], mc_c[COMP ? 6 : 1];  // compensated sums: running sum and compensation
#pragma unroll
    for (int n = 0; n < 6; ++n) m2[n] = psplat(R(0));
#pragma unroll
    for (int n = 0; n < (COMP ? 6 : 1); ++n) mc_s[n] = mc_c[n] = R(0);

    // two register sets of the walk's loads; chunk c uses set c & 1
    P wA[NW], wB[NW], cb[NH][NB];
    P vwA = psplat(R(0)), vwB = psplat(R(0));
    bool okA = false, okB = false;
    auto load_walk = [&](int ch, P (&w)[NW], P& vw, bool& ok) {
      const int pr = ch * kTilePairs + wpair;
      ok = wvalid && pr < npairs;
      if (ok) {
        const P v = vt[pr];
        vw = xwalk ? mk2(v.x, v.x + dv) : mk2(v.y, v.y);
        const unsigned k = 2u * pr;
        if (SX) {
#pragma unroll
          for (int q = 0; q < NW; ++q) w[q] = IO::ld(fsrc + wb[q] + k);
        } else {
          // the window starts one cell further for velocities toward lower indices
          const bool pos = vw.x > R(0);
#pragma unroll
          for (int q = 0; q < NW; ++q) w[q] = IO::ld(fsrc + (pos ? wb[q] : wb[q + 1]) + k);
        }
      }
    };
    auto load_cell = [&](int ch) {
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int prc = ch * kTilePairs + lane + 32 * h;
        if (cvalid && prc < npairs) {
          const unsigned k = 2u * prc;
          cb[h][0] = IO::ld(bsrc + o0 + k);
#pragma unroll
          for (int t = 1; t < NB; ++t) cb[h][t] = IO::ld(ain[t - 1] + o0 + k);
        }
      }
    };
    auto chunk = [&](int ch, const P (&w)[NW], P vw, bool ok) {
      load_cell(ch);
      P* Lx = Lb + (size_t)(gch & 1) * 2 * kTileCells * kTilePairs;
      P* Ly = Lx + kTileCells * kTilePairs;
      // --- walk phase
      if (ok) {
        P u[E + 3];
        if (SX) {
          // per node: the window of its own direction
#pragma unroll
          for (int q = 0; q < E + 3; ++q) {
            u[q].x = vw.x > R(0) ? w[q].x : w[q + 1].x;
            u[q].y = vw.y > R(0) ? w[q].y : w[q + 1].y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < E + 3; ++q) u[q] = w[q];
        }
        const bool px = vw.x > R(0), py = vw.y > R(0);
        const P cA = mk2(px ? R(1.0 / 6.0) : R(5.0 / 6.0), py ? R(1.0 / 6.0) : R(5.0 / 6.0));
        const P cB = mk2(px ? R(5.0 / 6.0) : R(1.0 / 6.0), py ? R(5.0 / 6.0) : R(1.0 / 6.0));
        const P sgnh = mk2(px ? R(0.5) : R(-0.5), py ? R(0.5) : R(-0.5));
        walk_line<P, R, E>(u, WK, cA, cB, sgnh, mk2(vw.x * wscale, vw.y * wscale), (xwalk ? Lx : Ly) + wout, wstride);
      }
      __syncthreads();
      // --- cell phase: lanes take pairs lane + 32 h of the chunk
      if (cvalid) {
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const int pl = lane + 32 * h, pr = ch * kTilePairs + pl;
          if (pr >= npairs) continue;
          const unsigned k = 2u * pr;
          const P L = padd(Lx[warp * kTilePairs + pl], Ly[warp * kTilePairs + pl]);
          const P base = cb[h][0];
          const P F = pfma(cL2, L, base);
          const uint32_t kb = s0 + ((o0 + k) << 3);
#pragma unroll
          for (int t = 0; t < nacc; ++t) {
            const P ai = MT::acc_src ? base : cb[h][1 + t];
            IO::st(aout[t] + o0 + k, pfma(aL2[t], L, ai), kb + 1 + t);
          }
          if (relax)
            *reinterpret_cast<P*>(fs + k) = F;
          else
            IO::st(fout + o0 + k, F, kb);
          const P v = vt[pr];
          P cx, cy;
          if constexpr (F32) {
            const float2 cg = __ffma2_rn(u0p, WK.m1, v);  // (v_x - u0_x, v_y - u0_y)
            cx = __fadd2_rn(splat2(cg.x), offp);
            cy = splat2(cg.y);
          } else {
            const R cxa = v.x - u0x;
            cx = mk2(cxa, cxa + dv);
            cy = psplat(v.y - u0y);
          }
          const P xf = pmul(cx, F), yf = pmul(cy, F);
          m2[0] = padd(m2[0], F);
          m2[1] = padd(m2[1], xf);
          m2[2] = padd(m2[2], yf);
          m2[3] = pfma(cx, xf, m2[3]);
          m2[4] = pfma(cy, xf, m2[4]);
          m2[5] = pfma(cy, yf, m2[5]);
        }
        if constexpr (COMP && F32) {
          // the paired runs of 16 nodes per lane into a Neumaier accumulator
          constexpr int kFlush = 8 / NH;  // chunks
          if ((ch & (kFlush - 1)) == kFlush - 1 || ch == nchunks - 1) {
#pragma unroll
            for (int n = 0; n < 6; ++n) {
              comp_add(mc_s[n], mc_c[n], m2[n].x + m2[n].y);
              m2[n] = psplat(R(0));
            }
          }
        }
      }
      ++gch;
    };
    load_walk(0, wA, vwA, okA);
    for (int ch = 0; ch < nchunks; ch += 2) {
      if (ch + 1 < nchunks) load_walk(ch + 1, wB, vwB, okB);
      chunk(ch, wA, vwA, okA);
      if (ch + 1 < nchunks) {
        if (ch + 2 < nchunks) load_walk(ch + 2, wA, vwA, okA);
        chunk(ch + 1, wB, vwB, okB);
      }
    }
    // --- the cell: moments, ES parameters, projection, relaxation
    if (cvalid) {
      R m[6];
      if constexpr (COMP && F32) {
#pragma unroll
        for (int n = 0; n < 6; ++n) m[n] = group_sum_comp<32>(mc_s[n], mc_c[n], 0xffffffffu);
      } else {
#pragma unroll
        for (int n = 0; n < 6; ++n) m[n] = warp_sum(m2[n].x + m2[n].y);
      }
      if (lane == 0) {
        double Uc[4];
        cons_from_sums(m, u0x, u0y, g.w, Uc);
        const size_t nc = g.nc;
#pragma unroll
        for (int q = 0; q < 4; ++q) A.U_out[q * nc + ccell] = A.kin_u_moments ? Uc[q] : A.Un[q * nc + ccell];
      }
      if (A.f_src) ++mine;
      if (relax) {
        __syncwarp();
        const R tau = pick<R>(V.m.tau, V.m.ftau) * (V.m.tau_rho ? pick<R>(g.w, g.fw) * m[0] : R(1));
        const R nu = tau / R(V.eps[ccell]), hh = pick<R>(A.h_coef, A.f_h_coef) * nu;
        CellPar<R> Pp;
        bool ok = es_params<R>(m, u0x, u0y, pick<R>(g.w, g.fw), pick<R>(V.m.beta, V.m.fbeta), hh, true, Pp);
        if constexpr (F32 && !SX) {
          if (ok) ok = project_rows(g, lane, Pp, vt);
        } else {
          if (ok) ok = project<R, W3, 32>(g, lane, Pp);
        }
        if (!ok && lane == 0) report_error(V.err, kErrNonRealizable, ccell);
        const R inv1h = R(1) / (R(1) + hh);
        const P h2 = psplat(hh), i2 = psplat(inv1h), nq = psplat(nu * inv1h);
        P aQ2[nacc > 0 ? nacc : 1];
#pragma unroll
        for (int t = 0; t < nacc; ++t) aQ2[t] = psplat(aQ[t]);
        const int ngroups = nvv / W3;
        if constexpr (F32 && !SX) {
          // float: the Gaussian through the projection's own pair functions
          // (bit-identical G), two register sets of the partial accumulators
          // loaded one group ahead
          const Gauss2 Q2 = gauss2(Pp);
          const float2 m1 = splat2(-1.0f), off = make_float2(0.0f, dv), two = splat2(2.0f * dv);
          const float2 a3 = splat2(Pp.a[3]), a1 = splat2(Pp.a[1]), a4 = splat2(Pp.a[4]);
          const float2 a2 = splat2(Pp.a[2]), a5 = splat2(Pp.a[5]), a0p1 = splat2(1.0f + Pp.a[0]);
          P paA[2][nacc > 0 ? nacc : 1], paB[2][nacc > 0 ? nacc : 1];
          auto load_g = [&](int gi, P (&pa)[2][nacc > 0 ? nacc : 1]) {
            const unsigned kg = (unsigned)gi * 4u;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
              for (int t = 0; t < nacc; ++t) pa[j][t] = IO::ldc(aout[t] + o0 + kg + 2 * j);
          };
          auto relax_g = [&](int gi, const P (&pa)[2][nacc > 0 ? nacc : 1]) {
            const unsigned kg = (unsigned)gi * 4u;
            const Row2 r = row2(Q2, vt[kg / 2], m1, off, two);
            const float2 y = __fmul2_rn(r.cyy, Q2.isT);
            const float2 c0 = __ffma2_rn(__ffma2_rn(a5, y, a2), y, a0p1), c1 = __ffma2_rn(a4, y, a1);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const unsigned k = kg + 2 * j;
              const float2 F = *reinterpret_cast<const float2*>(fs + k);
              float2 Fn = F, Q = splat2(0.0f);
              if (ok) {
                float2 G, x;
                gauss_pair(Q2, r, j ? r.c1 : r.c0, G, x);
                const float2 Gh = __fmul2_rn(G, __ffma2_rn(__ffma2_rn(a3, x, c1), x, c0));
                // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f*)/(1 + h)
                Fn = __fmul2_rn(__ffma2_rn(h2, Gh, F), i2);
                Q = __fmul2_rn(nq, __ffma2_rn(F, m1, Gh));
              }
              const uint32_t kb = s0 + ((o0 + k) << 3);
              IO::st(fout + o0 + k, Fn, kb);
#pragma unroll
              for (int t = 0; t < nacc; ++t) IO::st(aout[t] + o0 + k, __ffma2_rn(aQ2[t], Q, pa[j][t]), kb + 4 + t);
            }
          };
          if (lane < ngroups) load_g(lane, paA);
          for (int gi = lane; gi < ngroups; gi += 64) {
            if (gi + 32 < ngroups) load_g(gi + 32, paB);
            relax_g(gi, paA);
            if (gi + 32 < ngroups) {
              if (gi + 64 < ngroups) load_g(gi + 64, paA);
              relax_g(gi + 32, paB);
            }
          }
          continue;
        }
        // accumulator partials of the next group loaded one iteration ahead
        P pan[W3 / 2][nacc > 0 ? nacc : 1];
        auto load_pa = [&](int gi) {
#pragma unroll
          for (int j = 0; j < W3 / 2; ++j)
#pragma unroll
            for (int t = 0; t < nacc; ++t) pan[j][t] = IO::ldc(aout[t] + o0 + (unsigned)gi * W3 + 2 * j);
        };
        if (lane < ngroups) load_pa(lane);
        for (int gi = lane; gi < ngroups; gi += 32) {
          P pa[W3 / 2][nacc > 0 ? nacc : 1];
#pragma unroll
          for (int j = 0; j < W3 / 2; ++j)
#pragma unroll
            for (int t = 0; t < nacc; ++t) pa[j][t] = pan[j][t];
          if (gi + 32 < ngroups) load_pa(gi + 32);
          const unsigned kg = (unsigned)gi * W3;
          const P v = vt[kg / 2];
          // v_x - u_x of the group's first node and v_y - u_y, as the projection forms them
          const R cxg = v.x - Pp.ux, cy = v.y - Pp.uy;
          const auto row = ghat_row2(Pp, cy);
#pragma unroll
          for (int j = 0; j < W3; j += 2) {
            const unsigned k = kg + j;
            const P F = *reinterpret_cast<const P*>(fs + k);
            P Fn = F, Q = psplat(R(0));
            if (ok) {
              const R cxa = cxg + R(j) * dv;
              const P Gh = ghat2(Pp, row, mk2(cxa, cxa + dv));
              // f = (f* + h G_hat)/(1 + h); Q = nu (G_hat - f*)/(1 + h)
              Fn = pmul(pfma(h2, Gh, F), i2);
              Q = pmul(nq, mk2(Gh.x - F.x, Gh.y - F.y));
            }
            const uint32_t kb = s0 + ((o0 + k) << 3);
            IO::st(fout + o0 + k, Fn, kb);
#pragma unroll
            for (int t = 0; t < nacc; ++t) IO::st(aout[t] + o0 + k, pfma(aQ2[t], Q, pa[j / 2][t]), kb + 4 + t);
          }
        }
      }
    }
  }
  if (lane == 0 && A.ctr && mine) atomicAdd((unsigned long long*)A.ctr, (unsigned long long)mine);
}

}  // namespace esbgk
