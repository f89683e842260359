// cnn.cu -- the learned regime switch: a 3-layer convolutional network that
// predicts from the macroscopic state of a 5 x 5 neighbourhood the flag the
// criterion of Sec. 3.1.2 will give a cell at the next step.  Forward pass,
// backward pass (input and weight gradients), class-weighted cross-entropy
// and Adam, all hand-written.  The two 3 x 3 convolutions are implicit GEMMs
// on the tensor cores (bf16 operands, float32 accumulation,
// mma.sync.m16n8k16); the 1 x 1 head, the loss and the optimizer are float32
// on the CUDA cores.
//
// The 32 -> 32 convolution of the forward pass and its input gradient run on
// the 5th-generation tensor cores (tcgen05.mma with a tensor-memory
// accumulator, halo staged by TMA tensor copies: conv32_tc_kernel); the
// 5 -> 32 forward convolution and the weight gradients use mma.sync (the
// 5 -> 32 layer on the tcgen05 kernel, nine MMAs per tile, took 51.2 us per
// training batch against 37.9 us).
//
// Tiling (mma.sync kernels): a CTA owns 8 x 16 output cells of one image; its 4 warps own two
// rows of 16 cells each (one m16 tile per row) and all 32 output channels
// (four n8 tiles).  The input halo (10 x 18 cells, channels contiguous, cell
// stride padded by 8 bf16 so that the fragment loads of the 8 row groups
// fall in distinct banks) and the whole weight matrix are staged in shared
// memory; the GEMM depth runs over 9 taps x the input channels.
#include "cnn.h"

#include <cuda.h>

#include <cstring>
#include <string>

#include "common.cuh"

#include "../../include/esbgk.h"

namespace esbgk {
namespace cnn {

namespace {

using bf = __nv_bfloat16;
constexpr int TH = 8, TW = 16, HH = TH + 2, HW = TW + 2;
constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t ld32(const bf* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf lo, bf hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D += A (16x16, row) * B (16x8, col), bf16 in, float32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Stage the (TH+2) x (TW+2) halo of an input tile ([img][H][W][CIN] bf16)
// into shared memory with cell stride CS; zeros outside the image.
template <int CIN, int CS>
__device__ void load_halo(const bf* __restrict__ in, int img, int H, int W, int ty0, int tx0, bf* s) {
  constexpr int P = CIN / 2;
  for (int i = threadIdx.x; i < HH * HW * P; i += blockDim.x) {
    const int cell = i / P, pr = i % P;
    const int gy = ty0 + cell / HW - 1, gx = tx0 + cell % HW - 1;
    uint32_t v = 0;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = ld32(in + (((size_t)img * H + gy) * W + gx) * CIN + 2 * pr);
    *reinterpret_cast<uint32_t*>(s + cell * CS + 2 * pr) = v;
  }
}

enum { kFwd = 0, kDgrad = 1 };

// out[cell][o] = sum_{tap, c} in[cell + off(tap)][c] * wk[o][tap*CIN + c]
// (+ bias, relu) -- MODE kFwd: relu(acc + bias[o]); kDgrad: acc masked by
// (mask[cell][o] > 0), the relu derivative of the layer below.
template <int CIN, int MODE>
__global__ void __launch_bounds__(kThreads) conv_kernel(const bf* __restrict__ in, const bf* __restrict__ wk,
                                                        const float* __restrict__ bias, int H, int W,
                                                        bf* __restrict__ out, const bf* __restrict__ mask) {
  constexpr int CS = CIN + 8, K = 9 * CIN, KS = K + 8;
  __shared__ __align__(16) bf s_in[HH * HW * CS];
  __shared__ __align__(16) bf s_w[kHid * KS];
  __shared__ float s_b[kHid];
  const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * TH, img = blockIdx.z;
  for (int i = threadIdx.x; i < kHid * K / 2; i += blockDim.x) {
    const int o = i / (K / 2), k = 2 * (i % (K / 2));
    *reinterpret_cast<uint32_t*>(s_w + o * KS + k) = ld32(wk + o * K + k);
  }
  if (threadIdx.x < kHid) s_b[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
  load_halo<CIN, CS>(in, img, H, W, ty0, tx0, s_in);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;

#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int ky = tap / 3, kx = tap % 3;
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      uint32_t a[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int hrow = 2 * warp + m + ky;
        const bf* p0 = s_in + (hrow * HW + g + kx) * CS + kc * 16 + 2 * q;
        const bf* p1 = p0 + 8 * CS;
        a[m][0] = ld32(p0);
        a[m][1] = ld32(p1);
        a[m][2] = ld32(p0 + 8);
        a[m][3] = ld32(p1 + 8);
      }
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const bf* pw = s_w + (n * 8 + g) * KS + tap * CIN + kc * 16 + 2 * q;
        const uint32_t b[2] = {ld32(pw), ld32(pw + 8)};
        mma16816(acc[0][n], a[0], b);
        mma16816(acc[1][n], a[1], b);
      }
    }
  }

#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int gy = ty0 + 2 * warp + m;
    if (gy >= H) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gx = tx0 + g + 8 * h;
      if (gx >= W) continue;
      const size_t cell = ((size_t)img * H + gy) * W + gx;
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const int o = n * 8 + 2 * q;
        float v0 = acc[m][n][2 * h] + s_b[o], v1 = acc[m][n][2 * h + 1] + s_b[o + 1];
        if (MODE == kFwd) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        } else {
          const bf* mk = mask + cell * kHid + o;
          if (!(__bfloat162float(mk[0]) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk[1]) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<uint32_t*>(out + cell * kHid + o) = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 32 -> 32 channel 3 x 3 convolution on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory).  A CTA owns a row segment of
// TC_M = 128 consecutive cells of one image row: D[128 cells][32 out] is the
// sum of 18 MMAs of depth 16 (9 taps x 32 input channels),
// A[128 cells][16] x B[16][32].
// Shared-memory operands use the no-swizzle K-major layout of 8-row x
// 16-byte core matrices:
//   A: the input halo, 3 rows x (TC_M + 2) cells, stored as 4 planes of 8
//      channels ([plane][row][cell][8]); the rows of a tap's A operand are
//      consecutive cells of one halo row, so a core matrix (8 cells x 8
//      channels) is 128 contiguous bytes, the next 8 cells follow at +128 B
//      (stride byte offset) and the next 8 channels at +plane (leading byte
//      offset); a tap is only a different start address.
//   B: the weights as [k group of 8][32 out][8]: core matrices at +128 B
//      along N and +512 B along K.
constexpr int TC_M = 128, TC_HW = TC_M + 2;
// bytes of one 8-channel plane (3 x TC_HW cells of 16 B), padded to 128 B:
// the tensor copies write each plane at a 128-byte aligned address
constexpr int TC_PLANE = (3 * TC_HW * 16 + 127) / 128 * 128;
constexpr unsigned kTcHaloBytes = 4u * 3u * TC_HW * 16u;  // the four planes' boxes
constexpr int TC_WBYTES = kK2 / 8 * 512;                                  // 36 k groups x 512 B
constexpr size_t kTcSmem = 4 * (size_t)TC_PLANE + TC_WBYTES;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start address, leading and stride byte offsets (all >> 4), descriptor
  // version 1, base offset 0, no swizzle
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: bf16 A and B (both K-major), f32
// accumulator, M = 128, N = 32.
constexpr uint32_t kTcIdesc = (1u << 4)                // D format f32
                              | (1u << 7) | (1u << 10)  // A, B bf16
                              | ((32u >> 3) << 17)      // N >> 3
                              | ((128u >> 4) << 24);    // M >> 4

// Persistent: a CTA stages the weights and allocates its accumulator once,
// then loops over row segments (segment t: image t / (H * segs), row and
// segment within it).  Per segment: stage the halo, one thread issues the
// MMAs and commits to the mbarrier (phase = the CTA's segment count & 1),
// every warp reads its 32 cells back.
// TMA: the halo comes by four tensor copies (one per 8-channel plane, box 8
// channels x TC_HW cells x 3 rows, zeros outside the image) completing on an
// mbarrier; the next tile's copies are issued as soon as the current tile's
// MMAs have read the halo, so they overlap the read-back.  Without a tensor
// map the threads stage the halo with plain loads.
// MODE kFwd: out = relu(acc + bias) (the forward 32 -> 32 layer, weights
// w2f); kDgrad: out = acc masked by (mask > 0), the input gradient of that
// layer (weights w2d: transposed channels, flipped taps; mask = its input
// activations, the ReLU derivative of the layer below).
template <bool TMA, int MODE>
__global__ void __launch_bounds__(128) conv32_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                        const bf* __restrict__ in, const bf* __restrict__ wk,
                                                        const float* __restrict__ bias, int n, int H, int W,
                                                        bf* __restrict__ out, const bf* __restrict__ mask,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sa = tsm;                 // A halo, 4 planes
  unsigned char* sb = tsm + 4 * TC_PLANE;  // B weights
  __shared__ __align__(8) unsigned long long mbar, tbar;
  __shared__ uint32_t tmem_base;
  __shared__ float s_b[kHid];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int segs = (W + TC_M - 1) / TC_M;
  const int total = n * H * segs;

  if (warp == 0) {  // 32 columns of tensor memory for the f32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&tbar, 1);
    mbar_init_fence();
  }
  if (MODE == kFwd && tid < kHid) s_b[tid] = bias[tid];
  // weights W2f[o][k] (k = tap*32 + c) -> [k/8][o][k%8], 16-byte pieces
  for (int i = tid; i < kHid * kK2 / 8; i += blockDim.x) {
    const int o = i / (kK2 / 8), kg = i % (kK2 / 8);
    *reinterpret_cast<uint4*>(sb + kg * 512 + o * 16) = *reinterpret_cast<const uint4*>(wk + (size_t)o * kK2 + kg * 8);
  }
  // the weights written by the threads are read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  // tile t: image t / (H * segs), row and segment within it
  auto tile_of = [&](int t, int& img, int& y, int& x0) {
    img = t / (H * segs);
    const int r0 = t % (H * segs);
    y = r0 / segs;
    x0 = (r0 % segs) * TC_M;
  };
  // one thread: the tensor copies of tile t's halo (rows y-1..y+1, cells
  // x0-1..x0+TC_M of every plane; coordinates outside the image read zeros)
  auto issue = [&](int t) {
    int img, y, x0;
    tile_of(t, img, y, x0);
    const unsigned bar = smem_u32(&tbar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTcHaloBytes) : "memory");
#pragma unroll
    for (int pl = 0; pl < 4; ++pl)
      asm volatile(
          "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
          "%6}], [%7];" ::"r"(smem_u32(sa + pl * TC_PLANE)),
          "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(pl), "r"(x0 - 1), "r"(y - 1), "r"(img), "r"(bar)
          : "memory");
  };
  bool ok = true;
  unsigned phase = 0, tphase = 0;
  if (TMA && tid == 0 && (int)blockIdx.x < total) issue(blockIdx.x);
  for (int t = blockIdx.x; t < total && ok; t += gridDim.x, phase ^= 1u) {
    int img, y, x0;
    tile_of(t, img, y, x0);
    if constexpr (TMA) {
      // the halo of tile t has landed (bounded wait; the outcome is uniform);
      // the barrier also orders the previous tile's read-back before this
      // tile's MMAs overwrite the accumulator
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      ok = __syncthreads_and(mbar_wait(&tbar, tphase));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tphase ^= 1u;
      if (!ok) {
        if (tid == 0 && err) atomicCAS(err, 0, kErrTimeout);
        // the copies may still be in flight: wait for them once more (bounded)
        __syncthreads_and(mbar_wait(&tbar, tphase ^ 1u));
        break;
      }
    } else {
      // halo rows y-1..y+1, cells x0-1..x0+TC_M, zeros outside the image
      for (int i = tid; i < 3 * TC_HW * 4; i += blockDim.x) {
        const int pl = i % 4, cell = i / 4, r = cell / TC_HW, cx = cell % TC_HW;
        const int gy = y + r - 1, gx = x0 + cx - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
          v = *reinterpret_cast<const uint4*>(in + (((size_t)img * H + gy) * W + gx) * kHid + pl * 8);
        *reinterpret_cast<uint4*>(sa + pl * TC_PLANE + (r * TC_HW + cx) * 16) = v;
      }
      // operands written by the threads are read by the tensor cores (async
      // proxy); the previous segment's accumulator reads are complete
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll 1
      for (int j = 0; j < 18; ++j) {  // depth step j: tap j/2, input channels (j%2)*16 .. +15
        const int tap = j >> 1, ky = tap / 3, kx = tap % 3, cg = (j & 1) * 2;
        const uint64_t ad = smem_desc(a0 + cg * TC_PLANE + (ky * TC_HW + kx) * 16, TC_PLANE, 128);
        const uint64_t bd = smem_desc(b0 + (tap * 4 + cg) * 512, 512, 128);
        const uint32_t acc = j > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    // bounded wait for the MMAs; every thread waits (acquire), the outcome is uniform
    ok = __syncthreads_and(mbar_wait(&mbar, phase));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (tid == 0 && err) atomicCAS(err, 0, kErrTimeout);
      // the MMAs may still be in flight: wait for them once more (bounded)
      // before the tensor memory they write is freed below
      __syncthreads_and(mbar_wait(&mbar, phase));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      break;
    }
    // the MMAs have read the halo: the next tile's copies run during the read-back
    if (TMA && tid == 0 && t + (int)gridDim.x < total) issue(t + gridDim.x);
    // warp w reads tensor-memory lanes 32w..32w+31 (its cells), 32 columns (channels)
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(tmem + ((uint32_t)(32 * warp) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int gx = x0 + 32 * warp + lane;
    if (gx < W) {
      const size_t cell = ((size_t)img * H + y) * W + gx;
      uint32_t* dst = reinterpret_cast<uint32_t*>(out + cell * kHid);
      if constexpr (MODE == kFwd) {
#pragma unroll
        for (int o = 0; o < kHid; o += 2) {
          const float a = fmaxf(__uint_as_float(v[o]) + s_b[o], 0.f);
          const float b = fmaxf(__uint_as_float(v[o + 1]) + s_b[o + 1], 0.f);
          dst[o / 2] = pack2(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
        }
      } else {
        const uint4* mk = reinterpret_cast<const uint4*>(mask + cell * kHid);
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 8 channels per 16-byte piece of the mask
          const uint4 m4 = mk[q];
          const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int o = 8 * q + 2 * h;
            const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[h]);
            const float a = __bfloat162float(m2.x) > 0.f ? __uint_as_float(v[o]) : 0.f;
            const float b = __bfloat162float(m2.y) > 0.f ? __uint_as_float(v[o + 1]) : 0.f;
            dst[o / 2] = pack2(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem_base));
}

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of activations [img][H][W][32] bf16 as five dimensions
// (8 channels, 4 planes, W, H, img) with a box of one plane x TC_HW cells x
// 3 rows; false if it cannot be built (the threads then stage the halo).
static bool halo_map(CUtensorMap* m, const bf* in, int n, int H, int W) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || ((uintptr_t)in & 15u)) return false;
  const cuuint64_t dims[5] = {8, 4, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
  const cuuint64_t strides[4] = {16, 64, 64ull * W, 64ull * W * H};  // bytes, dimensions 1..4
  const cuuint32_t box[5] = {8, 1, TC_HW, 3, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf*>(in), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// mask: null for the forward layer (bias + ReLU), else the input gradient
// masked by mask > 0.
void launch_conv32_tc(const bf* in, const bf* wk, const float* bias, int n, int H, int W, bf* out, int* err,
                      cudaStream_t s, const bf* mask = nullptr) {
  static int nsm = 0;  // SMs of the device (queried once)
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const int total = n * H * ((W + TC_M - 1) / TC_M);
  const int cap = nsm * 5;  // resident CTAs at 43 KB of shared memory each
  const int grid = total < cap ? total : cap;
  alignas(64) CUtensorMap m;
  memset(&m, 0, sizeof m);
  const bool tma = halo_map(&m, in, n, H, W);
  if (mask)
    (tma ? conv32_tc_kernel<true, kDgrad> : conv32_tc_kernel<false, kDgrad>)<<<grid, 128, kTcSmem, s>>>(
        m, in, wk, nullptr, n, H, W, out, mask, err);
  else
    (tma ? conv32_tc_kernel<true, kFwd> : conv32_tc_kernel<false, kFwd>)<<<grid, 128, kTcSmem, s>>>(
        m, in, wk, bias, n, H, W, out, nullptr, err);
}

// Weight gradient of a 3 x 3 convolution, per CTA partial sums over the
// tiles it owns (persistent loop):
//   part[b][o][tap*CIN + c] = sum_cells dz[cell][o] * a[cell + off(tap)][c]
//   part[b][32*9*CIN + o]   = sum_cells dz[cell][o]
// GEMM with M = o (two m16 tiles), N = (tap, c), K = cells (a tile row of
// 16 cells per k16 step); warp w owns the n8 tiles w, w+4, ...
template <int CIN>
__global__ void __launch_bounds__(kThreads) wgrad_kernel(const bf* __restrict__ dz, const bf* __restrict__ a, int N,
                                                         int H, int W, float* __restrict__ part) {
  constexpr int CS = CIN + 8, DS = kHid + 8;
  constexpr int NT = 9 * CIN / 8, NPW = (NT + 3) / 4;
  constexpr int LEN = kHid * 9 * CIN;
  __shared__ __align__(16) bf s_a[HH * HW * CS];
  __shared__ __align__(16) bf s_dz[TH * TW * DS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
  const int ntiles = tiles_x * tiles_y * N;
  float acc[2][NPW][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NPW; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][j][e] = 0.f;
  float dbias = 0.f;

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int img = t / (tiles_x * tiles_y), r = t % (tiles_x * tiles_y);
    const int ty0 = (r / tiles_x) * TH, tx0 = (r % tiles_x) * TW;
    __syncthreads();  // the previous tile's reads are done
    load_halo<CIN, CS>(a, img, H, W, ty0, tx0, s_a);
    for (int i = threadIdx.x; i < TH * TW * (kHid / 2); i += blockDim.x) {
      const int cell = i / (kHid / 2), pr = i % (kHid / 2);
      const int gy = ty0 + cell / TW, gx = tx0 + cell % TW;
      uint32_t v = 0;
      if (gy < H && gx < W) v = ld32(dz + (((size_t)img * H + gy) * W + gx) * kHid + 2 * pr);
      *reinterpret_cast<uint32_t*>(s_dz + cell * DS + 2 * pr) = v;
    }
    __syncthreads();
    if (threadIdx.x < kHid)
      for (int cell = 0; cell < TH * TW; ++cell) dbias += __bfloat162float(s_dz[cell * DS + threadIdx.x]);
#pragma unroll 1
    for (int kc = 0; kc < TH; ++kc) {  // tile row = k16 step
      uint32_t af[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int o0 = 16 * m + g;
        const bf* d0 = s_dz + (kc * TW + 2 * q) * DS;
        af[m][0] = pack2(d0[o0], d0[DS + o0]);
        af[m][1] = pack2(d0[o0 + 8], d0[DS + o0 + 8]);
        af[m][2] = pack2(d0[8 * DS + o0], d0[9 * DS + o0]);
        af[m][3] = pack2(d0[8 * DS + o0 + 8], d0[9 * DS + o0 + 8]);
      }
#pragma unroll
      for (int j = 0; j < NPW; ++j) {
        const int nt = warp + 4 * j;
        if (nt < NT) {
          const int n0 = 8 * nt, tap = n0 / CIN, c = n0 % CIN + g;
          const int ky = tap / 3, kx = tap % 3;
          const bf* h0 = s_a + ((kc + ky) * HW + 2 * q + kx) * CS + c;
          const uint32_t b[2] = {pack2(h0[0], h0[CS]), pack2(h0[8 * CS], h0[9 * CS])};
          mma16816(acc[0][j], af[0], b);
          mma16816(acc[1][j], af[1], b);
        }
      }
    }
  }
  float* P = part + (size_t)blockIdx.x * (LEN + kHid);
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NPW; ++j) {
      const int nt = warp + 4 * j;
      if (nt < NT) {
        const int n = 8 * nt + 2 * q, o = 16 * m + g;
        P[o * 9 * CIN + n] = acc[m][j][0];
        P[o * 9 * CIN + n + 1] = acc[m][j][1];
        P[(o + 8) * 9 * CIN + n] = acc[m][j][2];
        P[(o + 8) * 9 * CIN + n + 1] = acc[m][j][3];
      }
    }
  if (threadIdx.x < kHid) P[LEN + threadIdx.x] = dbias;
}

// Fixed-order sum of the per-CTA partials of layer L (1 or 2) into the
// parameter-ordered gradient.
template <int CIN>
__global__ void reduce_wgrad_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad, int offW,
                                    int offB, int cin_real) {
  constexpr int LEN = kHid * 9 * CIN;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= LEN + kHid) return;
  float s = 0.f;
  for (int b = 0; b < nparts; ++b) s += part[(size_t)b * (LEN + kHid) + j];
  if (j >= LEN) {
    grad[offB + (j - LEN)] = s;
    return;
  }
  const int o = j / (9 * CIN), r = j % (9 * CIN), tap = r / CIN, c = r % CIN;
  if (c < cin_real) grad[offW + (o * 9 + tap) * cin_real + c] = s;
}

// 1 x 1 head: z = b3 + a2 . w3 per cell.  With labels: the class-weighted
// cross-entropy w (softplus(z) - y z) / M, dz = w (sigmoid(z) - y) / M,
// dL/da2 -> dz2 = dz w3 (a2 > 0) (bf16), and per-block partial sums of
// dL/dw3 = dz a2, dL/db3 = dz and the loss.
constexpr int kHeadThreads = 256, kHeadPart = kHid + 2;
__global__ void __launch_bounds__(kHeadThreads) head_kernel(const bf* __restrict__ a2, const float* __restrict__ theta,
                                                            int M, float* __restrict__ logits,
                                                            const uint8_t* __restrict__ y, float pos_weight,
                                                            float invM, bf* __restrict__ dz2, float* __restrict__ part) {
  __shared__ float s_red[kHeadThreads / 32][kHeadPart];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* w3 = theta + kOffW3;
  float av[kHid];
  float z = 0.f, dz = 0.f, L = 0.f;
  if (i < M) {
    const uint4* src = reinterpret_cast<const uint4*>(a2 + (size_t)i * kHid);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint4 u = src[v];
      const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        av[8 * v + 2 * k] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w4[k] & 0xffffu)));
        av[8 * v + 2 * k + 1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w4[k] >> 16)));
      }
    }
    z = theta[kOffB3];
#pragma unroll
    for (int c = 0; c < kHid; ++c) z = fmaf(av[c], w3[c], z);
    logits[i] = z;
    if (y) {
      const float yy = y[i] ? 1.f : 0.f, w = y[i] ? pos_weight : 1.f;
      const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus, stable
      const float sig = 1.f / (1.f + expf(-z));
      L = w * (sp - yy * z) * invM;
      dz = w * (sig - yy) * invM;
      uint32_t* dst = reinterpret_cast<uint32_t*>(dz2 + (size_t)i * kHid);
#pragma unroll
      for (int c = 0; c < kHid; c += 2) {
        const float g0 = av[c] > 0.f ? dz * w3[c] : 0.f, g1 = av[c + 1] > 0.f ? dz * w3[c + 1] : 0.f;
        dst[c / 2] = pack2(__float2bfloat16_rn(g0), __float2bfloat16_rn(g1));
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < kHid; ++c) av[c] = 0.f;
  }
  if (!y) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float vals[kHeadPart];
#pragma unroll
  for (int c = 0; c < kHid; ++c) vals[c] = dz * av[c];
  vals[kHid] = dz;
  vals[kHid + 1] = L;
#pragma unroll
  for (int c = 0; c < kHeadPart; ++c) {
    float v = vals[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kHeadPart) {
    float s = 0.f;
    for (int w = 0; w < kHeadThreads / 32; ++w) s += s_red[w][threadIdx.x];
    part[(size_t)blockIdx.x * kHeadPart + threadIdx.x] = s;
  }
}

__global__ void reduce_head_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                                   float* __restrict__ loss) {
  const int j = threadIdx.x;
  if (j >= kHeadPart) return;
  float s = 0.f;
  for (int b = 0; b < nparts; ++b) s += part[(size_t)b * kHeadPart + j];
  if (j < kHid)
    grad[kOffW3 + j] = s;
  else if (j == kHid)
    grad[kOffB3] = s;
  else
    *loss = s;
}

// bf16 GEMM operands of the convolutions from the float32 parameters.
__device__ __forceinline__ void pack_one(const Weights& w, int j, float v) {
  if (j < kOffB1) {
    const int o = j / (9 * kCin), r = j % (9 * kCin), tap = r / kCin, c = r % kCin;
    w.w1f[o * kK1 + tap * kCinPad + c] = __float2bfloat16_rn(v);
  } else if (j >= kOffW2 && j < kOffB2) {
    const int jj = j - kOffW2, o = jj / (9 * kHid), r = jj % (9 * kHid), tap = r / kHid, c = r % kHid;
    const bf b = __float2bfloat16_rn(v);
    w.w2f[o * kK2 + tap * kHid + c] = b;
    w.w2d[c * kK2 + (8 - tap) * kHid + o] = b;
  }
}

__global__ void pack_kernel(Weights w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kParams) pack_one(w, j, w.theta[j]);
}

// Adam (Kingma & Ba 2015) with bias correction c1 = 1/(1 - b1^t),
// c2 = 1/(1 - b2^t) computed on the host; then the bf16 operands.
__global__ void adam_kernel(Weights w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                            float lr, float b1, float b2, float c1, float c2, float eps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kParams) return;
  const float gj = g[j];
  const float mj = b1 * m[j] + (1.f - b1) * gj;
  const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  const float th = w.theta[j] - lr * (mj * c1) / (sqrtf(vj * c2) + eps);
  w.theta[j] = th;
  pack_one(w, j, th);
}

// Features of a cell: (log rho, s u_x, s u_y, log T, log10(eps s^2)) from
// U, s = dx_ref / dx: the criterion of Sec. 3.1.2 (divided by eps) sees
// velocity jumps over 2 dx and eps times squared temperature jumps over
// 2 dx, so these channels present the same physical state identically on
// every grid spacing.
__global__ void features_kernel(const double* __restrict__ U, const double* __restrict__ eps, int nc, double scale,
                                bf* __restrict__ x) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double rho = U[c], ux = U[nc + c] / rho, uy = U[2 * (size_t)nc + c] / rho;
  const double T = (U[3 * (size_t)nc + c] - 0.5 * rho * (ux * ux + uy * uy)) / rho;
  const float f[5] = {(float)log(rho), (float)(scale * ux), (float)(scale * uy), (float)log(T),
                      (float)log10(eps[c] * scale * scale)};
  uint32_t w[8];
  w[0] = pack2(__float2bfloat16_rn(f[0]), __float2bfloat16_rn(f[1]));
  w[1] = pack2(__float2bfloat16_rn(f[2]), __float2bfloat16_rn(f[3]));
  w[2] = pack2(__float2bfloat16_rn(f[4]), __float2bfloat16_rn(0.f));
#pragma unroll
  for (int k = 3; k < 8; ++k) w[k] = 0u;
  uint4* dst = reinterpret_cast<uint4*>(x + (size_t)c * kCinPad);
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

__global__ void judge_kernel(uint8_t* __restrict__ flags, uint8_t* __restrict__ pred, const float* __restrict__ logits,
                             int nc, int have_prev, unsigned long long* __restrict__ counters) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned p = 0, miss = 0, extra = 0, cells = 0;
  if (c < nc) {
    const uint8_t qf = flags[c];
    const uint8_t nxt = logits[c] > 0.f ? 1 : 0;
    if (have_prev) {
      const uint8_t pp = pred[c];
      p = pp;
      miss = qf && !pp;
      extra = pp && !qf;
      cells = 1;
    }
    flags[c] = (qf || nxt) ? 1 : 0;
    pred[c] = nxt;
  }
  const unsigned full = 0xffffffffu;
  p = __reduce_add_sync(full, p);
  miss = __reduce_add_sync(full, miss);
  extra = __reduce_add_sync(full, extra);
  cells = __reduce_add_sync(full, cells);
  if ((threadIdx.x & 31) == 0 && cells) {
    atomicAdd(counters + 0, (unsigned long long)p);
    atomicAdd(counters + 1, (unsigned long long)miss);
    atomicAdd(counters + 2, (unsigned long long)extra);
    atomicAdd(counters + 3, (unsigned long long)cells);
  }
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t weights_bytes() {
  return up256(kParams * sizeof(float)) + up256(kHid * kK1 * 2) + 2 * up256(kHid * kK2 * 2);
}

size_t carve_weights(unsigned char* p, Weights& w) {
  size_t o = 0;
  w.theta = (float*)(p + o);
  o += up256(kParams * sizeof(float));
  w.w1f = (bf*)(p + o);
  o += up256(kHid * kK1 * 2);
  w.w2f = (bf*)(p + o);
  o += up256(kHid * kK2 * 2);
  w.w2d = (bf*)(p + o);
  o += up256(kHid * kK2 * 2);
  return o;
}

void launch_pack(const Weights& w, cudaStream_t s) {
  cudaMemsetAsync(w.w1f, 0, kHid * kK1 * 2, s);  // padded input channels stay zero
  pack_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(w);
}

void launch_features(const double* U, const double* eps, int nc, double dx, bf* x, cudaStream_t s) {
  features_kernel<<<(nc + 255) / 256, 256, 0, s>>>(U, eps, nc, kDxRef / dx, x);
}

static dim3 conv_grid(int n, int H, int W) { return dim3((W + TW - 1) / TW, (H + TH - 1) / TH, n); }

void launch_forward(const Weights& w, const bf* x, int n, int H, int W, bf* a1, bf* a2, float* logits, int* err,
                    cudaStream_t s) {
  conv_kernel<kCinPad, kFwd><<<conv_grid(n, H, W), kThreads, 0, s>>>(x, w.w1f, w.theta + kOffB1, H, W, a1, nullptr);
  launch_conv32_tc(a1, w.w2f, w.theta + kOffB2, n, H, W, a2, err, s);
  const int M = n * H * W;
  head_kernel<<<(M + kHeadThreads - 1) / kHeadThreads, kHeadThreads, 0, s>>>(a2, w.theta, M, logits, nullptr, 0.f,
                                                                            0.f, nullptr, nullptr);
}

void launch_judge(uint8_t* flags, uint8_t* pred, const float* logits, int nc, int have_prev,
                  unsigned long long* counters, cudaStream_t s) {
  judge_kernel<<<(nc + 255) / 256, 256, 0, s>>>(flags, pred, logits, nc, have_prev, counters);
}

}  // namespace cnn
}  // namespace esbgk

// ---------------------------------------------------------------------------
// Training object (C ABI).

using namespace esbgk::cnn;

struct esbgk_cnn {
  int max_n, H, W;
  cudaStream_t stream;
  Weights w;
  float *m, *v, *grad, *logits, *part, *loss;
  __nv_bfloat16 *a1, *a2, *dz2, *dz1;
  int nparts;  // CTAs of the weight-gradient kernels
  int* err;    // device error word (kErrTimeout: a bounded wait for the tensor cores expired)
  long long t;
  std::string msg;
};

namespace {

struct CnnLayout {
  size_t w, m, v, grad, logits, part, loss, a1, a2, dz2, dz1, err, total;
  int nparts;
};

bool cnn_layout(int max_n, int H, int W, CnnLayout& L) {
  if (max_n < 1 || H < 1 || W < 1) return false;
  const long long M = (long long)max_n * H * W;
  if (M >= (1LL << 28)) return false;
  L.nparts = 2 * 152;
  size_t p = 0;
  auto take = [&](size_t b) {
    const size_t at = p;
    p += up256(b);
    return at;
  };
  L.w = take(weights_bytes());
  L.m = take(kParams * 4);
  L.v = take(kParams * 4);
  L.grad = take(kParams * 4);
  L.logits = take(M * 4);
  const size_t head_parts = (size_t)((M + kHeadThreads - 1) / kHeadThreads) * kHeadPart;
  const size_t wg_parts = (size_t)L.nparts * (kHid * kK2 + kHid);
  L.part = take(4 * (head_parts > wg_parts ? head_parts : wg_parts));
  L.loss = take(4);
  L.a1 = take(M * kHid * 2);
  L.a2 = take(M * kHid * 2);
  L.dz2 = take(M * kHid * 2);
  L.dz1 = take(M * kHid * 2);
  L.err = take(sizeof(int));
  L.total = p;
  return true;
}

int cnn_check(esbgk_cnn* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return ESBGK_OK;
  c->msg = std::string(where) + ": " + cudaGetErrorString(e);
  return ESBGK_E_CUDA;
}

// After a synchronisation: the device error word.
int cnn_sync_check(esbgk_cnn* c, const char* where) {
  int r = cnn_check(c, cudaStreamSynchronize(c->stream), where);
  if (r) return r;
  int e = 0;
  r = cnn_check(c, cudaMemcpy(&e, c->err, sizeof e, cudaMemcpyDeviceToHost), "read error word");
  if (r) return r;
  if (e == esbgk::kErrTimeout) {
    c->msg = "bounded wait for the tensor cores expired";
    return ESBGK_E_TIMEOUT;
  }
  return ESBGK_OK;
}

// Forward and backward passes of n images: gradient into c->grad, loss
// into c->loss (device).
void backward_launches(esbgk_cnn* c, const __nv_bfloat16* x, const uint8_t* y, int n, float pos_weight) {
  const int H = c->H, W = c->W, M = n * H * W;
  cudaStream_t s = c->stream;
  const dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, n);
  conv_kernel<kCinPad, kFwd><<<grid, kThreads, 0, s>>>(x, c->w.w1f, c->w.theta + kOffB1, H, W, c->a1, nullptr);
  launch_conv32_tc(c->a1, c->w.w2f, c->w.theta + kOffB2, n, H, W, c->a2, c->err, s);
  const int hb = (M + kHeadThreads - 1) / kHeadThreads;
  head_kernel<<<hb, kHeadThreads, 0, s>>>(c->a2, c->w.theta, M, c->logits, y, pos_weight, 1.f / M, c->dz2, c->part);
  reduce_head_kernel<<<1, 64, 0, s>>>(c->part, hb, c->grad, c->loss);
  wgrad_kernel<kHid><<<c->nparts, kThreads, 0, s>>>(c->dz2, c->a1, n, H, W, c->part);
  reduce_wgrad_kernel<kHid><<<(kHid * kK2 + kHid + 255) / 256, 256, 0, s>>>(c->part, c->nparts, c->grad, kOffW2,
                                                                            kOffB2, kHid);
  launch_conv32_tc(c->dz2, c->w.w2d, nullptr, n, H, W, c->dz1, c->err, s, c->a1);
  wgrad_kernel<kCinPad><<<c->nparts, kThreads, 0, s>>>(c->dz1, x, n, H, W, c->part);
  reduce_wgrad_kernel<kCinPad><<<(kHid * kK1 + kHid + 255) / 256, 256, 0, s>>>(c->part, c->nparts, c->grad, kOffW1,
                                                                              kOffB1, kCin);
}

}  // namespace

extern "C" {

size_t esbgk_cnn_workspace_bytes(int32_t max_images, int32_t H, int32_t W) {
  CnnLayout L;
  return cnn_layout(max_images, H, W, L) ? L.total : 0;
}

int esbgk_cnn_create(int32_t max_images, int32_t H, int32_t W, void* workspace, size_t workspace_bytes, void* stream,
                     esbgk_cnn** out) {
  if (!out) return ESBGK_E_ARG;
  *out = nullptr;
  CnnLayout L;
  if (!cnn_layout(max_images, H, W, L) || !workspace) return ESBGK_E_ARG;
  if (workspace_bytes < L.total || ((uintptr_t)workspace % 256) != 0) return ESBGK_E_WORKSPACE;
  esbgk_cnn* c = new (std::nothrow) esbgk_cnn();
  if (!c) return ESBGK_E_ARG;
  unsigned char* p = (unsigned char*)workspace;
  c->max_n = max_images;
  c->H = H;
  c->W = W;
  c->stream = (cudaStream_t)stream;
  carve_weights(p + L.w, c->w);
  c->m = (float*)(p + L.m);
  c->v = (float*)(p + L.v);
  c->grad = (float*)(p + L.grad);
  c->logits = (float*)(p + L.logits);
  c->part = (float*)(p + L.part);
  c->loss = (float*)(p + L.loss);
  c->a1 = (__nv_bfloat16*)(p + L.a1);
  c->a2 = (__nv_bfloat16*)(p + L.a2);
  c->dz2 = (__nv_bfloat16*)(p + L.dz2);
  c->dz1 = (__nv_bfloat16*)(p + L.dz1);
  c->err = (int*)(p + L.err);
  c->nparts = L.nparts;
  c->t = 0;
  const cudaError_t e = cudaMemsetAsync(workspace, 0, L.total, c->stream);
  if (e != cudaSuccess) {
    delete c;
    return ESBGK_E_CUDA;
  }
  *out = c;
  return ESBGK_OK;
}

void esbgk_cnn_destroy(esbgk_cnn* c) { delete c; }

int esbgk_cnn_set_params(esbgk_cnn* c, const float* theta) {
  if (!c || !theta) return ESBGK_E_ARG;
  int r = cnn_check(c, cudaMemcpyAsync(c->w.theta, theta, kParams * 4, cudaMemcpyHostToDevice, c->stream), "params");
  if (!r) r = cnn_check(c, cudaMemsetAsync(c->m, 0, kParams * 4, c->stream), "adam state");
  if (!r) r = cnn_check(c, cudaMemsetAsync(c->v, 0, kParams * 4, c->stream), "adam state");
  if (r) return r;
  launch_pack(c->w, c->stream);
  c->t = 0;
  r = cnn_check(c, cudaGetLastError(), "pack");
  return r ? r : cnn_check(c, cudaStreamSynchronize(c->stream), "set_params sync");
}

int esbgk_cnn_get_params(esbgk_cnn* c, float* theta) {
  if (!c || !theta) return ESBGK_E_ARG;
  int r = cnn_check(c, cudaMemcpyAsync(theta, c->w.theta, kParams * 4, cudaMemcpyDeviceToHost, c->stream), "params");
  return r ? r : cnn_check(c, cudaStreamSynchronize(c->stream), "get_params sync");
}

int esbgk_cnn_forward(esbgk_cnn* c, const void* x, int32_t n, float* logits) {
  if (!c || !x || !logits || n < 1 || n > c->max_n) return ESBGK_E_ARG;
  launch_forward(c->w, (const __nv_bfloat16*)x, n, c->H, c->W, c->a1, c->a2, logits, c->err, c->stream);
  return cnn_check(c, cudaGetLastError(), "cnn forward");
}

int esbgk_cnn_gradient(esbgk_cnn* c, const void* x, const uint8_t* y, int32_t n, float pos_weight, float* loss,
                       float* grad) {
  if (!c || !x || !y || n < 1 || n > c->max_n || !(pos_weight > 0.f)) return ESBGK_E_ARG;
  backward_launches(c, (const __nv_bfloat16*)x, y, n, pos_weight);
  int r = cnn_check(c, cudaGetLastError(), "cnn backward");
  if (!r && grad)
    r = cnn_check(c, cudaMemcpyAsync(grad, c->grad, kParams * 4, cudaMemcpyDeviceToHost, c->stream), "grad copy");
  if (!r && loss) r = cnn_check(c, cudaMemcpyAsync(loss, c->loss, 4, cudaMemcpyDeviceToHost, c->stream), "loss copy");
  return r ? r : cnn_sync_check(c, "gradient sync");
}

int esbgk_cnn_train_step(esbgk_cnn* c, const void* x, const uint8_t* y, int32_t n, float pos_weight, float lr,
                         float* loss) {
  if (!c || !x || !y || n < 1 || n > c->max_n || !(pos_weight > 0.f) || !(lr > 0.f)) return ESBGK_E_ARG;
  backward_launches(c, (const __nv_bfloat16*)x, y, n, pos_weight);
  c->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)c->t))), c2 = (float)(1.0 / (1.0 - pow(b2, (double)c->t)));
  adam_kernel<<<(kParams + 255) / 256, 256, 0, c->stream>>>(c->w, c->m, c->v, c->grad, lr, (float)b1, (float)b2, c1,
                                                            c2, 1e-8f);
  int r = cnn_check(c, cudaGetLastError(), "cnn train step");
  if (!r && loss) {
    r = cnn_check(c, cudaMemcpyAsync(loss, c->loss, 4, cudaMemcpyDeviceToHost, c->stream), "loss copy");
    if (!r) r = cnn_sync_check(c, "train sync");
  }
  return r;
}

int esbgk_cnn_sync(esbgk_cnn* c) {
  if (!c) return ESBGK_E_ARG;
  return cnn_sync_check(c, "cnn sync");
}

}  // extern "C"
