// Learned confidence in place of the right-image SGM pass.
//
// The paper keeps a disparity where the left-right check of Sec. 3.1 passes,
// which needs a second SGM pass with the right image as reference.  This
// path predicts that check's outcome from the left pass alone:
//
//   1. features (features_staged_kernel for D a multiple of 32,
//      features_px_kernel for other multiples of 8, features_vec_kernel /
//      features_kernel otherwise): seven channels per pixel of the left
//      pass's aggregated cost curve S (best cost, margin to the best cost
//      outside the winner's neighbourhood, curvature, disagreement of the
//      three path groups, winner, distance to the left border, matching cost
//      at the winner), each an integer over a power of two, stored as
//      bfloat16 [H][W][8].  The winner and its parabolic subpixel value come
//      out of the same pass, computed exactly like the plain select.  Then
//      visibility_kernel fills channel 7 from the winners of each row: the
//      occlusion test that the left-right check performs, read off the left
//      disparities alone.
//   2. infer_kernel: a 4-layer 3x3 network (8 -> 32 -> 32 -> 32 -> 1, ReLU,
//      sigmoid), bfloat16 weights and activations, fp32 accumulation on the
//      5th-generation tensor cores: tcgen05.mma with operands in shared
//      memory and accumulators in tensor memory, one warp issuing and eight
//      draining the accumulators, all four layers of an output tile fused in
//      shared memory (a layer's MMAs start on the rows its predecessor has
//      finished), the tiles of every pass of a call in one launch.
//   3. training kernels (fp32 CUDA cores): forward with the same bfloat16
//      roundings, weighted binary cross-entropy, data and weight gradients,
//      Adam.
//
// Implicit-GEMM layout of the inference kernel.  An output tile is TX x TY
// pixels; layer l (1..4) is evaluated on a region that extends 4 - l pixels
// past the tile on every side, enumerated row-major with a fixed pitch P, so
// that the input of tap (ky, kx) for output pixel m is input pixel
// m + ky P + kx.  Activations are stored as K-chunk planes [chunk][pixel][8
// channels] (16 bytes per pixel and chunk): eight consecutive pixels form one
// 8 x 16-byte core matrix of the no-swizzle K-major operand layout, so a tap
// is just a 16-byte shift of the descriptor's start address.
#include <math.h>

#include <cuda_bf16.h>

#include "sf_confnet.cuh"

namespace sf {
namespace confnet {

namespace {

// ---------------------------------------------------------------------------
// 1. features
// ---------------------------------------------------------------------------
constexpr int kMaxPerLane = SF_MAX_DISPARITY / 32;

// minimum over the warp (every lane gets it): one warp-reduction instruction
__device__ __forceinline__ uint32_t warp_min(uint32_t v) { return __reduce_min_sync(kFullMask, v); }

// One pixel's curve, spread over the warp: lane l holds d = l + 32 k.
struct Curve {
  uint32_t s[kMaxPerLane];
  uint32_t ks, kh, kd, ku;     // (value << 8 | d) minima: S, horizontal, downward, upward
};

// Features, winner and subpixel winner of one pixel; every lane takes part,
// lane `out_lane` writes.
__device__ __forceinline__ void finish_pixel(const FeatureArgs& a, Curve& c, int x, size_t pix, int lane,
                                             int out_lane) {
  c.ks = warp_min(c.ks);
  c.kh = warp_min(c.kh);
  c.kd = warp_min(c.kd);
  c.ku = warp_min(c.ku);
  const int ds = (int)(c.ks & 0xffu);
  const uint32_t s0 = c.ks >> 8;
  uint32_t far = 0xffffffffu, vm = 0u, vp = 0u;
#pragma unroll
  for (int k = 0; k < kMaxPerLane; k++) {
    const int d = lane + 32 * k;
    if (d < a.D) {
      if (d - ds >= 2 || ds - d >= 2) far = min(far, c.s[k]);
      if (d == ds - 1) vm = c.s[k];
      if (d == ds + 1) vp = c.s[k];
    }
  }
  far = warp_min(far);
  // S(d*-1), S(d*+1) from the lanes that hold them (0 when out of range)
  vm = __shfl_sync(kFullMask, vm, (ds + 31) & 31);
  vp = __shfl_sync(kFullMask, vp, (ds + 1) & 31);
  if (lane != out_lane) return;
  const int cstar = a.cost[pix * a.Dp + ds];
  const uint32_t s2 = far == 0xffffffffu ? s0 : far;
  int curv = 0;
  if (a.D > 1) {
    if (ds == 0)
      curv = 2 * ((int)vp - (int)s0);
    else if (ds == a.D - 1)
      curv = 2 * ((int)vm - (int)s0);
    else
      curv = (int)vm + (int)vp - 2 * (int)s0;
  }
  const int gh_d = (int)(c.kh & 0xffu), gd_d = (int)(c.kd & 0xffu), gu_d = (int)(c.ku & 0xffu);
  const int dis = min(abs(gh_d - ds), 16) + min(abs(gd_d - ds), 16) + min(abs(gu_d - ds), 16);
  const int margin = min(max(x - ds, 0), 64);
  // integers over powers of two: exact in fp32, then rounded once to bf16
  const float f[kF] = {(float)s0 * (1.0f / 1024.0f), (float)(s2 - s0) * (1.0f / 256.0f),
                       (float)curv * (1.0f / 256.0f), (float)dis * (1.0f / 16.0f),
                       (float)ds * (1.0f / 128.0f),   (float)margin * (1.0f / 64.0f),
                       (float)cstar * (1.0f / 64.0f), 0.0f};   // channel 7: visibility_kernel
  uint32_t packed[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    packed[i] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  reinterpret_cast<uint4*>(a.feat)[pix] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  a.dint[pix] = (int16_t)ds;
  float v = (float)ds;
  if (a.subpixel && ds > 0 && ds < a.D - 1) {
    const int am = (int)vm - (int)s0, bp = (int)vp - (int)s0;
    v = __fadd_rn((float)ds, __fdiv_rn((float)(am - bp), (float)(2 * (am + bp))));
  }
  a.dsub[pix] = v;
}

// Scalar form (any D): one warp per column pair (x, x + 16) of a 32-column
// strip row; the two columns share the words of the down sweep's partial sum.
__global__ void __launch_bounds__(256)
    features_kernel(FeatureArgs a) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int per_row = a.J * 16;
  if (warp >= a.H * per_row) return;
  const int y = warp / per_row, r = warp - y * per_row;
  const int j = r >> 4, pr = r & 15;
  const int xa = j * 32 + pr, xb = xa + 16;
  const bool in_a = xa < a.W, in_b = xb < a.W;
  const size_t pa = (size_t)y * a.W + xa, pb = (size_t)y * a.W + xb;
  const uint32_t* sd = a.sdown + (((size_t)y * a.J + j) * 16 + pr) * (size_t)a.dpad_shape;
  Curve ca, cb;
  ca.ks = ca.kh = ca.kd = ca.ku = 0xffffffffu;
  cb.ks = cb.kh = cb.kd = cb.ku = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < kMaxPerLane; k++) {
    const int d = lane + 32 * k;
    ca.s[k] = cb.s[k] = 0xffffffffu;
    if (d < a.D) {
      const uint32_t w = sd[d];
      if (in_a) {
        const uint32_t sv = a.S[pa * a.D + d];
        const uint32_t gh = (uint32_t)a.hfwd[pa * a.Dp + d] + (uint32_t)a.hbwd[pa * a.Dp + d];
        const uint32_t gd = w & 0xffffu;
        ca.s[k] = sv;
        ca.ks = min(ca.ks, (sv << 8) | (uint32_t)d);
        ca.kh = min(ca.kh, (gh << 8) | (uint32_t)d);
        ca.kd = min(ca.kd, (gd << 8) | (uint32_t)d);
        ca.ku = min(ca.ku, ((sv - gh - gd) << 8) | (uint32_t)d);
      }
      if (in_b) {
        const uint32_t sv = a.S[pb * a.D + d];
        const uint32_t gh = (uint32_t)a.hfwd[pb * a.Dp + d] + (uint32_t)a.hbwd[pb * a.Dp + d];
        const uint32_t gd = w >> 16;
        cb.s[k] = sv;
        cb.ks = min(cb.ks, (sv << 8) | (uint32_t)d);
        cb.kh = min(cb.kh, (gh << 8) | (uint32_t)d);
        cb.kd = min(cb.kd, (gd << 8) | (uint32_t)d);
        cb.ku = min(cb.ku, ((sv - gh - gd) << 8) | (uint32_t)d);
      }
    }
  }
  if (in_a) finish_pixel(a, ca, xa, pa, lane, 0);
  if (in_b) finish_pixel(a, cb, xb, pb, lane, 1);
}

// Vector form (D % 4 == 0): one warp per column pair (x, x + 16) of a
// 32-column strip row (the pair shares the words of the down sweep's partial
// sum); lane l holds disparities 4l .. 4l+3 (+128 for a second chunk) of
// both columns: 8-byte loads of S, 4-byte loads of the horizontal paths,
// 16-byte loads of the partial-sum words.
struct VecCurve {
  uint32_t ks, kh, kd, ku;
};

template <int NCH>
__device__ __forceinline__ void vec_finish(const FeatureArgs& a, const uint32_t* sv, VecCurve c, int x,
                                           size_t pix, int lane, int out_lane) {
  c.ks = warp_min(c.ks);
  c.kh = warp_min(c.kh);
  c.kd = warp_min(c.kd);
  c.ku = warp_min(c.ku);
  const int ds = (int)(c.ks & 0xffu);
  const uint32_t s0 = c.ks >> 8;
  uint32_t far = 0xffffffffu, vm = 0u, vp = 0u;
#pragma unroll
  for (int ch = 0; ch < NCH; ch++) {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int d = 128 * ch + 4 * lane + e;
      if (d < a.D) {
        if (d - ds >= 2 || ds - d >= 2) far = min(far, sv[4 * ch + e]);
        if (d == ds - 1) vm = sv[4 * ch + e];
        if (d == ds + 1) vp = sv[4 * ch + e];
      }
    }
  }
  far = warp_min(far);
  vm = __shfl_sync(kFullMask, vm, ((ds + 127) >> 2) & 31);   // lane of d* - 1
  vp = __shfl_sync(kFullMask, vp, ((ds + 1) >> 2) & 31);     // lane of d* + 1
  if (lane != out_lane) return;
  const int cstar = a.cost[pix * a.Dp + ds];
  const uint32_t s2 = far == 0xffffffffu ? s0 : far;
  int curv = 0;
  if (a.D > 1) {
    if (ds == 0)
      curv = 2 * ((int)vp - (int)s0);
    else if (ds == a.D - 1)
      curv = 2 * ((int)vm - (int)s0);
    else
      curv = (int)vm + (int)vp - 2 * (int)s0;
  }
  const int dis = min(abs((int)(c.kh & 0xffu) - ds), 16) + min(abs((int)(c.kd & 0xffu) - ds), 16) +
                  min(abs((int)(c.ku & 0xffu) - ds), 16);
  const int margin = min(max(x - ds, 0), 64);
  const float f[kF] = {(float)s0 * (1.0f / 1024.0f), (float)(s2 - s0) * (1.0f / 256.0f),
                       (float)curv * (1.0f / 256.0f), (float)dis * (1.0f / 16.0f),
                       (float)ds * (1.0f / 128.0f),   (float)margin * (1.0f / 64.0f),
                       (float)cstar * (1.0f / 64.0f), 0.0f};   // channel 7: visibility_kernel
  uint32_t packed[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    packed[i] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  reinterpret_cast<uint4*>(a.feat)[pix] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  a.dint[pix] = (int16_t)ds;
  float v = (float)ds;
  if (a.subpixel && ds > 0 && ds < a.D - 1) {
    const int am = (int)vm - (int)s0, bp = (int)vp - (int)s0;
    v = __fadd_rn((float)ds, __fdiv_rn((float)(am - bp), (float)(2 * (am + bp))));
  }
  a.dsub[pix] = v;
}

template <int NCH>
__global__ void __launch_bounds__(256)
    features_vec_kernel(FeatureArgs a) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int per_row = a.J * 16;
  if (warp >= a.H * per_row) return;
  const int y = warp / per_row, r = warp - y * per_row;
  const int j = r >> 4, pr = r & 15;
  const int xa = j * 32 + pr, xb = xa + 16;
  const bool in_a = xa < a.W, in_b = xb < a.W;
  const size_t pa = (size_t)y * a.W + xa, pb = (size_t)y * a.W + xb;
  const uint32_t* sd = a.sdown + (((size_t)y * a.J + j) * 16 + pr) * (size_t)a.dpad_shape;
  uint32_t sa[4 * NCH], sb[4 * NCH];
  VecCurve ca = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu}, cb = ca;
#pragma unroll
  for (int ch = 0; ch < NCH; ch++) {
    const int d0 = 128 * ch + 4 * lane;
    uint2 s4a = make_uint2(0xffffffffu, 0xffffffffu), s4b = s4a;
    uint32_t hfa = 0, hba = 0, hfb = 0, hbb = 0;
    uint4 w4 = make_uint4(0, 0, 0, 0);
    const bool live = d0 < a.D;
    if (live) {
      w4 = *reinterpret_cast<const uint4*>(sd + d0);
      if (in_a) {
        s4a = *reinterpret_cast<const uint2*>(a.S + pa * a.D + d0);
        hfa = *reinterpret_cast<const uint32_t*>(a.hfwd + pa * a.Dp + d0);
        hba = *reinterpret_cast<const uint32_t*>(a.hbwd + pa * a.Dp + d0);
      }
      if (in_b) {
        s4b = *reinterpret_cast<const uint2*>(a.S + pb * a.D + d0);
        hfb = *reinterpret_cast<const uint32_t*>(a.hfwd + pb * a.Dp + d0);
        hbb = *reinterpret_cast<const uint32_t*>(a.hbwd + pb * a.Dp + d0);
      }
    }
    const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
    const uint32_t ssa[4] = {s4a.x & 0xffffu, s4a.x >> 16, s4a.y & 0xffffu, s4a.y >> 16};
    const uint32_t ssb[4] = {s4b.x & 0xffffu, s4b.x >> 16, s4b.y & 0xffffu, s4b.y >> 16};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const uint32_t d = (uint32_t)(d0 + e);
      sa[4 * ch + e] = live ? ssa[e] : 0xffffffffu;
      sb[4 * ch + e] = live ? ssb[e] : 0xffffffffu;
      if (live) {
        const uint32_t gha = ((hfa >> (8 * e)) & 0xffu) + ((hba >> (8 * e)) & 0xffu);
        const uint32_t gda = ww[e] & 0xffffu;
        ca.ks = min(ca.ks, (ssa[e] << 8) | d);
        ca.kh = min(ca.kh, (gha << 8) | d);
        ca.kd = min(ca.kd, (gda << 8) | d);
        ca.ku = min(ca.ku, ((ssa[e] - gha - gda) << 8) | d);
        const uint32_t ghb = ((hfb >> (8 * e)) & 0xffu) + ((hbb >> (8 * e)) & 0xffu);
        const uint32_t gdb = ww[e] >> 16;
        cb.ks = min(cb.ks, (ssb[e] << 8) | d);
        cb.kh = min(cb.kh, (ghb << 8) | d);
        cb.kd = min(cb.kd, (gdb << 8) | d);
        cb.ku = min(cb.ku, ((ssb[e] - ghb - gdb) << 8) | d);
      }
    }
  }
  if (in_a) vec_finish<NCH>(a, sa, ca, xa, pa, lane, 0);
  if (in_b) vec_finish<NCH>(a, sb, cb, xb, pb, lane, 1);
}

// ---------------------------------------------------------------------------
// 2. weight packing for the tensor-core kernel
// ---------------------------------------------------------------------------
// Parameter vector offsets (same order as the flat layout of the ABI):
// W1 [32][3][3][8], b1, W2 [32][3][3][32], b2, W3, b3, W4 [1][3][3][32], b4.
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 9 * kF * kC, kOffW2 = kOffB1 + kC;
constexpr int kOffB2 = kOffW2 + 9 * kC * kC, kOffW3 = kOffB2 + kC;
constexpr int kOffB3 = kOffW3 + 9 * kC * kC, kOffW4 = kOffB3 + kC, kOffB4 = kOffW4 + 9 * kC;
static_assert(kOffB4 + 1 == kParamCount, "parameter layout");

__device__ __forceinline__ float layer_weight(const float* th, int layer, int co, int tap, int ci) {
  const int ky = tap / 3, kx = tap % 3;
  if (layer == 0) return th[kOffW1 + ((co * 3 + ky) * 3 + kx) * kF + ci];
  if (layer == 1) return th[kOffW2 + ((co * 3 + ky) * 3 + kx) * kC + ci];
  if (layer == 2) return th[kOffW3 + ((co * 3 + ky) * 3 + kx) * kC + ci];
  return th[kOffW4 + (ky * 3 + kx) * kC + ci];
}

// Packed blob: bf16 operand blocks of the four layers, then fp32 biases.
// Block = [K-chunk 0..1][n 0..N-1][8 k-elements].
//   layer 1: block j (0..4) pairs taps 2j and 2j+1 (tap 9 = zeros), 8 channels each
//   layers 2, 3: block 2t + s = tap t, input channels 16s .. 16s+15
//   layer 4: as layers 2, 3 with N = 16 (output 0 real, 1..15 zero)
__global__ void pack_kernel(const float* __restrict__ th, uint16_t* __restrict__ packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kWElems) {
    int layer, rem;
    if (i < kW1Elems) {
      layer = 0; rem = i;
    } else if (i < kW1Elems + kW2Elems) {
      layer = 1; rem = i - kW1Elems;
    } else if (i < kW1Elems + 2 * kW2Elems) {
      layer = 2; rem = i - kW1Elems - kW2Elems;
    } else {
      layer = 3; rem = i - kW1Elems - 2 * kW2Elems;
    }
    const int N = layer == 3 ? 16 : kC;
    const int e = rem % 8;
    const int n = (rem / 8) % N;
    const int chunk = (rem / (8 * N)) % 2;
    const int blk = rem / (16 * N);
    float w = 0.0f;
    if (layer == 0) {
      const int tap = 2 * blk + chunk;
      if (tap < 9) w = layer_weight(th, 0, n, tap, e);
    } else {
      const int tap = blk >> 1, s = blk & 1;
      if (layer < 3 || n == 0) w = layer_weight(th, layer, n, tap, 16 * s + 8 * chunk + e);
    }
    packed[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
  }
  if (i < kBiasFloats) {
    float* bias = reinterpret_cast<float*>(packed + kWElems);
    float v = 0.0f;
    if (i < kC) v = th[kOffB1 + i];
    else if (i < 2 * kC) v = th[kOffB2 + i - kC];
    else if (i < 3 * kC) v = th[kOffB3 + i - 2 * kC];
    else if (i == 3 * kC) v = th[kOffB4];
    bias[i] = v;
  }
}

// ---------------------------------------------------------------------------
// 3. tensor-core inference (tcgen05)
// ---------------------------------------------------------------------------
constexpr int kP = 64;                 // region pitch (pixels)
constexpr int kTX = kP - 8;            // output tile width
constexpr int kTY = 8;                 // output tile height
// rows of the region of layer l (0 = the features, 4 = the output tile)
__host__ __device__ constexpr int region_rows(int l) { return kTY + 8 - 2 * l; }
constexpr int kNPix0 = region_rows(0) * kP + 8, kNPix1 = region_rows(1) * kP + 8;
constexpr int kNPix2 = region_rows(2) * kP + 8, kNPix3 = region_rows(3) * kP + 8;
constexpr int kPlane0 = kNPix0 * 16, kPlane1 = kNPix1 * 16, kPlane2 = kNPix2 * 16;
constexpr int kPlane3 = kNPix3 * 16;
constexpr int kSmFeat = 0;
constexpr int kSmX = kSmFeat + kPlane0;             // layer-1 then layer-3 activations
constexpr int kSmY = kSmX + 4 * kPlane1;            // layer-2 activations
constexpr int kSmW = kSmY + 4 * kPlane2;            // packed weights
constexpr int kSmBias = kSmW + kWElems * 2;
constexpr int kMaxPairs = (region_rows(1) * kP / 128 + 1) / 2;   // M-tile pairs of the largest layer
constexpr int kSmBar = kSmBias + kBiasFloats * 4;                  // one mbarrier per M-tile pair
constexpr int kSmEp = kSmBar + 8 * (kMaxPairs + 1);              // + one for the final drain
constexpr int kSmTmem = kSmEp + 8 * kMaxPairs;                    // epilogue done, per M-tile pair
constexpr int kSmTotal = kSmTmem + 8;
constexpr int kEpiWarps = 8;                                       // epilogue warps (two per TMEM lane quarter)
constexpr int kIssuer = kEpiWarps;                                 // the warp that issues the MMAs
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = kEpiThreads + 32;
constexpr uint32_t kTmemCols = 256;
constexpr long long kMmaSpin = 1ll << 24;
static_assert(kPlane3 <= kPlane1, "layer-3 activations reuse the layer-1 buffer (its plane stride)");
static_assert((region_rows(1) * kP) % 128 == 0 && (region_rows(4) * kP) % 128 == 0, "whole M tiles");
static_assert(kSmTotal <= 227 * 1024, "shared memory");
static_assert(kSmX % 16 == 0 && kSmY % 16 == 0 && kSmW % 16 == 0 && kSmBar % 8 == 0, "alignment");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle, K-major:
//   start address, leading byte offset (next 8-element K chunk), stride byte
//   offset (next group of 8 rows), descriptor version 1.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, M = 128, N as given.
__host__ __device__ constexpr uint32_t instr_desc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// one lane of a converged warp (the warp's loop values stay uniform)
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n .reg .pred P;\n elect.sync _|P, 0xffffffff;\n selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// 32 consecutive fp32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return __uint_as_float(r);
}

// Offset (pixels) of tap t = 3 ky + kx in a pitch-kP region; tap 9 (the
// zero-weight partner of tap 8 in layer 1) reads the next pixel.
__device__ __forceinline__ int tap_off(int t) { return t < 9 ? (t / 3) * kP + (t % 3) : 2 * kP + 3; }

__global__ void __launch_bounds__(kThreads, 1) infer_kernel(InferArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* feat_s = sm + kSmFeat;
  uint8_t* bufx = sm + kSmX;
  uint8_t* bufy = sm + kSmY;
  const float* bias = reinterpret_cast<const float*>(sm + kSmBias);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmTmem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;

  // zero everything once (region slack stays finite), weights and biases in
  for (int i = tid; i < kSmW / 16; i += kThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  const uint4* wsrc = reinterpret_cast<const uint4*>(a.packed);
  for (int i = tid; i < (kWElems * 2 + kBiasFloats * 4) / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm + kSmW)[i] = wsrc[i];
  if (tid == 0) {
    for (int i = 0; i <= kMaxPairs; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + i)) : "memory");
    for (int i = 0; i < kMaxPairs; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(sm + kSmEp + 8 * i)),
                   "r"(kEpiThreads)
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t barp = smem_u32(bar);
  bool failed = false;

  const int tiles_x = (a.W + kTX - 1) / kTX, tiles_y = (a.H + kTY - 1) / kTY;
  const int per_pass = tiles_x * tiles_y, ntiles = per_pass * a.npass;
  const uint32_t w_base = smem_u32(sm + kSmW);
  const uint32_t w2_base = w_base + kW1Elems * 2, w3_base = w2_base + kW2Elems * 2;
  const uint32_t w4_base = w3_base + kW2Elems * 2;

  // features of a tile's region 0 (origin X0-4, Y0-4; zeros outside the
  // image) by asynchronous copies, so that the next tile's arrive while this
  // tile's layers 2-4 run
  auto fetch_features = [&](int t) {
    const int ps = t / per_pass, tl = t - ps * per_pass;
    const uint16_t* feat = a.pass[ps].feat;
    const int X0 = (tl % tiles_x) * kTX, Y0 = (tl / tiles_x) * kTY;
    for (int i = tid; i < region_rows(0) * kP; i += kEpiThreads) {
      const int gy = Y0 - 4 + i / kP, gx = X0 - 4 + i % kP;
      const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
      const void* src = in ? static_cast<const void*>(reinterpret_cast<const uint4*>(feat) + (size_t)gy * a.W + gx)
                           : feat;
      const unsigned d = smem_u32(feat_s + 16 * i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(in ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // descriptors of the operands at M tile 0; a tap, an input plane or an M
  // tile adds to the start-address field (16-byte units, no carry below 256 KB)
  uint64_t ad1[5], bd1[5];
#pragma unroll
  for (int j = 0; j < 5; j++) {
    const int o0 = tap_off(2 * j), o1 = tap_off(2 * j + 1);
    ad1[j] = mat_desc(smem_u32(feat_s) + 16u * (uint32_t)o0, 16u * (uint32_t)(o1 - o0), 128u);
    bd1[j] = mat_desc(w_base + (uint32_t)j * 2u * kC * 16u, kC * 16u, 128u);
  }
  const uint64_t ad2 = mat_desc(smem_u32(bufx), kPlane1, 128u), bd2 = mat_desc(w2_base, kC * 16u, 128u);
  const uint64_t ad3 = mat_desc(smem_u32(bufy), kPlane2, 128u), bd3 = mat_desc(w3_base, kC * 16u, 128u);
  const uint64_t ad4 = mat_desc(smem_u32(bufx), kPlane1, 128u), bd4 = mat_desc(w4_base, 16u * 16u, 128u);

  // epilogue of one M tile of a layer: this warp's 32 rows (its TMEM lane
  // quarter) -> bias, ReLU, bf16 -> the next layer's planes; the last layer
  // writes the probability and the decisions
  auto epilogue = [&](int layer, int mt, int X0, int Y0, const InferPass& out) {
    const int rg0 = 4 - (layer + 1);                  // region origin offset of the output
    const int wl = kP - 2 * (layer + 1);              // valid region width
    const int m = 128 * mt + 32 * quad + lane;
    const int i = m / kP, jj = m - i * kP;
    if (layer < 3) {
      uint8_t* dst = layer == 1 ? bufy : bufx;
      const int plane = layer == 1 ? kPlane2 : kPlane1;
      const float* bl = bias + kC * layer;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(kC * mt), v);
      const int gy = Y0 - rg0 + i, gx = X0 - rg0 + jj;
      const bool keep = jj < wl && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
#pragma unroll
      for (int cgrp = 0; cgrp < 4; cgrp++) {
        uint32_t w4[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const float lo = keep ? fmaxf(v[8 * cgrp + 2 * e] + bl[8 * cgrp + 2 * e], 0.0f) : 0.0f;
          const float hi = keep ? fmaxf(v[8 * cgrp + 2 * e + 1] + bl[8 * cgrp + 2 * e + 1], 0.0f) : 0.0f;
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
          w4[e] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(dst + cgrp * plane + 16 * m) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    } else {
      const float z = tmem_ld1(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(16 * mt)) + bias[3 * kC];
      const int gy = Y0 + i, gx = X0 + jj;
      if (jj < kTX && gy < a.H && gx < a.W) {
        const float prob = 1.0f / (1.0f + expf(-z));
        const size_t pix = (size_t)gy * a.W + gx;
        if (out.prob) out.prob[pix] = prob;
        if (out.valid || out.disp) {
          const bool ok = gx - (int)out.dint[pix] >= 0 && prob >= a.threshold;
          if (out.valid) out.valid[pix] = ok ? 1 : 0;
          if (out.disp) out.disp[pix] = ok ? out.dsub[pix] : __int_as_float(0x7fc00000);
        }
      }
    }
  };

  // Per layer the issuer commits the MMAs of each pair of M tiles to that
  // pair's mbarrier; the epilogue warps take the pairs as they complete
  // (warps 0-3 the even tile of a pair, 4-7 the odd one), so the epilogue of
  // one pair overlaps the MMAs of the next.  Layers overlap too: every
  // epilogue thread arrives on the pair's "done" mbarrier once its outputs
  // are in shared memory and its accumulator columns are read, and the
  // issuer starts pair pi of layer l + 1 once pairs 0 .. pi + 1 of layer l
  // are done (output rows of M tiles 2 pi, 2 pi + 1 read the input M tiles up
  // to 2 pi + 3: a 3x3 tap reaches 2 kP + 2 pixels ahead; those tiles' TMEM
  // columns are the ones reused).  The layer-3 activations take the layer-1
  // plane stride, so a write into M tile m of the shared buffer can only
  // meet reads of layer-1 M tiles <= m, all complete by then.  A CTA
  // barrier separates tiles.
  const bool epi = warp < kEpiWarps;
  const uint32_t epp = smem_u32(sm + kSmEp);
  uint32_t phases = 0;                                // parity of each pair's MMA mbarrier
  uint32_t ep_par = 0;                                // parity of each pair's "done" mbarrier (issuer)
  bool timed_out = false;                             // sticky per thread
  if (epi && blockIdx.x < ntiles) fetch_features(blockIdx.x);
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int ps = tile / per_pass, tl = tile - ps * per_pass;
    const InferPass& out = a.pass[ps];
    const int X0 = (tl % tiles_x) * kTX, Y0 = (tl / tiles_x) * kTY;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();

    for (int layer = 0; layer < 4; layer++) {
      const int nm = region_rows(layer + 1) * kP / 128;
      const int npairs = (nm + 1) / 2;
      const int prev_pairs = layer > 0 ? (region_rows(layer) * kP / 128 + 1) / 2 : 0;
      const int N = layer == 3 ? 16 : kC;
      if (warp == kIssuer) {
        // ---- issue: warp-uniform descriptors, one elected lane per MMA ----
        fence_after();
        const uint32_t idesc = instr_desc(N);
        const uint64_t ab = layer == 1 ? ad2 : layer == 2 ? ad3 : ad4;
        const uint64_t bb = layer == 1 ? bd2 : layer == 2 ? bd3 : bd4;
        const uint32_t plane16 = (layer == 2 ? kPlane2 : kPlane1) / 16;
        int q_next = 0;   // next pair of the previous layer to wait for
        // wait (bounded) until pairs < q_end of the previous layer are done
        auto wait_prev = [&](int q_end) {
          for (; q_next < q_end && !timed_out; q_next++) {
            long long spins = 0;
            while (!bar_try_wait(epp + 8u * (uint32_t)q_next, (ep_par >> q_next) & 1u)) {
              if (++spins > kMmaSpin) {
                timed_out = true;
                break;
              }
            }
            ep_par ^= 1u << q_next;
          }
          fence_after();
        };
        for (int pi = 0; pi < npairs && !timed_out; pi++) {
          if (layer > 0) wait_prev(min(pi + 2, prev_pairs));
          if (timed_out) break;
          for (int mt = 2 * pi; mt < 2 * pi + 2 && mt < nm; mt++) {
            if (layer == 0) {
#pragma unroll
              for (int j = 0; j < 5; j++)
                if (elect_one()) mma_bf16(tmem + (uint32_t)(kC * mt), ad1[j] + 128u * mt, bd1[j], idesc, j > 0);
            } else {
              const uint64_t am = ab + 128u * mt;
#pragma unroll
              for (int t = 0; t < 9; t++) {
#pragma unroll
                for (int s = 0; s < 2; s++)
                  if (elect_one())
                    mma_bf16(tmem + (uint32_t)(N * mt), am + 2u * s * plane16 + (uint32_t)tap_off(t),
                             bb + (uint32_t)(2 * t + s) * 2u * N, idesc, (t | s) != 0);
              }
            }
          }
          if (elect_one()) mma_commit(barp + 8u * (uint32_t)pi);
          __syncwarp();
        }
        // every phase of the previous layer is waited for, in order
        if (layer > 0) wait_prev(prev_pairs);
      } else if (!timed_out) {
        // ---- epilogue, pair by pair (bounded waits) ----
        for (int pi = 0; pi < npairs; pi++) {
          long long spins = 0;
          while (!bar_try_wait(barp + 8u * (uint32_t)pi, (phases >> pi) & 1u)) {
            if (++spins > kMmaSpin) {
              timed_out = true;
              break;
            }
          }
          phases ^= 1u << pi;
          if (timed_out) break;
          fence_after();
          const int mt = 2 * pi + half;
          if (mt < nm) epilogue(layer, mt, X0, Y0, out);
          if (layer < 3) {
            // outputs visible to the tensor cores, accumulator columns read
            fence_async_smem();
            fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(epp + 8u * (uint32_t)pi) : "memory");
          }
        }
        // every MMA of layer 1 has completed: the next tile's features may come in
        if (layer == 0 && !timed_out && tile + (int)gridDim.x < ntiles) fetch_features(tile + gridDim.x);
      }
    }
    fence_async_smem();
    fence_before();
    failed = __syncthreads_or(timed_out) != 0;
    if (failed && tid == 0 && a.err) atomicExch(a.err, 1);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy left in flight
  if (warp == kIssuer) {
    // no MMA left in flight before the TMEM is freed (a no-op unless a wait gave up)
    if (elect_one()) mma_commit(barp + 8u * (uint32_t)kMaxPairs);
    __syncwarp();
    long long spins = 0;
    while (!bar_try_wait(barp + 8u * (uint32_t)kMaxPairs, 0u) && ++spins <= kMmaSpin) {
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// 4. training kernels (fp32 CUDA cores)
// ---------------------------------------------------------------------------
constexpr int kTTX = 16, kTTY = 8;            // training tile (one thread per pixel)

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// fp32 copy of the parameters with every weight rounded to bf16 (biases kept)
__global__ void round_weights_kernel(const float* __restrict__ th, float* __restrict__ wr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParamCount) return;
  const bool is_bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) ||
                       (i >= kOffB3 && i < kOffW4) || i == kOffB4;
  wr[i] = is_bias ? th[i] : bf16_round(th[i]);
}

// Layer input as fp32: bf16 features (layer 1) or stored activations.
template <int CI>
__device__ __forceinline__ void load_in_tile(const void* in, bool in_bf16, float* tile, int b, int H, int W,
                                             int y0, int x0) {
  const int n = (kTTY + 2) * (kTTX + 2) * CI;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ci = i % CI, p = i / CI;
    const int ty = p / (kTTX + 2), tx = p % (kTTX + 2);
    const int gy = y0 - 1 + ty, gx = x0 - 1 + tx;
    float v = 0.0f;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
      const size_t idx = (((size_t)b * H + gy) * W + gx) * CI + ci;
      v = in_bf16 ? __bfloat162float(__ushort_as_bfloat16(reinterpret_cast<const uint16_t*>(in)[idx]))
                  : reinterpret_cast<const float*>(in)[idx];
    }
    tile[i] = v;
  }
}

// z = b + conv3x3(a_in, wr); out = bf16(relu(z)) (hidden layers) or z (last).
template <int CI, int CO, bool HIDDEN>
__global__ void __launch_bounds__(kTTX * kTTY) fwd_kernel(const void* in, int in_bf16, const float* wr, int woff,
                                                        int boff, float* out, int H, int W) {
  extern __shared__ float dsm[];
  float* tile = dsm;                                   // [(kTTY + 2) * (kTTX + 2) * CI]
  float* ws = dsm + (kTTY + 2) * (kTTX + 2) * CI;      // [CO * 9 * CI]
  const int tx_n = (W + kTTX - 1) / kTTX, ty_n = (H + kTTY - 1) / kTTY;
  const int b = blockIdx.x / (tx_n * ty_n), r = blockIdx.x % (tx_n * ty_n);
  const int y0 = (r / tx_n) * kTTY, x0 = (r % tx_n) * kTTX;
  load_in_tile<CI>(in, in_bf16 != 0, tile, b, H, W, y0, x0);
  for (int i = threadIdx.x; i < CO * 9 * CI; i += blockDim.x) ws[i] = wr[woff + i];
  __syncthreads();
  const int ly = threadIdx.x / kTTX, lx = threadIdx.x % kTTX;
  const int y = y0 + ly, x = x0 + lx;
  if (y >= H || x >= W) return;
  float acc[CO];
#pragma unroll
  for (int co = 0; co < CO; co++) acc[co] = wr[boff + co];
  for (int t = 0; t < 9; t++) {
    const float* ip = tile + ((ly + t / 3) * (kTTX + 2) + lx + t % 3) * CI;
    for (int ci = 0; ci < CI; ci++) {
      const float v = ip[ci];
#pragma unroll
      for (int co = 0; co < CO; co++) acc[co] = fmaf(ws[(co * 9 + t) * CI + ci], v, acc[co]);
    }
  }
  float* op = out + (((size_t)b * H + y) * W + x) * CO;
#pragma unroll
  for (int co = 0; co < CO; co++) op[co] = HIDDEN ? bf16_round(fmaxf(acc[co], 0.0f)) : acc[co];
}

// dz_in(p)[ci] = [a_in(p)[ci] > 0] * sum over taps, co of wr[co][t][ci] dz_out(p - t + 1)[co]
template <int CI, int CO>
__global__ void __launch_bounds__(kTTX * kTTY) bwd_data_kernel(const float* dz_out, const float* wr, int woff,
                                                             const float* a_in, float* dz_in, int H, int W) {
  extern __shared__ float dsm[];
  float* tile = dsm;                                   // [(kTTY + 2) * (kTTX + 2) * CO]
  float* ws = dsm + (kTTY + 2) * (kTTX + 2) * CO;      // [CO * 9 * CI]
  const int tx_n = (W + kTTX - 1) / kTTX, ty_n = (H + kTTY - 1) / kTTY;
  const int b = blockIdx.x / (tx_n * ty_n), r = blockIdx.x % (tx_n * ty_n);
  const int y0 = (r / tx_n) * kTTY, x0 = (r % tx_n) * kTTX;
  load_in_tile<CO>(dz_out, false, tile, b, H, W, y0, x0);
  for (int i = threadIdx.x; i < CO * 9 * CI; i += blockDim.x) ws[i] = wr[woff + i];
  __syncthreads();
  const int ly = threadIdx.x / kTTX, lx = threadIdx.x % kTTX;
  const int y = y0 + ly, x = x0 + lx;
  if (y >= H || x >= W) return;
  float acc[CI];
#pragma unroll
  for (int ci = 0; ci < CI; ci++) acc[ci] = 0.0f;
  for (int t = 0; t < 9; t++) {
    // dz_out at p - (ky - 1, kx - 1): tile coordinates (ly + 2 - ky, lx + 2 - kx)
    const float* dp = tile + ((ly + 2 - t / 3) * (kTTX + 2) + lx + 2 - t % 3) * CO;
    for (int co = 0; co < CO; co++) {
      const float g = dp[co];
#pragma unroll
      for (int ci = 0; ci < CI; ci++) acc[ci] = fmaf(ws[(co * 9 + t) * CI + ci], g, acc[ci]);
    }
  }
  const size_t base = (((size_t)b * H + y) * W + x) * CI;
#pragma unroll
  for (int ci = 0; ci < CI; ci++) dz_in[base + ci] = a_in[base + ci] > 0.0f ? acc[ci] : 0.0f;
}

// Partial weight and bias gradients of one tile: part[blk][CO*9*CI + CO].
template <int CI, int CO>
__global__ void __launch_bounds__(256) wgrad_kernel(const float* dz, const void* a_in, int in_bf16, float* part,
                                                  int H, int W) {
  __shared__ float tile[(kTTY + 2) * (kTTX + 2) * CI];
  __shared__ float dzs[kTTY * kTTX * CO];
  const int tx_n = (W + kTTX - 1) / kTTX, ty_n = (H + kTTY - 1) / kTTY;
  const int b = blockIdx.x / (tx_n * ty_n), r = blockIdx.x % (tx_n * ty_n);
  const int y0 = (r / tx_n) * kTTY, x0 = (r % tx_n) * kTTX;
  load_in_tile<CI>(a_in, in_bf16 != 0, tile, b, H, W, y0, x0);
  for (int i = threadIdx.x; i < kTTY * kTTX * CO; i += blockDim.x) {
    const int co = i % CO, p = i / CO;
    const int gy = y0 + p / kTTX, gx = x0 + p % kTTX;
    dzs[i] = (gy < H && gx < W) ? dz[(((size_t)b * H + gy) * W + gx) * CO + co] : 0.0f;
  }
  __syncthreads();
  constexpr int NW = CO * 9 * CI;
  float* out = part + (size_t)blockIdx.x * (NW + CO);
  for (int e = threadIdx.x; e < NW + CO; e += blockDim.x) {
    float acc = 0.0f;
    if (e < NW) {
      const int ci = e % CI, t = (e / CI) % 9, co = e / (9 * CI);
      for (int p = 0; p < kTTY * kTTX; p++) {
        const int ly = p / kTTX, lx = p % kTTX;
        acc = fmaf(dzs[p * CO + co], tile[((ly + t / 3) * (kTTX + 2) + lx + t % 3) * CI + ci], acc);
      }
    } else {
      const int co = e - NW;
      for (int p = 0; p < kTTY * kTTX; p++) acc += dzs[p * CO + co];
    }
    out[e] = acc;
  }
}

// grad[off + e] = sum over blocks of part[blk][e], in block order
__global__ void reduce_parts_kernel(const float* part, int nblk, int n, float* grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float acc = 0.0f;
  for (int k = 0; k < nblk; k++) acc += part[(size_t)k * n + e];
  grad[e] = acc;
}

// Loss partials per block: [sum w, sum w * (softplus(z) - y z)]
__global__ void loss_parts_kernel(const float* z, const uint8_t* lab, size_t n, float w_neg, float* part) {
  __shared__ float sw[256], sl[256];
  float aw = 0.0f, al = 0.0f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint8_t y = lab[i];
    const float w = y == 1 ? 1.0f : (y == 0 ? w_neg : 0.0f);
    if (w != 0.0f) {
      const float zz = z[i];
      const float sp = fmaxf(zz, 0.0f) + log1pf(expf(-fabsf(zz)));
      aw += w;
      al += w * (sp - (y == 1 ? zz : 0.0f));
    }
  }
  sw[threadIdx.x] = aw;
  sl[threadIdx.x] = al;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sw[threadIdx.x] += sw[threadIdx.x + o];
      sl[threadIdx.x] += sl[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sw[0];
    part[2 * blockIdx.x + 1] = sl[0];
  }
}

__global__ void loss_final_kernel(const float* part, int nblk, float* tot, float* loss_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float sw = 0.0f, sl = 0.0f;
  for (int k = 0; k < nblk; k++) {
    sw += part[2 * k];
    sl += part[2 * k + 1];
  }
  tot[0] = sw;
  if (loss_out) *loss_out = sw > 0.0f ? sl / sw : 0.0f;
}

// dz4 = w (sigmoid(z) - y) / sum w
__global__ void loss_grad_kernel(const float* z, const uint8_t* lab, size_t n, float w_neg, const float* tot,
                                 float* dz) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t y = lab[i];
  const float w = y == 1 ? 1.0f : (y == 0 ? w_neg : 0.0f);
  const float zz = z[i];
  const float e = expf(-fabsf(zz));
  const float sig = zz >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
  dz[i] = tot[0] > 0.0f ? w * (sig - (y == 1 ? 1.0f : 0.0f)) / tot[0] : 0.0f;
}

__global__ void adam_kernel(float* th, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// Per-pixel form (D % 8 == 0): one thread per pixel walks its curves in
// chunks of 32 disparities (whole 32-byte sectors of S, of the horizontal
// paths and of the partial-sum words, all loads issued before the
// arithmetic), then 8 at a time for a tail, and keeps every statistic
// online, so no warp reduction is needed:
//   - S0, d*: first strict minimum;
//   - S2 (min over |d - d*| >= 2): when a new minimum appears at d, the
//     candidates so far are those at d' <= d - 2, whose minimum is the prefix
//     minimum lagged by two; afterwards every d >= d* + 2 joins;
//   - S(d* - 1) is the value preceding the new minimum, S(d* + 1) is taken
//     when d = d* + 1 (0 where out of range, as in the other forms);
//   - the three group winners as (value << 8 | d) minima.
constexpr uint32_t kBig = 0xffffffffu;   // "no value yet" in the online minima

struct PxState {
  uint32_t kh, kd, ku, s0, m2, lag, prev, vm, vp;
  int ds;
};

// Eight disparities d0 .. d0+7: S words (two u16 each), horizontal bytes
// (forward and backward, four per word), partial-sum words (the pixel's half).
__device__ __forceinline__ void px_step8(PxState& st, int d0, const uint32_t* sw, uint32_t f0, uint32_t f1,
                                         uint32_t b0, uint32_t b1, const uint32_t* ww, int hi) {
#pragma unroll
  for (int e = 0; e < 8; e++) {
    const uint32_t d = (uint32_t)(d0 + e);
    const uint32_t sv = (e & 1) ? sw[e >> 1] >> 16 : sw[e >> 1] & 0xffffu;
    const uint32_t fb = e < 4 ? f0 : f1, bb = e < 4 ? b0 : b1;
    const uint32_t gh = ((fb >> (8 * (e & 3))) & 0xffu) + ((bb >> (8 * (e & 3))) & 0xffu);
    const uint32_t gd = hi ? ww[e] >> 16 : ww[e] & 0xffffu;
    st.kh = min(st.kh, (gh << 8) | d);
    st.kd = min(st.kd, (gd << 8) | d);
    st.ku = min(st.ku, ((sv - gh - gd) << 8) | d);
    if (sv < st.s0) {
      st.s0 = sv;
      st.ds = (int)d;
      st.m2 = st.lag;
      st.vm = d > 0 ? st.prev : 0u;
      st.vp = 0u;
    } else {
      if ((int)d >= st.ds + 2) st.m2 = min(st.m2, sv);
      if ((int)d == st.ds + 1) st.vp = sv;
    }
    st.lag = min(st.lag, st.prev);
    st.prev = sv;
  }
}

// Staged form's statistics: the three group winners as in px_step8; S0, d*,
// S2 and the neighbours of d* at the granularity of blocks of eight
// disparities (one 16-byte word of S): the first block holding the strict
// minimum (bb, s0), and m2 = the minimum over blocks at least two blocks away
// from bb (the prefix minimum lagged by two blocks when a new best block
// appears, every block from bb + 2 on afterwards).  Blocks bb - 1 .. bb + 1
// are read again once d* is known (blk_finish).
struct BlkState {
  uint32_t kh, kd, ku, s0, m2, lag, prev;
  int bb;
};

__device__ __forceinline__ void blk_step8(BlkState& st, int d0, const uint32_t* sw, uint32_t f0, uint32_t f1,
                                          uint32_t b0, uint32_t b1, const uint32_t* ww, int hi) {
#pragma unroll
  for (int e = 0; e < 8; e++) {
    const uint32_t d = (uint32_t)(d0 + e);
    const uint32_t sv = (e & 1) ? sw[e >> 1] >> 16 : sw[e >> 1] & 0xffffu;
    const uint32_t fb = e < 4 ? f0 : f1, bb = e < 4 ? b0 : b1;
    const uint32_t gh = ((fb >> (8 * (e & 3))) & 0xffu) + ((bb >> (8 * (e & 3))) & 0xffu);
    const uint32_t gd = hi ? ww[e] >> 16 : ww[e] & 0xffffu;
    st.kh = min(st.kh, (gh << 8) | d);
    st.kd = min(st.kd, (gd << 8) | d);
    st.ku = min(st.ku, ((sv - gh - gd) << 8) | d);
  }
  // the block's minimum from its packed words, then the block statistics
  const uint32_t p = __vminu2(__vminu2(sw[0], sw[1]), __vminu2(sw[2], sw[3]));
  const uint32_t bm = min(p & 0xffffu, p >> 16);
  const int b = d0 >> 3;
  if (bm < st.s0) {
    st.s0 = bm;
    st.bb = b;
    st.m2 = st.lag;
  } else if (b >= st.bb + 2) {
    st.m2 = min(st.m2, bm);
  }
  st.lag = min(st.lag, st.prev);
  st.prev = bm;
}

// d*, S(d* - 1), S(d* + 1) and S2 from blocks bb - 1 .. bb + 1 of the
// pixel's S row, then the common tail.
__device__ __forceinline__ void blk_finish(const FeatureArgs& a, const BlkState& st, size_t pix, int x);

// Features, winner and subpixel winner of pixel `pix` (column x) from its
// online statistics.
__device__ __forceinline__ void px_finish(const FeatureArgs& a, const PxState& st, size_t pix, int x) {
  const uint32_t kh = st.kh, kd = st.kd, ku = st.ku, s0 = st.s0, m2 = st.m2, vm = st.vm, vp = st.vp;
  const int ds = st.ds;
  const int cstar = a.cost[pix * a.Dp + ds];
  const uint32_t s2 = m2 == kBig ? s0 : m2;
  int curv = 0;
  if (a.D > 1) {
    if (ds == 0)
      curv = 2 * ((int)vp - (int)s0);
    else if (ds == a.D - 1)
      curv = 2 * ((int)vm - (int)s0);
    else
      curv = (int)vm + (int)vp - 2 * (int)s0;
  }
  const int dis = min(abs((int)(kh & 0xffu) - ds), 16) + min(abs((int)(kd & 0xffu) - ds), 16) +
                  min(abs((int)(ku & 0xffu) - ds), 16);
  const int margin = min(max(x - ds, 0), 64);
  const float f[kF] = {(float)s0 * (1.0f / 1024.0f), (float)(s2 - s0) * (1.0f / 256.0f),
                       (float)curv * (1.0f / 256.0f), (float)dis * (1.0f / 16.0f),
                       (float)ds * (1.0f / 128.0f),   (float)margin * (1.0f / 64.0f),
                       (float)cstar * (1.0f / 64.0f), 0.0f};   // channel 7: visibility_kernel
  uint32_t packed[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    packed[i] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  reinterpret_cast<uint4*>(a.feat)[pix] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  a.dint[pix] = (int16_t)ds;
  float v = (float)ds;
  if (a.subpixel && ds > 0 && ds < a.D - 1) {
    const int am = (int)vm - (int)s0, bp = (int)vp - (int)s0;
    v = __fadd_rn((float)ds, __fdiv_rn((float)(am - bp), (float)(2 * (am + bp))));
  }
  a.dsub[pix] = v;
}

__device__ __forceinline__ void blk_finish(const FeatureArgs& a, const BlkState& st, size_t pix, int x) {
  const int nb = a.D >> 3, b = st.bb;
  const uint4* srow = reinterpret_cast<const uint4*>(a.S + pix * a.D);
  // S of blocks b - 1 .. b + 1 (kBig outside the curve), as 12 words of two
  uint32_t w[12];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const int bj = b - 1 + j;
    uint4 q = make_uint4(kBig, kBig, kBig, kBig);
    if (bj >= 0 && bj < nb) q = __ldg(srow + bj);
    w[4 * j + 0] = q.x;
    w[4 * j + 1] = q.y;
    w[4 * j + 2] = q.z;
    w[4 * j + 3] = q.w;
  }
  auto v = [&](int i) { return (i & 1) ? w[i >> 1] >> 16 : w[i >> 1] & 0xffffu; };
  // first disparity of block b reaching the minimum
  int e0 = 7;
#pragma unroll
  for (int e = 7; e >= 0; e--)
    if (v(8 + e) == st.s0) e0 = e;
  PxState ps{st.kh, st.kd, st.ku, st.s0, st.m2, 0u, 0u, 0u, 0u, 8 * b + e0};
  // d* sits at index i0 = 8 + e0 of v (8..15), so indices 0..6 and 17..23
  // are always two or more away; the others are selected by constant
  // indices (no indexed register array)
  const int i0 = 8 + e0;
  uint32_t vm = 0u, vp = 0u;
#pragma unroll
  for (int e = 0; e < 8; e++) {
    vm = e == e0 ? v(7 + e) : vm;
    vp = e == e0 ? v(9 + e) : vp;
  }
#pragma unroll
  for (int i = 0; i < 7; i++) ps.m2 = min(ps.m2, min(v(i), v(17 + i)));
#pragma unroll
  for (int i = 7; i < 17; i++) ps.m2 = (i <= i0 - 2 || i >= i0 + 2) ? min(ps.m2, v(i)) : ps.m2;
  // (past either end of the curve v reads 0xffff, above every S; the
  // neighbours there are 0 as in the other forms)
  ps.vm = ps.ds > 0 ? vm : 0u;
  ps.vp = ps.ds < a.D - 1 ? vp : 0u;
  px_finish(a, ps, pix, x);
}


__global__ void __launch_bounds__(256, 2)
    features_px_kernel(FeatureArgs a) {
  const size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (size_t)a.W * a.H) return;
  const int y = (int)(pix / a.W), x = (int)(pix - (size_t)y * a.W);
  const int j = x >> 5, pr = x & 15, hi = (x >> 4) & 1;
  const uint4* srow = reinterpret_cast<const uint4*>(a.S + pix * a.D);       // 8 disparities each
  const uint4* hfr = reinterpret_cast<const uint4*>(a.hfwd + pix * a.Dp);    // 16 disparities each
  const uint4* hbr = reinterpret_cast<const uint4*>(a.hbwd + pix * a.Dp);
  const uint4* sdr =
      reinterpret_cast<const uint4*>(a.sdown + (((size_t)y * a.J + j) * 16 + pr) * (size_t)a.dpad_shape);
  PxState st{kBig, kBig, kBig, kBig, kBig, kBig, kBig, 0u, 0u, 0};
  int d0 = 0;
  for (; d0 + 32 <= a.D; d0 += 32) {
    uint4 sv[4], fv[2], bv[2], wv[8];
#pragma unroll
    for (int i = 0; i < 4; i++) sv[i] = __ldg(srow + (d0 >> 3) + i);
#pragma unroll
    for (int i = 0; i < 2; i++) {
      fv[i] = __ldg(hfr + (d0 >> 4) + i);
      bv[i] = __ldg(hbr + (d0 >> 4) + i);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) wv[i] = __ldg(sdr + (d0 >> 2) + i);
#pragma unroll
    for (int g = 0; g < 4; g++) {
      const uint32_t sw[4] = {sv[g].x, sv[g].y, sv[g].z, sv[g].w};
      const uint4 f = fv[g >> 1], b = bv[g >> 1];
      const uint32_t f0 = (g & 1) ? f.z : f.x, f1 = (g & 1) ? f.w : f.y;
      const uint32_t b0 = (g & 1) ? b.z : b.x, b1 = (g & 1) ? b.w : b.y;
      const uint32_t ww[8] = {wv[2 * g].x,     wv[2 * g].y,     wv[2 * g].z,     wv[2 * g].w,
                              wv[2 * g + 1].x, wv[2 * g + 1].y, wv[2 * g + 1].z, wv[2 * g + 1].w};
      px_step8(st, d0 + 8 * g, sw, f0, f1, b0, b1, ww, hi);
    }
  }
  for (; d0 < a.D; d0 += 8) {
    const uint4 s8 = __ldg(srow + (d0 >> 3));
    const uint2 f8 = __ldg(reinterpret_cast<const uint2*>(a.hfwd + pix * a.Dp) + (d0 >> 3));
    const uint2 b8 = __ldg(reinterpret_cast<const uint2*>(a.hbwd + pix * a.Dp) + (d0 >> 3));
    const uint4 wa = __ldg(sdr + (d0 >> 2)), wb = __ldg(sdr + (d0 >> 2) + 1);
    const uint32_t sw[4] = {s8.x, s8.y, s8.z, s8.w};
    const uint32_t ww[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    px_step8(st, d0, sw, f8.x, f8.y, b8.x, b8.y, ww, hi);
  }
  px_finish(a, st, pix, x);
}

// Staged form (D % 32 == 0): a block of 128 threads takes 128 columns of
// one row.  Each chunk of 32 disparities of S, of the two horizontal paths
// and of the partial-sum words comes into shared memory by coalesced 16-byte
// asynchronous copies (double-buffered: the next chunk's copies run while
// this one is consumed); each thread then reads its own pixel's rows, padded
// by 16 bytes so that a warp's 16-byte reads spread over all banks, and
// updates the group winners per disparity and S0 / S2 per block of eight
// (blk_step8), reading the three blocks around the best one again at the end.
constexpr int kStThreads = 128;
constexpr int kStS = 80, kStH = 48, kStW = 144;              // padded row bytes
constexpr int kStStage = kStThreads * (kStS + 2 * kStH) + 4 * 16 * kStW;
constexpr int kStSmem = 2 * kStStage;

__device__ __forceinline__ void cp16(uint8_t* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

__global__ void __launch_bounds__(kStThreads)
    features_staged_kernel(FeatureArgs a) {
  extern __shared__ __align__(16) uint8_t fsm[];
  const int segs = (a.W + kStThreads - 1) / kStThreads;
  const int y = blockIdx.x / segs, x0 = (blockIdx.x - y * segs) * kStThreads;
  const int tid = threadIdx.x, x = x0 + tid;
  const int ncols = min(kStThreads, a.W - x0);
  const int strips = (ncols + 31) / 32, j0 = x0 / 32;
  const size_t row0 = (size_t)y * a.W + x0;
  auto load_chunk = [&](int d0, int stage) {
    uint8_t* sS = fsm + stage * kStStage;
    uint8_t* sF = sS + kStThreads * kStS;
    uint8_t* sB = sF + kStThreads * kStH;
    uint8_t* sW = sB + kStThreads * kStH;
    for (int c = tid; c < kStThreads * 4; c += kStThreads) {
      const int px = c >> 2, part = c & 3;
      if (px < ncols) cp16(sS + px * kStS + part * 16, a.S + (row0 + px) * a.D + d0 + part * 8);
    }
    for (int c = tid; c < kStThreads * 2; c += kStThreads) {
      const int px = c >> 1, part = c & 1;
      if (px < ncols) {
        cp16(sF + px * kStH + part * 16, a.hfwd + (row0 + px) * a.Dp + d0 + part * 16);
        cp16(sB + px * kStH + part * 16, a.hbwd + (row0 + px) * a.Dp + d0 + part * 16);
      }
    }
    for (int c = tid; c < 4 * 16 * 8; c += kStThreads) {
      const int r = c >> 3, part = c & 7, sl = r >> 4, pr = r & 15;
      if (sl < strips)
        cp16(sW + r * kStW + part * 16,
             a.sdown + (((size_t)y * a.J + j0 + sl) * 16 + pr) * (size_t)a.dpad_shape + d0 + part * 4);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  BlkState st{kBig, kBig, kBig, kBig, kBig, kBig, kBig, 0};
  const int hi = (x >> 4) & 1, wrow = ((tid >> 5) << 4) + (x & 15);
  const int nchunks = a.D / 32;
  load_chunk(0, 0);
  for (int k = 0; k < nchunks; k++) {
    if (k + 1 < nchunks) {
      load_chunk(32 * (k + 1), (k + 1) & 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (tid < ncols) {
      const uint8_t* sS = fsm + (k & 1) * kStStage;
      const uint8_t* sF = sS + kStThreads * kStS;
      const uint8_t* sB = sF + kStThreads * kStH;
      const uint8_t* sW = sB + kStThreads * kStH;
      const uint4* ps = reinterpret_cast<const uint4*>(sS + tid * kStS);
      const uint4* pf = reinterpret_cast<const uint4*>(sF + tid * kStH);
      const uint4* pb = reinterpret_cast<const uint4*>(sB + tid * kStH);
      const uint4* pw = reinterpret_cast<const uint4*>(sW + wrow * kStW);
#pragma unroll
      for (int g = 0; g < 4; g++) {
        const uint4 sv = ps[g], wa = pw[2 * g], wb = pw[2 * g + 1];
        const uint4 f = pf[g >> 1], b = pb[g >> 1];
        const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
        const uint32_t ww[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        blk_step8(st, 32 * k + 8 * g, sw, (g & 1) ? f.z : f.x, (g & 1) ? f.w : f.y, (g & 1) ? b.z : b.x,
                  (g & 1) ? b.w : b.y, ww, hi);
      }
    }
    __syncthreads();
  }
  if (tid < ncols) blk_finish(a, st, row0 + tid, x);
}

// Channel 7, the visibility margin: pixel x of a row matches right-image
// column u(x) = x - d*(x); with m(x) the minimum of u over the pixels right of
// x, v = clamp(m - u, -16, 16) (16 for the last pixel), stored as v / 16.
// One block per row: each thread takes a contiguous segment, the minima of
// the segments to its right come from a block-wide suffix scan, then the
// thread walks its segment right to left.
constexpr int kVisThreads = 256;

__global__ void __launch_bounds__(kVisThreads)
    visibility_kernel(const int16_t* __restrict__ dint, uint16_t* __restrict__ feat, int W) {
  __shared__ int warp_suffix[kVisThreads / 32];
  constexpr int kNone = 0x7fffffff;
  const int y = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int seg = (W + kVisThreads - 1) / kVisThreads;
  const int x0 = min(t * seg, W), x1 = min(x0 + seg, W);
  const int16_t* row = dint + (size_t)y * W;
  int tot = kNone;
  for (int x = x0; x < x1; x++) tot = min(tot, x - (int)row[x]);
  // inclusive suffix minimum over the lanes >= lane of this warp
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) incl = min(incl, __shfl_down_sync(kFullMask, incl, o));
  if (lane == 0) warp_suffix[wp] = incl;
  __syncthreads();
  int m = __shfl_down_sync(kFullMask, incl, 1);
  if (lane == 31) m = kNone;
  for (int w = wp + 1; w < kVisThreads / 32; w++) m = min(m, warp_suffix[w]);
  uint16_t* f = feat + (size_t)y * W * kF + 7;
  for (int x = x1 - 1; x >= x0; x--) {
    const int u = x - (int)row[x];
    const int v = m == kNone ? 16 : max(min(m - u, 16), -16);
    f[(size_t)x * kF] = __bfloat16_as_ushort(__float2bfloat16_rn((float)v * (1.0f / 16.0f)));
    m = min(m, u);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_features(const FeatureArgs& a, cudaStream_t s) {
  count_launches(2);
  if (a.D % 32 == 0) {
    static bool attr_set = false;
    if (!attr_set) {
      const cudaError_t e =
          cudaFuncSetAttribute(features_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    const size_t blocks = (size_t)a.H * ((a.W + kStThreads - 1) / kStThreads);
    features_staged_kernel<<<(unsigned)blocks, kStThreads, kStSmem, s>>>(a);
  } else if (a.D % 8 == 0) {
    const size_t threads = (size_t)a.W * a.H;
    features_px_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  } else if (a.D % 4 == 0) {
    const size_t threads = (size_t)a.J * 16 * a.H * 32;
    if (a.D <= 128)
      features_vec_kernel<1><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    else
      features_vec_kernel<2><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  } else {
    const size_t threads = (size_t)a.J * 16 * a.H * 32;
    features_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  }
  visibility_kernel<<<(unsigned)a.H, kVisThreads, 0, s>>>(a.dint, a.feat, a.W);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* params, void* packed, cudaStream_t s) {
  count_launches(1);
  pack_kernel<<<(kWElems + 255) / 256, 256, 0, s>>>(params, reinterpret_cast<uint16_t*>(packed));
  return cudaGetLastError();
}

cudaError_t launch_infer(const InferArgs& a, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (a.npass < 1 || a.npass > kMaxInferPass) return cudaErrorInvalidValue;
  const int ntiles = ((a.W + kTX - 1) / kTX) * ((a.H + kTY - 1) / kTY) * a.npass;
  count_launches(1);
  infer_kernel<<<(unsigned)std::min(ntiles, sms), kThreads, kSmTotal, s>>>(a);
  return cudaGetLastError();
}

template <int CI, int CO, bool HIDDEN>
void fwd(const void* in, int in_bf16, const float* wr, int woff, int boff, float* out, int H, int W, int nblk,
         cudaStream_t s) {
  const size_t smem = ((size_t)(kTTY + 2) * (kTTX + 2) * CI + (size_t)CO * 9 * CI) * 4;
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(fwd_kernel<CI, CO, HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    set = true;
  }
  fwd_kernel<CI, CO, HIDDEN><<<nblk, kTTX * kTTY, smem, s>>>(in, in_bf16, wr, woff, boff, out, H, W);
}

template <int CI, int CO>
void bwd_data(const float* dz_out, const float* wr, int woff, const float* a_in, float* dz_in, int H, int W,
              int nblk, cudaStream_t s) {
  const size_t smem = ((size_t)(kTTY + 2) * (kTTX + 2) * CO + (size_t)CO * 9 * CI) * 4;
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(bwd_data_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    set = true;
  }
  bwd_data_kernel<CI, CO><<<nblk, kTTX * kTTY, smem, s>>>(dz_out, wr, woff, a_in, dz_in, H, W);
}

size_t train_workspace_bytes(int B, int W, int H) {
  const size_t npx = (size_t)B * W * H;
  const size_t nblk = (size_t)B * ((H + kTTY - 1) / kTTY) * ((W + kTTX - 1) / kTTX);
  size_t o = 0;
  auto carve = [&](size_t bytes) { o = align_up(o + bytes, 256); };
  carve(kParamCount * 4);          // rounded weights
  carve(kParamCount * 4);          // gradient
  carve(3 * npx * kC * 4);         // a1, a2, a3
  carve(npx * 4);                  // z4
  carve(2 * npx * kC * 4);         // dz ping-pong
  carve(nblk * (9 * kC * kC + kC) * 4);   // weight-gradient partials
  carve(2 * 1024 * 4 + 256);       // loss partials and totals
  return o;
}

cudaError_t launch_train_step(const TrainArgs& t, cudaStream_t s) {
  const int B = t.B, W = t.W, H = t.H;
  const size_t npx = (size_t)B * W * H;
  const int nblk = B * ((H + kTTY - 1) / kTTY) * ((W + kTTX - 1) / kTTX);
  uint8_t* ws = reinterpret_cast<uint8_t*>(t.workspace);
  size_t o = 0;
  auto carve = [&](size_t bytes) {
    uint8_t* p = ws + o;
    o = align_up(o + bytes, 256);
    return p;
  };
  float* wr = reinterpret_cast<float*>(carve(kParamCount * 4));
  float* grad = reinterpret_cast<float*>(carve(kParamCount * 4));
  float* a1 = reinterpret_cast<float*>(carve(3 * npx * kC * 4));
  float* a2 = a1 + npx * kC;
  float* a3 = a2 + npx * kC;
  float* z4 = reinterpret_cast<float*>(carve(npx * 4));
  float* dzA = reinterpret_cast<float*>(carve(2 * npx * kC * 4));
  float* dzB = dzA + npx * kC;
  float* part = reinterpret_cast<float*>(carve((size_t)nblk * (9 * kC * kC + kC) * 4));
  float* lpart = reinterpret_cast<float*>(carve(2 * 1024 * 4 + 256));
  float* ltot = lpart + 2 * 1024;
  int launches = 0;
  round_weights_kernel<<<(kParamCount + 255) / 256, 256, 0, s>>>(t.params, wr);
  fwd<kF, kC, true>(t.features, 1, wr, kOffW1, kOffB1, a1, H, W, nblk, s);
  fwd<kC, kC, true>(a1, 0, wr, kOffW2, kOffB2, a2, H, W, nblk, s);
  fwd<kC, kC, true>(a2, 0, wr, kOffW3, kOffB3, a3, H, W, nblk, s);
  fwd<kC, 1, false>(a3, 0, wr, kOffW4, kOffB4, z4, H, W, nblk, s);
  launches += 5;
  if (t.logits_out) {
    cudaError_t e = cudaMemcpyAsync(t.logits_out, z4, npx * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (!t.labels) {
    count_launches(launches);
    return cudaGetLastError();
  }
  const int lblk = (int)std::min<size_t>(1024, (npx + 255) / 256);
  loss_parts_kernel<<<lblk, 256, 0, s>>>(z4, t.labels, npx, t.w_neg, lpart);
  loss_final_kernel<<<1, 32, 0, s>>>(lpart, lblk, ltot, t.loss_out);
  loss_grad_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, s>>>(z4, t.labels, npx, t.w_neg, ltot, dzA);
  launches += 3;
  // layer 4 (CI = 32, CO = 1)
  wgrad_kernel<kC, 1><<<nblk, 256, 0, s>>>(dzA, a3, 0, part, H, W);
  reduce_parts_kernel<<<(9 * kC + 1 + 255) / 256, 256, 0, s>>>(part, nblk, 9 * kC + 1, grad + kOffW4);
  bwd_data<kC, 1>(dzA, wr, kOffW4, a3, dzB, H, W, nblk, s);
  // layer 3
  wgrad_kernel<kC, kC><<<nblk, 256, 0, s>>>(dzB, a2, 0, part, H, W);
  reduce_parts_kernel<<<(9 * kC * kC + kC + 255) / 256, 256, 0, s>>>(part, nblk, 9 * kC * kC + kC, grad + kOffW3);
  bwd_data<kC, kC>(dzB, wr, kOffW3, a2, dzA, H, W, nblk, s);
  // layer 2
  wgrad_kernel<kC, kC><<<nblk, 256, 0, s>>>(dzA, a1, 0, part, H, W);
  reduce_parts_kernel<<<(9 * kC * kC + kC + 255) / 256, 256, 0, s>>>(part, nblk, 9 * kC * kC + kC, grad + kOffW2);
  bwd_data<kC, kC>(dzA, wr, kOffW2, a1, dzB, H, W, nblk, s);
  // layer 1
  wgrad_kernel<kF, kC><<<nblk, 256, 0, s>>>(dzB, t.features, 1, part, H, W);
  reduce_parts_kernel<<<(9 * kF * kC + kC + 255) / 256, 256, 0, s>>>(part, nblk, 9 * kF * kC + kC, grad + kOffW1);
  launches += 11;
  if (t.grad_out) {
    cudaError_t e = cudaMemcpyAsync(t.grad_out, grad, kParamCount * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (t.adam_m && t.adam_v) {
    const float c1 = 1.0f - powf(t.beta1, (float)t.step), c2 = 1.0f - powf(t.beta2, (float)t.step);
    adam_kernel<<<(kParamCount + 255) / 256, 256, 0, s>>>(t.params, t.adam_m, t.adam_v, grad, kParamCount, t.lr,
                                                          t.beta1, t.beta2, t.eps, c1, c2);
    launches += 1;
  }
  count_launches(launches);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* params, float* m, float* v, const float* grad, int n, float lr, float beta1,
                        float beta2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  count_launches(1);
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(params, m, v, grad, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace confnet
}  // namespace sf
