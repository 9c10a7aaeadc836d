// Device helpers for the fused SGM kernels: packed u16x2 integer arithmetic,
// byte <-> u16x2 repacking and chunk-group reductions.
//
// Packing used throughout: one 32-bit register holds the same disparity d of
// two different image lines (two columns, or two rows), one per 16-bit lane.
// The SGM recurrence is lane-wise, so one instruction advances two lines.
#pragma once

#include <stdint.h>

namespace sf {

constexpr int kDC = 16;                      // disparities per thread
constexpr uint32_t kInf2 = 0x3fff3fffu;      // "no neighbour" in both lanes
constexpr uint32_t kPadCost2 = 0x40004000u;  // cost of a padding disparity d >= D

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// PTX prmt in its default mode: a selector nibble with bit 3 set replicates
// the sign bit of the chosen byte (the CUDA __byte_perm intrinsic ignores
// that bit, so it cannot produce the zero bytes used below).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

// Two 16-byte vectors of uint8 values (line A, line B; 16 consecutive d)
// -> 16 u16x2 registers (A in the low lane, B in the high lane).  Only for
// values < 128 (matching costs): sign-replicating selector nibbles produce
// the zero high bytes in the same instruction.
__device__ __forceinline__ void bytes_to_pairs(const uint4& a, const uint4& b, uint32_t* r) {
  const uint32_t aw[4] = {a.x, a.y, a.z, a.w};
  const uint32_t bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int w = 0; w < 4; w++) {
    r[4 * w + 0] = prmt(aw[w], bw[w], 0xC480u);
    r[4 * w + 1] = prmt(aw[w], bw[w], 0xD591u);
    r[4 * w + 2] = prmt(aw[w], bw[w], 0xE6A2u);
    r[4 * w + 3] = prmt(aw[w], bw[w], 0xF7B3u);
  }
}

// Same repacking for any byte values (0..255, e.g. path costs up to
// cmax + P2): pick the bytes, then clear the high byte of each lane.
__device__ __forceinline__ void bytes_to_pairs_u8(const uint4& a, const uint4& b, uint32_t* r) {
  const uint32_t aw[4] = {a.x, a.y, a.z, a.w};
  const uint32_t bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int w = 0; w < 4; w++) {
    r[4 * w + 0] = prmt(aw[w], bw[w], 0x4400u) & 0x00ff00ffu;
    r[4 * w + 1] = prmt(aw[w], bw[w], 0x5511u) & 0x00ff00ffu;
    r[4 * w + 2] = prmt(aw[w], bw[w], 0x6622u) & 0x00ff00ffu;
    r[4 * w + 3] = prmt(aw[w], bw[w], 0x7733u) & 0x00ff00ffu;
  }
}

// Inverse of bytes_to_pairs for values < 256: 16 u16x2 registers -> the low
// lanes as 16 bytes (a) and the high lanes as 16 bytes (b).
__device__ __forceinline__ void pairs_to_bytes(const uint32_t* r, uint4& a, uint4& b) {
  uint32_t aw[4], bw[4];
#pragma unroll
  for (int w = 0; w < 4; w++) {
    const uint32_t t1 = prmt(r[4 * w + 0], r[4 * w + 1], 0x6240u);  // a0 a1 b0 b1
    const uint32_t t2 = prmt(r[4 * w + 2], r[4 * w + 3], 0x6240u);  // a2 a3 b2 b3
    aw[w] = prmt(t1, t2, 0x5410u);
    bw[w] = prmt(t1, t2, 0x7632u);
  }
  a = make_uint4(aw[0], aw[1], aw[2], aw[3]);
  b = make_uint4(bw[0], bw[1], bw[2], bw[3]);
}

// Lane-wise min over a group of G consecutive threads (G divides 32).
// `mask` names the lanes executing the call (whole groups only).
template <int G>
__device__ __forceinline__ uint32_t group_min2(uint32_t v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v = vmin2(v, __shfl_xor_sync(mask, v, o, G));
  return v;
}

// One SGM step for 16 disparities of two lines:
//   Lnew(d) = C(d) + min(Lp(d), min(Lp(d-1), Lp(d+1)) + P1, m + P2) - m
// with Lp the predecessor state, m = min_d Lp (both lanes), `left` / `right`
// the predecessor values at d0-1 / d0+16 from the neighbouring chunks.
// Returns the lane-wise minimum of the new values over these 16 d.
__device__ __forceinline__ uint32_t sgm_step16(const uint32_t* Lp, const uint32_t* C, uint32_t left,
                                               uint32_t right, uint32_t m, uint32_t p1x2,
                                               uint32_t p2x2, uint32_t* Ln) {
  const uint32_t q = m + p2x2;
  uint32_t acc = 0xffffffffu;
#pragma unroll
  for (int i = 0; i < kDC; i++) {
    const uint32_t lm = (i == 0) ? left : Lp[i - 1];
    const uint32_t lp = (i == kDC - 1) ? right : Lp[i + 1];
    uint32_t t = vmin2(lm, lp) + p1x2;
    t = vmin2(t, Lp[i]);
    t = vmin2(t, q);
    Ln[i] = t + C[i] - m;  // lane-safe: t >= m per lane
    acc = vmin2(acc, Ln[i]);
  }
  return acc;
}

}  // namespace sf
