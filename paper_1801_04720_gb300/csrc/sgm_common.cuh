// Device helpers for the fused SGM kernels: packed u16x2 integer arithmetic,
// byte <-> u16x2 repacking and chunk-group reductions.
//
// Packing used throughout: one 32-bit register holds the same disparity d of
// two different image lines (two columns, or two rows), one per 16-bit lane.
// The SGM recurrence is lane-wise, so one instruction advances two lines.
// A thread owns DC consecutive disparities (DC = 8 or 16) of its two lines.
#pragma once

#include <stdint.h>

namespace sf {

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

// DC bytes of one line as a vector type (4 -> uint32_t, 8 -> uint2,
// 16 -> uint4, 32 -> two uint4).
template <int DC> struct ByteVec;
template <> struct ByteVec<4> {
  using T = uint32_t;
  __device__ static void words(const T& v, uint32_t* w) { w[0] = v; }
  __device__ static T make(const uint32_t* w) { return w[0]; }
  __device__ static T zero() { return 0u; }
};
template <> struct ByteVec<8> {
  using T = uint2;
  __device__ static void words(const T& v, uint32_t* w) { w[0] = v.x; w[1] = v.y; }
  __device__ static T make(const uint32_t* w) { return make_uint2(w[0], w[1]); }
  __device__ static T zero() { return make_uint2(0, 0); }
};
template <> struct ByteVec<16> {
  using T = uint4;
  __device__ static void words(const T& v, uint32_t* w) { w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w; }
  __device__ static T make(const uint32_t* w) { return make_uint4(w[0], w[1], w[2], w[3]); }
  __device__ static T zero() { return make_uint4(0, 0, 0, 0); }
};
struct __align__(16) Bytes32 {
  uint4 lo, hi;
};
template <> struct ByteVec<32> {
  using T = Bytes32;
  __device__ static void words(const T& v, uint32_t* w) {
    w[0] = v.lo.x; w[1] = v.lo.y; w[2] = v.lo.z; w[3] = v.lo.w;
    w[4] = v.hi.x; w[5] = v.hi.y; w[6] = v.hi.z; w[7] = v.hi.w;
  }
  __device__ static T make(const uint32_t* w) {
    return T{make_uint4(w[0], w[1], w[2], w[3]), make_uint4(w[4], w[5], w[6], w[7])};
  }
  __device__ static T zero() { return T{make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)}; }
};

// Streaming (evict-first) store of DC bytes.
__device__ __forceinline__ void store_cs(uint32_t* p, const uint32_t& v) {
  __stcs(reinterpret_cast<unsigned int*>(p), static_cast<unsigned int>(v));
}
__device__ __forceinline__ void store_cs(uint2* p, const uint2& v) { __stcs(p, v); }
__device__ __forceinline__ void store_cs(uint4* p, const uint4& v) { __stcs(p, v); }
__device__ __forceinline__ void store_cs(Bytes32* p, const Bytes32& v) {
  __stcs(reinterpret_cast<uint4*>(p), v.lo);
  __stcs(reinterpret_cast<uint4*>(p) + 1, v.hi);
}

// Two lines' DC uint8 values -> DC u16x2 registers (line A low lane, line B
// high lane).  Only for values < 128 (matching costs): sign-replicating
// selector nibbles produce the zero high bytes in the same instruction.
template <int DC>
__device__ __forceinline__ void bytes_to_pairs(const typename ByteVec<DC>::T& a,
                                               const typename ByteVec<DC>::T& b, uint32_t* r) {
  uint32_t aw[DC / 4], bw[DC / 4];
  ByteVec<DC>::words(a, aw);
  ByteVec<DC>::words(b, bw);
#pragma unroll
  for (int w = 0; w < DC / 4; w++) {
    r[4 * w + 0] = prmt(aw[w], bw[w], 0xC480u);
    r[4 * w + 1] = prmt(aw[w], bw[w], 0xD591u);
    r[4 * w + 2] = prmt(aw[w], bw[w], 0xE6A2u);
    r[4 * w + 3] = prmt(aw[w], bw[w], 0xF7B3u);
  }
}

// Same repacking for any byte values (0..255, e.g. path costs up to
// cmax + P2): pick the bytes, then clear the high byte of each lane.
template <int DC>
__device__ __forceinline__ void bytes_to_pairs_u8(const typename ByteVec<DC>::T& a,
                                                  const typename ByteVec<DC>::T& b, uint32_t* r) {
  uint32_t aw[DC / 4], bw[DC / 4];
  ByteVec<DC>::words(a, aw);
  ByteVec<DC>::words(b, bw);
#pragma unroll
  for (int w = 0; w < DC / 4; w++) {
    r[4 * w + 0] = prmt(aw[w], bw[w], 0x4400u) & 0x00ff00ffu;
    r[4 * w + 1] = prmt(aw[w], bw[w], 0x5511u) & 0x00ff00ffu;
    r[4 * w + 2] = prmt(aw[w], bw[w], 0x6622u) & 0x00ff00ffu;
    r[4 * w + 3] = prmt(aw[w], bw[w], 0x7733u) & 0x00ff00ffu;
  }
}

// Inverse for values < 256: DC u16x2 registers -> the low lanes as DC bytes
// (a) and the high lanes as DC bytes (b).
template <int DC>
__device__ __forceinline__ void pairs_to_bytes(const uint32_t* r, typename ByteVec<DC>::T& a,
                                               typename ByteVec<DC>::T& b) {
  uint32_t aw[DC / 4], bw[DC / 4];
#pragma unroll
  for (int w = 0; w < DC / 4; w++) {
    const uint32_t t1 = prmt(r[4 * w + 0], r[4 * w + 1], 0x6240u);  // a0 a1 b0 b1
    const uint32_t t2 = prmt(r[4 * w + 2], r[4 * w + 3], 0x6240u);  // a2 a3 b2 b3
    aw[w] = prmt(t1, t2, 0x5410u);
    bw[w] = prmt(t1, t2, 0x7632u);
  }
  a = ByteVec<DC>::make(aw);
  b = ByteVec<DC>::make(bw);
}

// Lane-wise min of DC registers as a tree (short dependency chain).
template <int DC>
__device__ __forceinline__ uint32_t tree_min(const uint32_t* v) {
  uint32_t a[DC / 2];
#pragma unroll
  for (int i = 0; i < DC / 2; i++) a[i] = vmin2(v[2 * i], v[2 * i + 1]);
#pragma unroll
  for (int n = DC / 4; n >= 1; n >>= 1) {
#pragma unroll
    for (int i = 0; i < n; i++) a[i] = vmin2(a[2 * i], a[2 * i + 1]);
  }
  return a[0];
}

// Lane-wise min over a group of G consecutive threads (G divides 32).
// `mask` names the lanes executing the call (whole groups only).  A whole
// warp (G = 32) reduces each 16-bit lane with one warp-wide min reduction
// (redux.sync) instead of five shuffle levels.
template <int G>
__device__ __forceinline__ uint32_t group_min2(uint32_t v, unsigned mask = 0xffffffffu) {
  if constexpr (G == 32) {
    const uint32_t lo = __reduce_min_sync(mask, v & 0xffffu);
    const uint32_t hi = __reduce_min_sync(mask, v >> 16);
    return lo | (hi << 16);
  } else {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v = vmin2(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
}

// One SGM step for DC disparities of two lines (no reduction):
//   Lnew(d) = C(d) + min(Lp(d), min(Lp(d-1), Lp(d+1)) + P1, m + P2) - m
// with Lp the predecessor state, m = min_d Lp (both lanes), `left` / `right`
// the predecessor values at d0-1 / d0+DC from the neighbouring chunks.  Every
// lane stays below 2^16 and t >= m per lane, so plain 32-bit adds are exact.
template <int DC>
__device__ __forceinline__ void sgm_update(const uint32_t* Lp, const uint32_t* C, uint32_t left,
                                           uint32_t right, uint32_t m, uint32_t p1x2,
                                           uint32_t p2x2, uint32_t* Ln) {
  const uint32_t q = m + p2x2;
#pragma unroll
  for (int i = 0; i < DC; i++) {
    const uint32_t lm = (i == 0) ? left : Lp[i - 1];
    const uint32_t lp = (i == DC - 1) ? right : Lp[i + 1];
    uint32_t t = vmin2(lm, lp) + p1x2;
    t = vmin2(t, Lp[i]);
    t = vmin2(t, q);
    Ln[i] = t + C[i] - m;
  }
}

// cp.async of N = 8 or 16 bytes; pred = false writes zeros and reads nothing.
template <int N>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = pred ? N : 0;
  if (N == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(n)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(gmem_src), "n"(N),
                 "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace sf
