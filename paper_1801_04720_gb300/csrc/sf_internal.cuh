// Internal declarations shared by the libsf translation units (CUDA side only).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sf.h"

namespace sf {

constexpr uint32_t kFullMask = 0xffffffffu;

// Traversal directions r = (rx, ry) in path-mask bit order.
__host__ __device__ constexpr int dir_x(int r) {
  return r == 0 ? 1 : r == 1 ? -1 : r == 2 ? 0 : r == 3 ? 0 : r == 4 ? 1 : r == 5 ? -1 : r == 6 ? 1 : -1;
}
__host__ __device__ constexpr int dir_y(int r) {
  return r == 0 ? 0 : r == 1 ? 0 : r == 2 ? 1 : r == 3 ? -1 : r == 4 ? 1 : r == 5 ? -1 : r == 6 ? -1 : 1;
}

__host__ __device__ inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Census string of the pixel at (cx, cy) of a shared-memory tile with row
// stride `ts`; the tile already holds edge-clamped pixels, so every window
// neighbour is in the tile.  Window numbering: row-major, centre skipped,
// bit 0 first.
template <int RX, int RY>
__device__ __forceinline__ uint64_t census_window(const uint8_t* tile, int ts, int cx, int cy) {
  // bits 0..31 and 32.. gathered in two 32-bit words (the bit index is a
  // compile-time constant, so each bit is one compare and one merge)
  const uint8_t c = tile[cy * ts + cx];
  uint32_t lo = 0, hi = 0;
  int k = 0;
#pragma unroll
  for (int dy = -RY; dy <= RY; dy++) {
#pragma unroll
    for (int dx = -RX; dx <= RX; dx++) {
      if (dx == 0 && dy == 0) continue;
      const uint32_t b = tile[(cy + dy) * ts + cx + dx] < c ? 1u : 0u;
      if (k < 32)
        lo |= b << (k & 31);
      else
        hi |= b << (k & 31);
      k++;
    }
  }
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t census_window_rt(const uint8_t* tile, int ts, int cx, int cy,
                                                     int rx, int ry) {
  const uint8_t c = tile[cy * ts + cx];
  uint64_t bits = 0;
  int k = 0;
  for (int dy = -ry; dy <= ry; dy++) {
    for (int dx = -rx; dx <= rx; dx++) {
      if (dx == 0 && dy == 0) continue;
      bits |= (uint64_t)(tile[(cy + dy) * ts + cx + dx] < c) << k;
      k++;
    }
  }
  return bits;
}

// ---- tracing / launch accounting (api.cu) -----------------------------------
void count_launches(int n);
void trace_begin(int stage, cudaStream_t s);
void trace_end(cudaStream_t s);

// RAII bracket around the launches of one stage.
struct StageTrace {
  cudaStream_t s;
  StageTrace(int stage, cudaStream_t st) : s(st) { trace_begin(stage, st); }
  ~StageTrace() { trace_end(s); }
};

// ---- launchers (each returns cudaGetLastError() of its launches) ----------
cudaError_t launch_census(const uint8_t* img, int W, int H, int pitch, int cw, int ch, uint64_t* out,
                          cudaStream_t s);
// the census of n images of one size (one launch per eight)
cudaError_t launch_census_images(const uint8_t* const* imgs, uint64_t* const* outs, int n, int W, int H,
                                 int pitch, int cw, int ch, cudaStream_t s);
cudaError_t launch_cost_volume(const uint8_t* ref, const uint8_t* other, int W, int H, int pitch,
                               int cw, int ch, int D, int ref_is_right, uint8_t* cost,
                               cudaStream_t s);
// guide: reference image [H][gpitch] for the intensity-adaptive P2, or nullptr
cudaError_t launch_aggregate(const uint8_t* cost, int W, int H, int D, int P1, int P2,
                             uint32_t path_mask, uint16_t* S, cudaStream_t s,
                             const uint8_t* guide = nullptr, int gpitch = 0);
// unique: uniqueness ratio in percent (0 = off), applied where dsub is written
cudaError_t launch_select(const uint16_t* S, int W, int H, int D, int subpixel, int16_t* dint,
                          float* dsub, cudaStream_t s, int unique = 0);
cudaError_t launch_lr_check(const int16_t* dL, const int16_t* dR, const float* dL_sub, int W, int H,
                            int tol, uint8_t* valid, float* disp, cudaStream_t s);
// both pairs' left-right checks and the combination in one launch
struct CheckCombineArgs {
  const int16_t* dL0;
  const int16_t* dR0;
  const float* dsub0;
  const int16_t* dL1;
  const int16_t* dR1;
  const float* dsub1;
  const float2* flow;
  int W, H, tol;
  float f, B, cx, cy;
  float* D0;       // checked disparity maps (NaN where removed)
  float* D1;
  float4* s4;
  float* motion;   // optional
  float* point;    // optional
  uint8_t* valid;
};
cudaError_t launch_check_combine(const CheckCombineArgs& a, cudaStream_t s);
cudaError_t launch_combine(const float* D0, const float* D1, const float* flow, int W, int H,
                           float f, float B, float cx, float cy, float* s4, float* motion,
                           float* point, uint8_t* valid, cudaStream_t s);
// trajectories through K frames (sequence.cu)
cudaError_t launch_chain(const float* const* disps, const float* const* flows, int K, int W, int H, float f,
                         float B, float cx, float cy, float* points, uint8_t* valid, cudaStream_t s);
// densification (densify.cu); mode 0 background, 1 edge-aware (guide needed)
cudaError_t launch_fill_map(const float* in, int W, int H, const uint8_t* guide, int gpitch, int mode, float* out,
                            cudaStream_t s);
cudaError_t launch_densify(const float* s4_in, const float* flow, int W, int H, float f, float B, float cx, float cy,
                           const uint8_t* guide, int gpitch, int mode, float* s4_out, float* motion, float* point,
                           uint8_t* valid, cudaStream_t s);

}  // namespace sf
