// Host/device interface of the fused SGM kernels (sgm_fused.cu).
#pragma once

#include <algorithm>

#include "sf_internal.cuh"

namespace sf {
namespace fused {

constexpr int kTW = 32;     // owned columns per strip
constexpr int kMaxPass = 4;

// Launch shape chosen by D: a thread owns DC disparities of two lines; the
// disparities of a line pair are spread over `chunks` consecutive threads (a
// power of two); the band sweeps carry `halo` extra columns on each side of
// a strip and walk bands of halo + 1 rows.
struct Shape {
  int dc, chunks, halo;
};
inline Shape shape_for(int D) {
  Shape s;
  s.dc = D > 128 ? 16 : 8;
  s.chunks = 1;
  while (s.chunks * s.dc < D) s.chunks <<= 1;
  s.halo = s.dc == 8 ? 16 : 8;
  return s;
}
inline int padded_d(int D) { return ((D + 15) / 16) * 16; }
inline int band_rows(int D) { return shape_for(D).halo + 1; }

struct PassIO {
  const uint8_t* cost;   // [H][W][Dp] uint8, this pass's reference image
  const uint8_t* hfwd;   // [H][W][Dp] uint8, L of path (+1,0)
  const uint8_t* hbwd;   // [H][W][Dp] uint8, L of path (-1,0)
  int16_t* dint;         // winner per pixel (UP), or nullptr
  float* dsub;           // subpixel winner (UP), or nullptr
  uint16_t* S;           // full aggregated cost [H][W][D] (UP), or nullptr
};

struct HLineArgs {
  int W, H, D, Dp, npass, P1, P2;
  uint32_t path_mask;
  int* err;              // set to 1 when a bounded copy wait gives up
  const uint8_t* cost[kMaxPass];
  uint8_t* hfwd[kMaxPass];
  uint8_t* hbwd[kMaxPass];
};

struct SweepArgs {
  int W, H, D, Dp, P1, P2, J, nb, items, subpixel;
  uint32_t path_mask;
  int en_h0, en_h1;
  uint32_t* sdown;       // tile layout [pass][H][J][16][chunks][dc] u32
  uint8_t* bs;           // band-end states [pass][2][3][W][Dp] u8
  int* flags;            // [pass][J] bands completed
  int* task_counter;     // next task of the queue (zeroed before the launch)
  int* err;              // set to 1 when a bounded wait gives up
  long long spin_limit;
  PassIO io[kMaxPass];
};

inline size_t sdown_bytes(int W, int H, int D, int npass) {
  const int J = (W + kTW - 1) / kTW;
  const Shape s = shape_for(D);
  return (size_t)npass * H * J * 16 * s.chunks * s.dc * sizeof(uint32_t);
}
inline size_t bs_bytes(int W, int D, int npass) { return (size_t)npass * 2 * 3 * W * padded_d(D); }
inline size_t cost_pair_smem(int W, int D) { return (size_t)W * 16 + (size_t)W * padded_d(D); }

cudaError_t launch_cost_pair(const uint64_t* cL, const uint64_t* cR, int W, int H, int D, int Dp,
                             int cmax, uint8_t* CL, uint8_t* CR, cudaStream_t s);
cudaError_t launch_hline(const HLineArgs& a, cudaStream_t s);
cudaError_t launch_sweep(const SweepArgs& a, bool up, cudaStream_t s);

}  // namespace fused
}  // namespace sf
