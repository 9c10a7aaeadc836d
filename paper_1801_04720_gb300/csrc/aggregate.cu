// Semi-global aggregation of a stored cost volume (Sec. 3.1, "eight different
// paths").  One warp walks one path line; lane l owns the K consecutive
// disparities [l*K, l*K + K).  The min over d of the previous step comes from
// a warp-wide redux; the d-1 / d+1 neighbours at lane boundaries from
// shuffles.  Directions run one after another, each adding its L_r into S.
// With a guide image the P2 of each step adapts to the intensity step, as in
// the SGM the paper cites: P2 / |I(p) - I(p-r)| rounded down, at least P1,
// P2 itself where the intensities are equal.
#include "sf_internal.cuh"

namespace sf {

namespace {

constexpr uint32_t kInf = 0x3fffffffu;

template <int K>
__global__ void __launch_bounds__(256)
    aggregate_direction_kernel(const uint8_t* __restrict__ cost, const uint8_t* __restrict__ guide,
                               int gpitch, int W, int H, int D, int P1, int P2, int rx, int ry,
                               uint16_t* __restrict__ S, int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nlines = (rx == 0) ? W : (ry == 0) ? H : W + H - 1;
  if (warp >= nlines) return;
  int x, y;
  if (rx == 0) {
    x = warp;
    y = ry > 0 ? 0 : H - 1;
  } else if (ry == 0) {
    y = warp;
    x = rx > 0 ? 0 : W - 1;
  } else {
    const int ystart = ry > 0 ? 0 : H - 1;
    if (warp < W) {
      x = warp;
      y = ystart;
    } else {
      x = rx > 0 ? 0 : W - 1;
      y = ystart + ry * (warp - W + 1);
    }
  }
  const int d0 = lane * K;
  uint32_t L[K];
  uint32_t prev_min = 0;
  bool first = true;
  while (x >= 0 && x < W && y >= 0 && y < H) {
    const size_t base = ((size_t)y * W + x) * D;
    uint32_t c[K];
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = (d0 + k < D) ? (uint32_t)cost[base + d0 + k] : kInf;
    if (first) {
#pragma unroll
      for (int k = 0; k < K; k++) L[k] = c[k];
      first = false;
    } else {
      uint32_t left = __shfl_up_sync(kFullMask, L[K - 1], 1);
      uint32_t right = __shfl_down_sync(kFullMask, L[0], 1);
      if (lane == 0) left = kInf;
      if (lane == 31) right = kInf;
      int p2 = P2;
      if (guide) {
        const int step = abs((int)guide[(size_t)y * gpitch + x] - (int)guide[(size_t)(y - ry) * gpitch + (x - rx)]);
        if (step > 0) p2 = max(P1, P2 / step);
      }
      const uint32_t q = prev_min + (uint32_t)p2;
      uint32_t nl[K];
#pragma unroll
      for (int k = 0; k < K; k++) {
        const uint32_t lm = (k == 0) ? left : L[k - 1];
        const uint32_t lp = (k == K - 1) ? right : L[k + 1];
        uint32_t t = min(L[k], min(lm, lp) + (uint32_t)P1);
        t = min(t, q);
        nl[k] = (d0 + k < D) ? c[k] + t - prev_min : kInf;
      }
#pragma unroll
      for (int k = 0; k < K; k++) L[k] = nl[k];
    }
    uint32_t m = L[0];
#pragma unroll
    for (int k = 1; k < K; k++) m = min(m, L[k]);
    prev_min = __reduce_min_sync(kFullMask, m);
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (d0 + k < D) {
        uint16_t* s = S + base + d0 + k;
        *s = (uint16_t)(accumulate ? (uint32_t)*s + L[k] : L[k]);
      }
    }
    x += rx;
    y += ry;
  }
}

}  // namespace

cudaError_t launch_aggregate(const uint8_t* cost, int W, int H, int D, int P1, int P2,
                             uint32_t path_mask, uint16_t* S, cudaStream_t s, const uint8_t* guide,
                             int gpitch) {
  StageTrace trace(SF_STAGE_AGGREGATE, s);
  if ((path_mask & 0xffu) == 0) return cudaMemsetAsync(S, 0, sizeof(uint16_t) * W * H * D, s);
  int accumulate = 0;
  for (int r = 0; r < SF_NUM_PATHS; r++) {
    if (!((path_mask >> r) & 1u)) continue;
    const int rx = dir_x(r), ry = dir_y(r);
    const int nlines = (rx == 0) ? W : (ry == 0) ? H : W + H - 1;
    const int threads = 256, warps_per_block = threads / 32;
    const int blocks = (nlines + warps_per_block - 1) / warps_per_block;
    if (D <= 32)
      aggregate_direction_kernel<1><<<blocks, threads, 0, s>>>(cost, guide, gpitch, W, H, D, P1, P2, rx, ry, S,
                                                                accumulate);
    else if (D <= 64)
      aggregate_direction_kernel<2><<<blocks, threads, 0, s>>>(cost, guide, gpitch, W, H, D, P1, P2, rx, ry, S,
                                                                accumulate);
    else if (D <= 128)
      aggregate_direction_kernel<4><<<blocks, threads, 0, s>>>(cost, guide, gpitch, W, H, D, P1, P2, rx, ry, S,
                                                                accumulate);
    else
      aggregate_direction_kernel<8><<<blocks, threads, 0, s>>>(cost, guide, gpitch, W, H, D, P1, P2, rx, ry, S,
                                                                accumulate);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    accumulate = 1;
  }
  return cudaSuccess;
}

}  // namespace sf
