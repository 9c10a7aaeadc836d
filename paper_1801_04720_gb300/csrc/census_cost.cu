// Census transform and Hamming matching-cost volume (SGM matching cost,
// Sec. 3.1 of arXiv 1801.04720).
#include <algorithm>

#include "sf_internal.cuh"

namespace sf {

namespace {

constexpr int kCensusTX = 32, kCensusTY = 8;

// Images of one size whose census one launch computes (blockIdx.z).
constexpr int kCensusMaxImages = 8;
struct CensusJob {
  const uint8_t* img[kCensusMaxImages];
  uint64_t* out[kCensusMaxImages];
};

// One thread per pixel; the block stages its (TY + 2ry) x (TX + 2rx) window
// of edge-clamped pixels in shared memory.
template <int RX, int RY>
__global__ void __launch_bounds__(kCensusTX* kCensusTY)
    census_kernel(const __grid_constant__ CensusJob job, int W, int H, int pitch, int rx, int ry) {
  extern __shared__ uint8_t tile[];
  const uint8_t* __restrict__ img = job.img[blockIdx.z];
  uint64_t* __restrict__ out = job.out[blockIdx.z];
  const int RXv = RX > 0 ? RX : rx, RYv = RY > 0 ? RY : ry;
  const int tw = kCensusTX + 2 * RXv, th = kCensusTY + 2 * RYv;
  const int x0 = blockIdx.x * kCensusTX - RXv, y0 = blockIdx.y * kCensusTY - RYv;
  for (int i = threadIdx.y * kCensusTX + threadIdx.x; i < tw * th; i += kCensusTX * kCensusTY) {
    const int ty = i / tw, tx = i - ty * tw;
    const int gx = clampi(x0 + tx, 0, W - 1), gy = clampi(y0 + ty, 0, H - 1);
    tile[i] = img[(size_t)gy * pitch + gx];
  }
  __syncthreads();
  const int x = blockIdx.x * kCensusTX + threadIdx.x, y = blockIdx.y * kCensusTY + threadIdx.y;
  if (x >= W || y >= H) return;
  uint64_t bits;
  if (RX > 0)
    bits = census_window<RX, RY>(tile, tw, threadIdx.x + RX, threadIdx.y + RY);
  else
    bits = census_window_rt(tile, tw, threadIdx.x + rx, threadIdx.y + ry, rx, ry);
  out[(size_t)y * W + x] = bits;
}

// The 9 x 7 window (the method's), four horizontally adjacent pixels a
// thread: for one offset the four pixels' neighbours are four consecutive
// bytes of the tile row, one byte permute of two aligned tile words; they
// are compared with the four centres at once (unsigned byte compare by
// SWAR: the low seven bits through an add that cannot carry between bytes,
// the top bit by a logic function), and each verdict, the top bit of its
// byte, moves to bit k % 8 of that byte in group word k / 8.  Byte j of the
// eight group words is then pixel j's 62-bit string, bit k for the k-th
// offset in the same row-major order as census_window.
constexpr int kC97TX = 128, kC97TY = 8;   // a warp per row: 32 threads x 4 columns
constexpr int kC97TW = kC97TX + 8;        // tile row: 4 clamped columns on each side
constexpr int kC97TH = kC97TY + 6;
constexpr int kC97Words = kC97TW / 4;

__device__ __forceinline__ uint32_t bytes_at(uint32_t lo, uint32_t hi, int s) {
  // bytes s .. s + 3 of the 8-byte sequence lo:hi (s in 0..4)
  return s == 0 ? lo : s == 4 ? hi : __byte_perm(lo, hi, (uint32_t)(s | (s + 1) << 4 | (s + 2) << 8 | (s + 3) << 12));
}

__global__ void __launch_bounds__(256)
    census97_kernel(const __grid_constant__ CensusJob job, int W, int H, int pitch) {
  __shared__ __align__(16) uint8_t tile[kC97TH * kC97TW];
  const uint8_t* __restrict__ img = job.img[blockIdx.z];
  uint64_t* __restrict__ out = job.out[blockIdx.z];
  const int bx = blockIdx.x * kC97TX, by = blockIdx.y * kC97TY;
  const int tid = threadIdx.x;
  for (int i = tid; i < kC97TH * kC97TW; i += 256) {
    const int ty = i / kC97TW, tx = i - ty * kC97TW;
    const int gx = clampi(bx - 4 + tx, 0, W - 1), gy = clampi(by - 3 + ty, 0, H - 1);
    tile[i] = img[(size_t)gy * pitch + gx];
  }
  __syncthreads();
  const int lane = tid & 31, row = tid >> 5;
  const int y = by + row, x0 = bx + 4 * lane;
  if (y >= H || x0 >= W) return;
  // pixel x0 sits at tile column 4 + 4 lane: word lane + 1 of its tile row
  const uint32_t* tw = reinterpret_cast<const uint32_t*>(tile) + lane + 1;
  const uint32_t c = tw[(row + 3) * kC97Words];
  const uint32_t K = 0x80808080u - (c & 0x7f7f7f7fu);
  uint32_t g[8];
#pragma unroll
  for (int i = 0; i < 8; i++) g[i] = 0u;
  int k = 0;
#pragma unroll
  for (int dy = -3; dy <= 3; dy++) {
    const uint32_t* rw = tw + (row + 3 + dy) * kC97Words;
    const uint32_t A = rw[-1], B = rw[0], C = rw[1];
#pragma unroll
    for (int dx = -4; dx <= 4; dx++) {
      if (dx == 0 && dy == 0) continue;
      const uint32_t n = dx < 0 ? bytes_at(A, B, 4 + dx) : bytes_at(B, C, dx);
      const uint32_t t = (n & 0x7f7f7f7fu) + K;        // top bit: low seven bits of n >= those of c
      const uint32_t lt = (~n & c) | (~(n ^ c) & ~t);  // top bit: n < c
      g[k >> 3] |= (lt >> (7 - (k & 7))) & (0x01010101u << (k & 7));
      k++;
    }
  }
  uint64_t* o = out + (size_t)y * W + x0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    if (x0 + j >= W) break;
    const uint32_t sel = (uint32_t)(j | (j + 4) << 4);
    const uint32_t lo = __byte_perm(__byte_perm(g[0], g[1], sel), __byte_perm(g[2], g[3], sel), 0x5410);
    const uint32_t hi = __byte_perm(__byte_perm(g[4], g[5], sel), __byte_perm(g[6], g[7], sel), 0x5410);
    o[j] = ((uint64_t)hi << 32) | lo;
  }
}

// Cost volume of one image row segment [xs, xs + kCostTX): the block computes
// the census strings it needs from the raw images, then writes
// cost[y][x][d] with consecutive threads on consecutive d (coalesced).
constexpr int kCostTX = 32, kCostThreads = 256;

__global__ void __launch_bounds__(kCostThreads)
    cost_kernel(const uint8_t* __restrict__ ref, const uint8_t* __restrict__ other, int W, int H,
                int pitch, int rx, int ry, int D, int ref_is_right, int cmax,
                uint8_t* __restrict__ cost) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int y = blockIdx.y;
  const int xs = blockIdx.x * kCostTX;
  const int nref = min(kCostTX, W - xs);
  // candidate range in the other image
  const int o_lo = ref_is_right ? xs : max(0, xs - (D - 1));
  const int o_hi = ref_is_right ? min(W, xs + nref + D - 1) : xs + nref;  // exclusive
  const int nother = o_hi - o_lo;
  uint64_t* c_ref = reinterpret_cast<uint64_t*>(smem);
  uint64_t* c_oth = c_ref + kCostTX;
  uint8_t* tile = reinterpret_cast<uint8_t*>(c_oth + (kCostTX + SF_MAX_DISPARITY));
  const int th = 2 * ry + 1;
  // ref tile
  {
    const int tw = nref + 2 * rx;
    for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
      const int ty = i / tw, tx = i - ty * tw;
      tile[i] = ref[(size_t)clampi(y - ry + ty, 0, H - 1) * pitch + clampi(xs - rx + tx, 0, W - 1)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nref; i += blockDim.x)
      c_ref[i] = census_window_rt(tile, tw, i + rx, ry, rx, ry);
    __syncthreads();
  }
  // other tile
  {
    const int tw = nother + 2 * rx;
    for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
      const int ty = i / tw, tx = i - ty * tw;
      tile[i] =
          other[(size_t)clampi(y - ry + ty, 0, H - 1) * pitch + clampi(o_lo - rx + tx, 0, W - 1)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nother; i += blockDim.x)
      c_oth[i] = census_window_rt(tile, tw, i + rx, ry, rx, ry);
    __syncthreads();
  }
  const int total = nref * D;
  uint8_t* row = cost + ((size_t)y * W + xs) * D;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int px = i / D, d = i - px * D;
    const int x = xs + px;
    const int xo = ref_is_right ? x + d : x - d;
    int c = cmax;
    if (xo >= 0 && xo < W) c = __popcll(c_ref[px] ^ c_oth[xo - o_lo]);
    row[i] = (uint8_t)c;
  }
}

}  // namespace

cudaError_t launch_census_images(const uint8_t* const* imgs, uint64_t* const* outs, int n, int W, int H,
                                 int pitch, int cw, int ch, cudaStream_t s) {
  StageTrace trace(SF_STAGE_CENSUS, s);
  const int rx = cw / 2, ry = ch / 2;
  dim3 block(kCensusTX, kCensusTY);
  const size_t smem = (size_t)(kCensusTX + 2 * rx) * (kCensusTY + 2 * ry);
  for (int i0 = 0; i0 < n; i0 += kCensusMaxImages) {
    const int m = std::min(kCensusMaxImages, n - i0);
    CensusJob job{};
    for (int i = 0; i < m; i++) {
      job.img[i] = imgs[i0 + i];
      job.out[i] = outs[i0 + i];
    }
    count_launches(1);
    if (cw == 9 && ch == 7) {
      dim3 grid97((W + kC97TX - 1) / kC97TX, (H + kC97TY - 1) / kC97TY, m);
      census97_kernel<<<grid97, 256, 0, s>>>(job, W, H, pitch);
    } else {
      dim3 grid((W + kCensusTX - 1) / kCensusTX, (H + kCensusTY - 1) / kCensusTY, m);
      census_kernel<0, 0><<<grid, block, smem, s>>>(job, W, H, pitch, rx, ry);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_census(const uint8_t* img, int W, int H, int pitch, int cw, int ch, uint64_t* out,
                          cudaStream_t s) {
  return launch_census_images(&img, &out, 1, W, H, pitch, cw, ch, s);
}

cudaError_t launch_cost_volume(const uint8_t* ref, const uint8_t* other, int W, int H, int pitch,
                               int cw, int ch, int D, int ref_is_right, uint8_t* cost,
                               cudaStream_t s) {
  StageTrace trace(SF_STAGE_COST, s);
  count_launches(1);
  const int rx = cw / 2, ry = ch / 2;
  dim3 grid((W + kCostTX - 1) / kCostTX, H);
  const size_t smem = sizeof(uint64_t) * (2 * kCostTX + SF_MAX_DISPARITY) +
                      (size_t)(kCostTX + SF_MAX_DISPARITY + 2 * rx) * (2 * ry + 1);
  cost_kernel<<<grid, kCostThreads, smem, s>>>(ref, other, W, H, pitch, rx, ry, D, ref_is_right,
                                               cw * ch - 1, cost);
  return cudaGetLastError();
}

}  // namespace sf
