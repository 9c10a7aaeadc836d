// Densification of the sparse scene flow: the paper's future work (Sec. 5);
// its Table 1 also reports the dense result the benchmark makes from a sparse
// submission by filling the gaps (Sec. 4.1).
//
// A sparse map (NaN = missing) is filled along each row, then, for the rows
// with nothing kept, along each column of the row-filled map.  Within a line
// a missing pixel between kept values a (before) and b (after) takes
//   mode 0 (background): min(a, b), the farther surface for a disparity;
//   mode 1 (edge-aware): the value whose guide intensity is closer to the
//                        pixel's own, min(a, b) on a tie;
// with one kept side it takes that value; a line with nothing kept stays
// missing.
//
// Kernels (no scratch: the output buffer carries the intermediate state):
//   fill_rows_kernel: one warp per row.  A forward pass over 32-pixel chunks
//     finds, with a ballot and a carry from the previous chunks, the nearest
//     kept pixel at or before each pixel and parks its index in the output
//     (as the bits of the float); a backward pass finds the nearest kept
//     pixel after it the same way and writes the filled value.  Groups of
//     chunks issue their loads together.
//   fill_cols_kernel: the rows the row pass left missing (the same in every
//     column) are marked once per block; one thread per column fills them
//     from the nearest filled rows above and below.
//   backproject_kernel: (u, v) from the flow, the filled d0 and d1, and the
//     back-projection of Sec. 3.3 at every pixel.
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

namespace {

struct FillArgs {
  const float* in[2];     // map m: element (y, x) at in[m][(y * W + x) * istride]
  float* out[2];          // likewise with ostride
  int istride, ostride, nmaps, W, H, mode;
  const uint8_t* guide;   // [H][gpitch], mode 1
  int gpitch;
};

__device__ __forceinline__ float fnan() { return __int_as_float(0x7fc00000); }

// the fill value between kept values va (at guide index ia) and vb (ib) for
// the pixel at guide index ip
__device__ __forceinline__ float choose(const FillArgs& a, float va, float vb, size_t ip, size_t ia, size_t ib) {
  if (a.mode == 1) {
    const int g = a.guide[ip];
    const int da = abs(g - (int)a.guide[ia]), db = abs(g - (int)a.guide[ib]);
    if (da < db) return va;
    if (db < da) return vb;
  }
  return fminf(va, vb);
}

// Chunks of 32 pixels handled per group: their loads are issued together
// (the carries between chunks are register work), so a row costs a few
// memory round trips instead of one per chunk.
constexpr int kFillGroup = 8;

__global__ void __launch_bounds__(256) fill_rows_kernel(const FillArgs a) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= a.nmaps * a.H) return;
  const int m = warp / a.H, y = warp - m * a.H;
  const float* in = a.in[m];
  float* out = a.out[m];
  const int W = a.W;
  const size_t row = (size_t)y * W;
  auto at_in = [&](int x) { return in[(row + x) * a.istride]; };
  const unsigned below = (2u << lane) - 1u;   // lanes 0 .. lane
  const unsigned above = ~((1u << lane) - 1u); // lanes lane .. 31
  const int nch = (W + 31) / 32;
  // forward: index of the nearest kept pixel at or before x (-1: none),
  // parked in the output as the bits of the float
  int carry = -1;
  for (int c0 = 0; c0 < nch; c0 += kFillGroup) {
    float v[kFillGroup];
#pragma unroll
    for (int u = 0; u < kFillGroup; u++) {
      const int x = (c0 + u) * 32 + lane;
      v[u] = (c0 + u < nch && x < W) ? at_in(x) : fnan();
    }
#pragma unroll
    for (int u = 0; u < kFillGroup; u++) {
      const int c = (c0 + u) * 32, x = c + lane;
      const bool ok = x < W && !isnan(v[u]);
      const unsigned b = __ballot_sync(0xffffffffu, ok);
      const unsigned mb = b & below;
      const int left = mb ? c + 31 - __clz(mb) : carry;
      if (c0 + u < nch && x < W) out[(row + x) * a.ostride] = ok ? v[u] : __int_as_float(left);
      if (b) carry = c + 31 - __clz(b);
    }
  }
  __syncwarp();
  // backward: the nearest kept pixel at or after x, and the filled value
  carry = -1;
  for (int c0 = nch - 1; c0 >= 0; c0 -= kFillGroup) {
    float v[kFillGroup];
    int left[kFillGroup], right[kFillGroup];
#pragma unroll
    for (int u = 0; u < kFillGroup; u++) {
      const int x = (c0 - u) * 32 + lane;
      const bool in_row = c0 - u >= 0 && x < W;
      v[u] = in_row ? at_in(x) : fnan();
      left[u] = in_row ? __float_as_int(out[(row + x) * a.ostride]) : -1;   // the parked index where v is NaN
    }
#pragma unroll
    for (int u = 0; u < kFillGroup; u++) {
      const int c = (c0 - u) * 32, x = c + lane;
      const bool ok = c0 - u >= 0 && x < W && !isnan(v[u]);
      const unsigned b = __ballot_sync(0xffffffffu, ok);
      const unsigned mb = b & above;
      right[u] = mb ? c + __ffs(mb) - 1 : carry;
      if (b) carry = c + __ffs(b) - 1;
    }
    // the gaps' values: the gathers of every chunk of the group together
#pragma unroll
    for (int u = 0; u < kFillGroup; u++) {
      const int x = (c0 - u) * 32 + lane;
      if (c0 - u < 0 || x >= W || !isnan(v[u])) continue;
      const int l = left[u], r = right[u];
      float res;
      if (l >= 0 && r >= 0)
        res = choose(a, at_in(l), at_in(r), (size_t)y * a.gpitch + x, (size_t)y * a.gpitch + l,
                     (size_t)y * a.gpitch + r);
      else if (l >= 0)
        res = at_in(l);
      else if (r >= 0)
        res = at_in(r);
      else
        res = fnan();
      out[(row + x) * a.ostride] = res;
    }
  }
}

// The row pass leaves a row either filled at every x or missing at every x
// (nothing kept in it), so the rows the column pass must fill are the same in
// every column.  A block marks them once (a bit per row in shared memory,
// read from its own first column, which no other block writes and this one
// writes only after the marks are made), then each thread fills its own
// column at those rows only: the nearest rows above and below that the row
// pass filled.
constexpr int kMaxRowWords = (32767 + 31) / 32;

__global__ void __launch_bounds__(256) fill_cols_kernel(const FillArgs a) {
  __shared__ uint32_t empty[kMaxRowWords];
  const int W = a.W, H = a.H;
  const int cols_per_map = (W + blockDim.x - 1) / blockDim.x;
  const int m = blockIdx.x / cols_per_map;
  const int x0 = (blockIdx.x - m * cols_per_map) * blockDim.x;
  const int x = x0 + threadIdx.x;
  float* out = a.out[m];
  const int words = (H + 31) / 32;
  // one row per thread, a ballot per warp: bit y of the marks is row y
  for (int y0 = 0; y0 < 32 * words; y0 += blockDim.x) {
    const int y = y0 + (int)threadIdx.x;
    const bool e = y < H && isnan(out[((size_t)y * W + x0) * a.ostride]);
    const uint32_t bits = __ballot_sync(0xffffffffu, e);
    if ((threadIdx.x & 31) == 0 && y < 32 * words) empty[y >> 5] = bits;
  }
  __syncthreads();
  if (x >= W) return;
  auto at = [&](int y) -> float& { return out[((size_t)y * W + x) * a.ostride]; };
  auto is_empty = [&](int y) { return (empty[y >> 5] >> (y & 31)) & 1u; };
  int ya = -1, yb = -1;   // nearest filled rows above and below the current run of empty rows
  for (int w = 0; w < words; w++) {
    uint32_t bits = empty[w];
    while (bits) {
      const int y = 32 * w + __ffs(bits) - 1;
      bits &= bits - 1;
      if (yb <= y) {        // the first empty row of a run: find its neighbours
        ya = y - 1;
        while (ya >= 0 && is_empty(ya)) ya--;
        yb = y + 1;
        while (yb < H && is_empty(yb)) yb++;
      }
      float r;
      if (ya >= 0 && yb < H)
        r = choose(a, at(ya), at(yb), (size_t)y * a.gpitch + x, (size_t)ya * a.gpitch + x, (size_t)yb * a.gpitch + x);
      else if (ya >= 0)
        r = at(ya);
      else if (yb < H)
        r = at(yb);
      else
        r = fnan();
      at(y) = r;
    }
  }
}

// Dense scene flow: filled d0, d1 already in s4 channels 2 and 3.
__global__ void __launch_bounds__(256)
    backproject_kernel(const float2* __restrict__ flow, int W, int H, float f, float B, float cx, float cy,
                       float4* __restrict__ s4, float* __restrict__ motion, float* __restrict__ point,
                       uint8_t* __restrict__ valid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  const int y = i / W, x = i - y * W;
  const float2 uv = flow[i];
  const float4 cur = s4[i];
  const float d0 = cur.z, d1 = cur.w;
  const bool ok = !isnan(d0) && !isnan(d1) && d0 > 0.0f && d1 > 0.0f;
  valid[i] = ok;
  const float nan = fnan();
  if (!ok) {
    s4[i] = make_float4(nan, nan, nan, nan);
    if (motion) motion[3 * i] = motion[3 * i + 1] = motion[3 * i + 2] = nan;
    if (point) point[3 * i] = point[3 * i + 1] = point[3 * i + 2] = nan;
    return;
  }
  const float xp = __fadd_rn((float)x, uv.x);
  const float yp = __fadd_rn((float)y, uv.y);
  s4[i] = make_float4(uv.x, uv.y, d0, d1);
  const float z0 = __fdiv_rn(f * B, d0), z1 = __fdiv_rn(f * B, d1);
  const float p0x = __fdiv_rn(((float)x - cx) * B, d0), p0y = __fdiv_rn(((float)y - cy) * B, d0);
  const float p1x = __fdiv_rn((xp - cx) * B, d1), p1y = __fdiv_rn((yp - cy) * B, d1);
  if (motion) {
    motion[3 * i] = p1x - p0x;
    motion[3 * i + 1] = p1y - p0y;
    motion[3 * i + 2] = z1 - z0;
  }
  if (point) {
    point[3 * i] = p0x;
    point[3 * i + 1] = p0y;
    point[3 * i + 2] = z0;
  }
}

cudaError_t launch_fill(const FillArgs& a, cudaStream_t s) {
  const long long rows = (long long)a.nmaps * a.H;
  fill_rows_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(a);
  const long long blocks = (long long)a.nmaps * ((a.W + 255) / 256);
  fill_cols_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fill_map(const float* in, int W, int H, const uint8_t* guide, int gpitch, int mode, float* out,
                            cudaStream_t s) {
  StageTrace trace(SF_STAGE_DENSIFY, s);
  FillArgs a{};
  a.in[0] = in;
  a.out[0] = out;
  a.istride = a.ostride = 1;
  a.nmaps = 1;
  a.W = W;
  a.H = H;
  a.mode = mode;
  a.guide = guide;
  a.gpitch = gpitch;
  return launch_fill(a, s);
}

cudaError_t launch_densify(const float* s4_in, const float* flow, int W, int H, float f, float B, float cx, float cy,
                           const uint8_t* guide, int gpitch, int mode, float* s4_out, float* motion, float* point,
                           uint8_t* valid, cudaStream_t s) {
  StageTrace trace(SF_STAGE_DENSIFY, s);
  FillArgs a{};
  a.in[0] = s4_in + 2;     // d0
  a.in[1] = s4_in + 3;     // d1 (the warped disparity of t+1, at the reference pixel)
  a.out[0] = s4_out + 2;
  a.out[1] = s4_out + 3;
  a.istride = a.ostride = 4;
  a.nmaps = 2;
  a.W = W;
  a.H = H;
  a.mode = mode;
  a.guide = guide;
  a.gpitch = gpitch;
  cudaError_t e = launch_fill(a, s);
  if (e != cudaSuccess) return e;
  const int n = W * H;
  backproject_kernel<<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float2*>(flow), W, H, f, B, cx, cy,
                                                     reinterpret_cast<float4*>(s4_out), motion, point, valid);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sf
