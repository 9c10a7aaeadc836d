// Winner-take-all with parabolic subpixel refinement and the left-right
// consistency check (Sec. 3.1), and the scene-flow combination (Sec. 3.3,
// Eq. 3-5) of arXiv 1801.04720.
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

namespace {

// One warp per pixel; lanes stride over d.  The smallest d with the minimal
// aggregated cost wins (ties resolve to the smaller disparity).  With a
// uniqueness ratio u > 0 a winner whose cost S0 is not clearly below every
// disparity two or more away (100 S2 < (100 + u) S0) gets a NaN subpixel
// value, which the left-right check treats as removed.
__global__ void __launch_bounds__(256)
    select_kernel(const uint16_t* __restrict__ S, int W, int H, int D, int subpixel, int unique,
                  int16_t* __restrict__ dint, float* __restrict__ dsub) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= W * H) return;
  const uint16_t* s = S + (size_t)warp * D;
  uint32_t best = 0xffffffffu, best_d = 0xffffffffu;
  for (int d = lane; d < D; d += 32) {
    const uint32_t v = s[d];
    if (v < best) {
      best = v;
      best_d = d;
    }
  }
  const uint32_t m = __reduce_min_sync(kFullMask, best);
  const uint32_t dstar = __reduce_min_sync(kFullMask, best == m ? best_d : 0xffffffffu);
  uint32_t s2 = 0xffffffffu;
  if (unique && dsub) {
    for (int d = lane; d < D; d += 32)
      if (d + 1 < (int)dstar || d > (int)dstar + 1) s2 = min(s2, (uint32_t)s[d]);
    s2 = __reduce_min_sync(kFullMask, s2);
  }
  if (lane == 0) {
    dint[warp] = (int16_t)dstar;
    if (dsub) {
      float v = (float)dstar;
      if (subpixel && dstar > 0 && (int)dstar < D - 1) {
        const int a = (int)s[dstar - 1] - (int)m;
        const int b = (int)s[dstar + 1] - (int)m;
        // exact integers; IEEE division (no fast math) rounds once
        v = __fadd_rn((float)dstar, __fdiv_rn((float)(a - b), (float)(2 * (a + b))));
      }
      if (s2 != 0xffffffffu && 100ull * s2 < (uint64_t)(100 + unique) * m) v = __int_as_float(0x7fc00000);
      dsub[warp] = v;
    }
  }
}

__global__ void lr_check_kernel(const int16_t* __restrict__ dL, const int16_t* __restrict__ dR,
                                const float* __restrict__ dL_sub, int W, int H, int tol,
                                uint8_t* __restrict__ valid, float* __restrict__ disp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  const int y = i / W, x = i - y * W;
  const int dl = dL[i];
  const int xr = x - dl;
  bool ok = false;
  // a left winner removed before the check (NaN subpixel value) stays removed
  if (xr >= 0 && !isnan(dL_sub[i])) ok = abs(dl - (int)dR[y * W + xr]) <= tol;
  valid[i] = ok;
  disp[i] = ok ? dL_sub[i] : __int_as_float(0x7fc00000);
}

__device__ __forceinline__ bool usable(float d) { return !isnan(d) && d > 0.0f; }

// The combination at pixel (x, y) = index i: Eq. 4 / 5 with the disparity
// of t+1 read through d1_at(tx, ty) (a stored map, or the left-right check
// evaluated on the fly), back-projection and motion.
template <class Tap>
__device__ __forceinline__ void combine_pixel(int i, int x, int y, int W, int H, float d0, float2 uv, Tap d1_at,
                                              float f, float B, float cx, float cy, float4* __restrict__ s4,
                                              float* __restrict__ motion, float* __restrict__ point,
                                              uint8_t* __restrict__ valid) {
  // x' = x + F(x) as a float32 round-to-nearest sum (Eq. 4 / 5 target)
  const float xp = __fadd_rn((float)x, uv.x);
  const float yp = __fadd_rn((float)y, uv.y);
  bool ok = usable(d0) && xp >= 0.0f && xp <= (float)(W - 1) && yp >= 0.0f && yp <= (float)(H - 1);
  float d1 = 0.0f;
  if (ok) {
    const float x0 = floorf(xp), y0 = floorf(yp);
    const float fx = xp - x0, fy = yp - y0;  // exact
    const int ix = (int)x0, iy = (int)y0;
    // Eq. 5; a tap whose weight is exactly zero (fx == 0 or fy == 0) is not read
    const float v00 = d1_at(ix, iy);
    ok = usable(v00);
    d1 = __fmul_rn(__fmul_rn(1.0f - fx, 1.0f - fy), v00);
    if (fx != 0.0f) {
      const float v10 = d1_at(ix + 1, iy);
      ok = ok && usable(v10);
      d1 = __fadd_rn(d1, __fmul_rn(__fmul_rn(fx, 1.0f - fy), v10));
    }
    if (fy != 0.0f) {
      const float v01 = d1_at(ix, iy + 1);
      ok = ok && usable(v01);
      d1 = __fadd_rn(d1, __fmul_rn(__fmul_rn(1.0f - fx, fy), v01));
    }
    if (fx != 0.0f && fy != 0.0f) {
      const float v11 = d1_at(ix + 1, iy + 1);
      ok = ok && usable(v11);
      d1 = __fadd_rn(d1, __fmul_rn(__fmul_rn(fx, fy), v11));
    }
  }
  valid[i] = ok;
  const float nan = __int_as_float(0x7fc00000);
  if (!ok) {
    s4[i] = make_float4(nan, nan, nan, nan);
    if (motion) motion[3 * i] = motion[3 * i + 1] = motion[3 * i + 2] = nan;
    if (point) point[3 * i] = point[3 * i + 1] = point[3 * i + 2] = nan;
    return;
  }
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

__global__ void combine_kernel(const float* __restrict__ D0, const float* __restrict__ D1,
                               const float2* __restrict__ flow, int W, int H, float f, float B,
                               float cx, float cy, float4* __restrict__ s4,
                               float* __restrict__ motion, float* __restrict__ point,
                               uint8_t* __restrict__ valid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W * H) return;
  const int y = i / W, x = i - y * W;
  combine_pixel(i, x, y, W, H, D0[i], flow[i], [&](int tx, int ty) { return D1[(size_t)ty * W + tx]; }, f, B,
                cx, cy, s4, motion, point, valid);
}

// The left-right check of Sec. 3.1 at (x, y) of one pair: the subpixel
// disparity where the integer winners agree within tol (and the left winner
// was not removed before the check), NaN elsewhere.
__device__ __forceinline__ float lr_checked(const int16_t* __restrict__ dL, const int16_t* __restrict__ dR,
                                            const float* __restrict__ dsub, int W, int x, int y, int tol) {
  const size_t i = (size_t)y * W + x;
  const int dl = dL[i];
  const int xr = x - dl;
  const float v = dsub[i];
  if (xr < 0 || isnan(v)) return __int_as_float(0x7fc00000);
  return abs(dl - (int)dR[(size_t)y * W + xr]) <= tol ? v : __int_as_float(0x7fc00000);
}

// Both pairs' left-right checks and the combination in one pass: D0 and D1
// at the pixel are written as maps, and the Eq. 5 taps of D1 evaluate the
// check of the pair at t+1 themselves (no grid-wide wait for the D1 map).
__global__ void check_combine_kernel(const CheckCombineArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = a.W;
  if (i >= W * a.H) return;
  const int y = i / W, x = i - y * W;
  const float d0 = lr_checked(a.dL0, a.dR0, a.dsub0, W, x, y, a.tol);
  a.D0[i] = d0;
  a.D1[i] = lr_checked(a.dL1, a.dR1, a.dsub1, W, x, y, a.tol);
  combine_pixel(i, x, y, W, a.H, d0, a.flow[i],
                [&](int tx, int ty) { return lr_checked(a.dL1, a.dR1, a.dsub1, W, tx, ty, a.tol); }, a.f, a.B,
                a.cx, a.cy, a.s4, a.motion, a.point, a.valid);
}

}  // namespace

cudaError_t launch_select(const uint16_t* S, int W, int H, int D, int subpixel, int16_t* dint,
                          float* dsub, cudaStream_t s, int unique) {
  StageTrace trace(SF_STAGE_SELECT, s);
  count_launches(1);
  const long long threads = (long long)W * H * 32;
  select_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(S, W, H, D, subpixel, unique, dint, dsub);
  return cudaGetLastError();
}

cudaError_t launch_lr_check(const int16_t* dL, const int16_t* dR, const float* dL_sub, int W, int H,
                            int tol, uint8_t* valid, float* disp, cudaStream_t s) {
  StageTrace trace(SF_STAGE_LRCHECK, s);
  count_launches(1);
  const int n = W * H;
  lr_check_kernel<<<(n + 255) / 256, 256, 0, s>>>(dL, dR, dL_sub, W, H, tol, valid, disp);
  return cudaGetLastError();
}

cudaError_t launch_check_combine(const CheckCombineArgs& a, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COMBINE, s);
  count_launches(1);
  const int n = a.W * a.H;
  check_combine_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_combine(const float* D0, const float* D1, const float* flow, int W, int H,
                           float f, float B, float cx, float cy, float* s4, float* motion,
                           float* point, uint8_t* valid, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COMBINE, s);
  count_launches(1);
  const int n = W * H;
  combine_kernel<<<(n + 255) / 256, 256, 0, s>>>(D0, D1, reinterpret_cast<const float2*>(flow), W,
                                                 H, f, B, cx, cy, reinterpret_cast<float4*>(s4),
                                                 motion, point, valid);
  return cudaGetLastError();
}

}  // namespace sf
