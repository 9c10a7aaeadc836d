// More than two frames (the paper's future work, Sec. 5: more than two frame
// pairs with an intermediate validation).
//
// chain_kernel follows every reference pixel x_0 of frame 0 through K frames:
// x_{k+1} = x_k + F_k(x_k), F_0 read at the pixel itself and F_k for k >= 1
// interpolated bilinearly at x_k (Eq. 5, taps of weight zero skipped).  The
// positions are float32 round-to-nearest operations in a fixed order (they
// decide which pixels are read and whether the chain stays in the image), so
// no multiply-add is contracted.  Frame k's disparity is the Eq. 5
// interpolation of D^k at x_k with every tap of nonzero weight usable (not
// NaN, positive); the chain is valid iff every x_k lies in the image and
// every disparity is usable, and its output is the 3D point of every frame,
// P_k = ((x_k - cx) B / d_k, (y_k - cy) B / d_k, f B / d_k).  Two frames give
// the combination of Sec. 3.3 (P_1 - P_0 its motion).
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

namespace {

struct ChainArgs {
  const float* D[SF_MAX_FRAMES];      // K maps [H][W], NaN = removed
  const float2* F[SF_MAX_FRAMES];     // K-1 flows [H][W]
  int K, W, H;
  float f, B, cx, cy;
  float* points;                      // [K][H][W][3]
  uint8_t* valid;                     // [H][W]
};

__device__ __forceinline__ bool usable(float d) { return !isnan(d) && d > 0.0f; }

// Eq. 5 weights times taps, summed in the order (0,0), (1,0), (0,1), (1,1)
__device__ __forceinline__ float2 bilerp_flow(const float2* m, int W, int ix, int iy, float fx, float fy) {
  const float2 t00 = m[(size_t)iy * W + ix];
  const float w00 = __fmul_rn(1.0f - fx, 1.0f - fy);
  float u = __fmul_rn(w00, t00.x), v = __fmul_rn(w00, t00.y);
  if (fx != 0.0f) {
    const float2 t = m[(size_t)iy * W + ix + 1];
    const float w = __fmul_rn(fx, 1.0f - fy);
    u = __fadd_rn(u, __fmul_rn(w, t.x));
    v = __fadd_rn(v, __fmul_rn(w, t.y));
  }
  if (fy != 0.0f) {
    const float2 t = m[(size_t)(iy + 1) * W + ix];
    const float w = __fmul_rn(1.0f - fx, fy);
    u = __fadd_rn(u, __fmul_rn(w, t.x));
    v = __fadd_rn(v, __fmul_rn(w, t.y));
  }
  if (fx != 0.0f && fy != 0.0f) {
    const float2 t = m[(size_t)(iy + 1) * W + ix + 1];
    const float w = __fmul_rn(fx, fy);
    u = __fadd_rn(u, __fmul_rn(w, t.x));
    v = __fadd_rn(v, __fmul_rn(w, t.y));
  }
  return make_float2(u, v);
}

__global__ void __launch_bounds__(256) chain_kernel(const __grid_constant__ ChainArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = a.W, H = a.H;
  if (i >= W * H) return;
  const size_t plane = (size_t)W * H;
  const int y = i / W, x = i - y * W;
  float px = (float)x, py = (float)y;
  bool ok = true;
  int k = 0;
  for (; k < a.K && ok; k++) {
    float d;
    if (k == 0) {
      d = a.D[0][i];
      ok = usable(d);
    } else {
      float2 uv;
      if (k == 1) {
        uv = a.F[0][i];
      } else {
        const float x0 = floorf(px), y0 = floorf(py);
        uv = bilerp_flow(a.F[k - 1], W, (int)x0, (int)y0, px - x0, py - y0);
      }
      px = __fadd_rn(px, uv.x);
      py = __fadd_rn(py, uv.y);
      if (!(px >= 0.0f && px <= (float)(W - 1) && py >= 0.0f && py <= (float)(H - 1))) {
        ok = false;
        break;
      }
      const float x0 = floorf(px), y0 = floorf(py);
      const float fx = px - x0, fy = py - y0;   // exact
      const int ix = (int)x0, iy = (int)y0;
      const float* Dk = a.D[k];
      const float v00 = Dk[(size_t)iy * W + ix];
      ok = usable(v00);
      d = __fmul_rn(__fmul_rn(1.0f - fx, 1.0f - fy), v00);
      if (fx != 0.0f) {
        const float t = Dk[(size_t)iy * W + ix + 1];
        ok = ok && usable(t);
        d = __fadd_rn(d, __fmul_rn(__fmul_rn(fx, 1.0f - fy), t));
      }
      if (fy != 0.0f) {
        const float t = Dk[(size_t)(iy + 1) * W + ix];
        ok = ok && usable(t);
        d = __fadd_rn(d, __fmul_rn(__fmul_rn(1.0f - fx, fy), t));
      }
      if (fx != 0.0f && fy != 0.0f) {
        const float t = Dk[(size_t)(iy + 1) * W + ix + 1];
        ok = ok && usable(t);
        d = __fadd_rn(d, __fmul_rn(__fmul_rn(fx, fy), t));
      }
    }
    if (ok && a.points) {
      float* P = a.points + ((size_t)k * plane + i) * 3;
      P[0] = __fdiv_rn((px - a.cx) * a.B, d);
      P[1] = __fdiv_rn((py - a.cy) * a.B, d);
      P[2] = __fdiv_rn(a.f * a.B, d);
    }
  }
  if (a.valid) a.valid[i] = ok;
  if (!ok && a.points) {
    const float nan = __int_as_float(0x7fc00000);
    for (int j = 0; j < a.K; j++) {
      float* P = a.points + ((size_t)j * plane + i) * 3;
      P[0] = P[1] = P[2] = nan;
    }
  }
}

}  // namespace

cudaError_t launch_chain(const float* const* disps, const float* const* flows, int K, int W, int H, float f,
                         float B, float cx, float cy, float* points, uint8_t* valid, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COMBINE, s);
  if (K < 2 || K > SF_MAX_FRAMES) return cudaErrorInvalidValue;
  ChainArgs a{};
  for (int k = 0; k < K; k++) a.D[k] = disps[k];
  for (int k = 0; k + 1 < K; k++) a.F[k] = reinterpret_cast<const float2*>(flows[k]);
  a.K = K;
  a.W = W;
  a.H = H;
  a.f = f;
  a.B = B;
  a.cx = cx;
  a.cy = cy;
  a.points = points;
  a.valid = valid;
  const int n = W * H;
  chain_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sf
