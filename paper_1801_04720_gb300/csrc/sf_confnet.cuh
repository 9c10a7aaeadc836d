// Host/device interface of the learned-confidence kernels (confnet.cu).
#pragma once

#include <algorithm>

#include "sf_internal.cuh"

namespace sf {
namespace confnet {

constexpr int kF = SF_CONFNET_FEATURES;   // feature channels (8)
constexpr int kC = SF_CONFNET_CHANNELS;   // hidden channels (32)
constexpr int kParamCount = 9 * kF * kC + kC + 2 * (9 * kC * kC + kC) + 9 * kC + 1;
// packed bf16 operand blocks (see pack_kernel) and fp32 biases
constexpr int kW1Elems = 5 * 2 * kC * 8;
constexpr int kW2Elems = 18 * 2 * kC * 8;
constexpr int kW4Elems = 18 * 2 * 16 * 8;
constexpr int kWElems = kW1Elems + 2 * kW2Elems + kW4Elems;
constexpr int kBiasFloats = 3 * kC + 4;
constexpr size_t kPackedBytes = (size_t)kWElems * 2 + (size_t)kBiasFloats * 4;

// Inputs of the features pass for one left-reference SGM pass.
struct FeatureArgs {
  int W, H, D, Dp, J;
  int dpad_shape;          // disparities per pixel in the S_down tiles (chunks x dc)
  int subpixel;
  const uint16_t* S;       // [H][W][D] all eight paths
  const uint32_t* sdown;   // tile layout of the down sweep (three downward paths)
  const uint8_t* hfwd;     // [H][W][Dp] path (+1,0)
  const uint8_t* hbwd;     // [H][W][Dp] path (-1,0)
  const uint8_t* cost;     // [H][W][Dp]
  uint16_t* feat;          // bf16 [H][W][8]
  int16_t* dint;           // winner
  float* dsub;             // subpixel winner
};

// One pass (stereo pair) of a network launch.
struct InferPass {
  const uint16_t* feat;    // bf16 [H][W][8]
  const int16_t* dint;     // winners (valid / disp outputs)
  const float* dsub;
  float* prob;             // [H][W] or nullptr
  uint8_t* valid;          // [H][W] or nullptr
  float* disp;             // [H][W] or nullptr (dsub where accepted, NaN elsewhere)
};
constexpr int kMaxInferPass = 4;

// One launch covers the tiles of every pass (all of one size), so the
// persistent blocks share the whole set of tiles.
struct InferArgs {
  int W, H, npass;
  const void* packed;      // kPackedBytes, 16-byte aligned
  InferPass pass[kMaxInferPass];
  float threshold;
  int* err;                // set to 1 if a bounded wait gave up (may be nullptr)
};

struct TrainArgs {
  int B, W, H;
  float* params;           // fp32 [kParamCount], updated in place when adam_m/adam_v are given
  float* adam_m;
  float* adam_v;
  const uint16_t* features;   // bf16 [B][H][W][8]
  const uint8_t* labels;      // [B][H][W]: 1 accept, 0 reject, 255 ignore; nullptr: forward only
  float lr, beta1, beta2, eps, w_neg;
  int step;
  float* grad_out;         // [kParamCount] or nullptr
  float* loss_out;         // device float or nullptr
  float* logits_out;       // [B][H][W] or nullptr
  void* workspace;
};

cudaError_t launch_features(const FeatureArgs& a, cudaStream_t s);
cudaError_t launch_pack(const float* params, void* packed, cudaStream_t s);
cudaError_t launch_infer(const InferArgs& a, cudaStream_t s);
size_t train_workspace_bytes(int B, int W, int H);
cudaError_t launch_train_step(const TrainArgs& t, cudaStream_t s);
cudaError_t launch_adam(float* params, float* m, float* v, const float* grad, int n, float lr, float beta1,
                        float beta2, float eps, int step, cudaStream_t s);

}  // namespace confnet
}  // namespace sf
