// Parameters of the learned-confidence network: seeded initialisation on the
// device, and a small versioned file format for saving and loading them.
//
// Initialisation: every weight of layer l (ci inputs) is sqrt(2 / (9 ci))
// times a standard normal sample (He et al. 2015), every bias 0.  The
// samples come from a counter-based generator, so each parameter depends
// only on (seed, its index): splitmix64 (Steele, Lea and Flood 2014) hashes
// seed and index into two 24-bit uniforms in (0, 1], which the Box-Muller
// transform (Box and Muller 1958) turns into one normal sample.
//
// File: little-endian "SFCN", uint32 version (1), uint32 features (8),
// uint32 channels (32), uint32 count (21121), then count float32 values in
// the parameter order of sf.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "sf_confnet.cuh"

namespace {

using sf::confnet::kC;
using sf::confnet::kF;
using sf::confnet::kParamCount;

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// [offset of layer l's weights, of its biases, of the next layer) and its
// input channels, for l = 0..3
struct LayerSpan {
  int w, b, end, ci;
};
__host__ __device__ inline LayerSpan layer_span(int l) {
  const int ci[4] = {kF, kC, kC, kC}, co[4] = {kC, kC, kC, 1};
  int o = 0;
  for (int k = 0; k < l; k++) o += 9 * ci[k] * co[k] + co[k];
  return {o, o + 9 * ci[l] * co[l], o + 9 * ci[l] * co[l] + co[l], ci[l]};
}

__global__ void init_kernel(float* __restrict__ params, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParamCount) return;
  int l = 0;
  while (l < 3 && i >= layer_span(l).end) l++;
  const LayerSpan sp = layer_span(l);
  if (i >= sp.b) {
    params[i] = 0.0f;
    return;
  }
  const uint64_t h1 = splitmix64(seed ^ splitmix64(2ull * (uint64_t)i));
  const uint64_t h2 = splitmix64(seed ^ splitmix64(2ull * (uint64_t)i + 1ull));
  const float u1 = (float)((h1 >> 40) + 1ull) * (1.0f / 16777216.0f);   // (0, 1]
  const float u2 = (float)(h2 >> 40) * (1.0f / 16777216.0f);            // [0, 1)
  const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  params[i] = z * sqrtf(2.0f / (9.0f * (float)sp.ci));
}

constexpr char kMagic[4] = {'S', 'F', 'C', 'N'};
constexpr uint32_t kVersion = 1;

}  // namespace

extern "C" {

sf_status sf_confnet_init(float* params, uint64_t seed, void* stream) {
  if (!params || ((uintptr_t)params & 3u)) return SF_ERR_INVALID_ARG;
  init_kernel<<<(kParamCount + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, seed);
  if (cudaGetLastError() != cudaSuccess) return SF_ERR_CUDA;
  return SF_OK;
}

sf_status sf_confnet_save(const float* params, const char* path) {
  if (!params || !path) return SF_ERR_INVALID_ARG;
  std::vector<float> host(kParamCount);
  if (cudaMemcpy(host.data(), params, sizeof(float) * kParamCount, cudaMemcpyDeviceToHost) != cudaSuccess) {
    (void)cudaGetLastError();
    return SF_ERR_CUDA;
  }
  FILE* f = fopen(path, "wb");
  if (!f) return SF_ERR_INVALID_ARG;
  const uint32_t head[4] = {kVersion, (uint32_t)kF, (uint32_t)kC, (uint32_t)kParamCount};
  bool ok = fwrite(kMagic, 1, 4, f) == 4 && fwrite(head, sizeof(uint32_t), 4, f) == 4 &&
            fwrite(host.data(), sizeof(float), host.size(), f) == host.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? SF_OK : SF_ERR_INVALID_ARG;
}

sf_status sf_confnet_load(const char* path, float* params) {
  if (!params || !path) return SF_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return SF_ERR_INVALID_ARG;
  char magic[4];
  uint32_t head[4];
  std::vector<float> host(kParamCount);
  bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, kMagic, 4) == 0 &&
            fread(head, sizeof(uint32_t), 4, f) == 4 && head[0] == kVersion && head[1] == (uint32_t)kF &&
            head[2] == (uint32_t)kC && head[3] == (uint32_t)kParamCount &&
            fread(host.data(), sizeof(float), host.size(), f) == host.size();
  char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0;   // nothing after the parameters
  fclose(f);
  if (!ok) return SF_ERR_INVALID_ARG;
  if (cudaMemcpy(params, host.data(), sizeof(float) * kParamCount, cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

}  // extern "C"
