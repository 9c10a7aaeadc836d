// Frame pipeline: scene flow from host buffers with the copies overlapped.
//
// sf_scene_flow_host copies one frame in, computes it and copies it out
// before returning, so the copy engines and the SMs take turns.  A pipeline
// keeps `depth` staging slots in device memory and three streams:
//
//   copy-in : H2D of frame k into slot k % depth
//   compute : sf_scene_flow of frame k (one frame at a time, one workspace)
//   copy-out: D2H of frame k's outputs
//
// ordered by three events per slot: `in_done` (inputs landed) gates the
// compute; `computed` gates the copy-out and the next copy-in into the slot
// (the compute has finished reading its inputs); `out_done` gates the next
// compute into the slot (the copy-out has finished reading its outputs).
// Frame k+1's inputs and frame k-1's outputs therefore move while frame k
// computes.  The computation is exactly sf_scene_flow's.
#include <mutex>
#include <new>
#include <vector>

#include "sf_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Slot {
  size_t img[4] = {0, 0, 0, 0}, flow = 0, s4 = 0, motion = 0, point = 0, valid = 0;
  cudaEvent_t in_done = nullptr, computed = nullptr, out_done = nullptr;
  int64_t ticket = -1;
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) (void)cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) (void)cudaSetDevice(prev);
  }
};

}  // namespace

struct sf_pipeline {
  int W = 0, H = 0, depth = 0, device = 0;
  sf_sgm_params p{};
  sf_camera cam{};
  uint8_t* mem = nullptr;      // one device allocation: workspace, then the slots
  size_t ws_bytes = 0;
  std::vector<Slot> slots;
  cudaStream_t in = nullptr, compute = nullptr, out = nullptr;
  int64_t next = 0;
  std::mutex mu;
};

namespace {

void release(sf_pipeline* pl) {
  if (!pl) return;
  for (Slot& s : pl->slots) {
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.computed) cudaEventDestroy(s.computed);
    if (s.out_done) cudaEventDestroy(s.out_done);
  }
  if (pl->in) cudaStreamDestroy(pl->in);
  if (pl->compute) cudaStreamDestroy(pl->compute);
  if (pl->out) cudaStreamDestroy(pl->out);
  if (pl->mem) cudaFree(pl->mem);
  delete pl;
}

sf_status fail(sf_pipeline* pl) {
  (void)cudaGetLastError();
  release(pl);
  return SF_ERR_CUDA;
}

}  // namespace

extern "C" {

sf_status sf_pipeline_create(int32_t W, int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                             int32_t depth, sf_pipeline** out) {
  if (!out) return SF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || !cam || depth < 2 || depth > 8 || W <= 0 || H <= 0) return SF_ERR_INVALID_ARG;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  const size_t ws = sf_workspace_size(W, H, p);
  if (ws == 0) return SF_ERR_INVALID_ARG;
  sf_pipeline* pl = new (std::nothrow) sf_pipeline();
  if (!pl) return SF_ERR_CUDA;
  pl->W = W;
  pl->H = H;
  pl->depth = depth;
  pl->p = *p;
  pl->cam = *cam;
  if (cudaGetDevice(&pl->device) != cudaSuccess) return fail(pl);
  const size_t N = (size_t)W * H;
  size_t o = up(ws);
  pl->ws_bytes = ws;
  pl->slots.resize(depth);
  for (Slot& s : pl->slots) {
    for (int k = 0; k < 4; k++) { s.img[k] = o; o = up(o + N); }
    s.flow = o; o = up(o + N * 2 * sizeof(float));
    s.s4 = o; o = up(o + N * 4 * sizeof(float));
    s.motion = o; o = up(o + N * 3 * sizeof(float));
    s.point = o; o = up(o + N * 3 * sizeof(float));
    s.valid = o; o = up(o + N);
  }
  if (cudaMalloc(&pl->mem, o) != cudaSuccess) return fail(pl);
  for (Slot& s : pl->slots) {
    if (cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) != cudaSuccess)
      return fail(pl);
  }
  if (cudaStreamCreateWithFlags(&pl->in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&pl->compute, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&pl->out, cudaStreamNonBlocking) != cudaSuccess)
    return fail(pl);
  *out = pl;
  return SF_OK;
}

sf_status sf_pipeline_submit(sf_pipeline* pl, const uint8_t* left_t, const uint8_t* right_t,
                             const uint8_t* left_t1, const uint8_t* right_t1, const float* flow,
                             float* s4_out, float* motion_out, float* point_out, uint8_t* valid_out,
                             int64_t* ticket) {
  if (!pl || !left_t || !right_t || !left_t1 || !right_t1 || !flow || !s4_out || !valid_out)
    return SF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(pl->mu);
  DeviceGuard guard(pl->device);
  const size_t N = (size_t)pl->W * pl->H;
  const int64_t k = pl->next;
  Slot& s = pl->slots[(size_t)(k % pl->depth)];
  uint8_t* m = pl->mem;
#define SF_PL_TRY(expr)          \
  do {                           \
    if ((expr) != cudaSuccess) { \
      (void)cudaGetLastError();  \
      return SF_ERR_CUDA;        \
    }                            \
  } while (0)
  // copy-in: after the slot's previous frame has finished reading its inputs
  SF_PL_TRY(cudaStreamWaitEvent(pl->in, s.computed, 0));
  const uint8_t* imgs[4] = {left_t, right_t, left_t1, right_t1};
  for (int i = 0; i < 4; i++)
    SF_PL_TRY(cudaMemcpyAsync(m + s.img[i], imgs[i], N, cudaMemcpyHostToDevice, pl->in));
  SF_PL_TRY(cudaMemcpyAsync(m + s.flow, flow, N * 2 * sizeof(float), cudaMemcpyHostToDevice, pl->in));
  SF_PL_TRY(cudaEventRecord(s.in_done, pl->in));
  // compute: after the inputs landed and the slot's previous outputs left
  SF_PL_TRY(cudaStreamWaitEvent(pl->compute, s.in_done, 0));
  SF_PL_TRY(cudaStreamWaitEvent(pl->compute, s.out_done, 0));
  float* d_motion = motion_out ? reinterpret_cast<float*>(m + s.motion) : nullptr;
  float* d_point = point_out ? reinterpret_cast<float*>(m + s.point) : nullptr;
  const sf_status st =
      sf_scene_flow(m + s.img[0], m + s.img[1], m + s.img[2], m + s.img[3], pl->W,
                    reinterpret_cast<const float*>(m + s.flow), pl->W, pl->H, &pl->p, &pl->cam,
                    reinterpret_cast<float*>(m + s.s4), d_motion, d_point, m + s.valid, nullptr, nullptr,
                    m, pl->ws_bytes, pl->compute);
  if (st != SF_OK) return st;
  SF_PL_TRY(cudaEventRecord(s.computed, pl->compute));
  // copy-out
  SF_PL_TRY(cudaStreamWaitEvent(pl->out, s.computed, 0));
  SF_PL_TRY(cudaMemcpyAsync(s4_out, m + s.s4, N * 4 * sizeof(float), cudaMemcpyDeviceToHost, pl->out));
  SF_PL_TRY(cudaMemcpyAsync(valid_out, m + s.valid, N, cudaMemcpyDeviceToHost, pl->out));
  if (motion_out)
    SF_PL_TRY(cudaMemcpyAsync(motion_out, d_motion, N * 3 * sizeof(float), cudaMemcpyDeviceToHost, pl->out));
  if (point_out)
    SF_PL_TRY(cudaMemcpyAsync(point_out, d_point, N * 3 * sizeof(float), cudaMemcpyDeviceToHost, pl->out));
  SF_PL_TRY(cudaEventRecord(s.out_done, pl->out));
#undef SF_PL_TRY
  s.ticket = k;
  pl->next = k + 1;
  if (ticket) *ticket = k;
  return SF_OK;
}

sf_status sf_pipeline_wait(sf_pipeline* pl, int64_t ticket) {
  if (!pl) return SF_ERR_INVALID_ARG;
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lock(pl->mu);
    if (ticket < 0 || ticket >= pl->next) return SF_ERR_INVALID_ARG;
    // the slot's event was last recorded for this frame or a later one; the
    // copy-out stream is in order, so the later record completes after it
    ev = pl->slots[(size_t)(ticket % pl->depth)].out_done;
  }
  if (cudaEventSynchronize(ev) != cudaSuccess) {
    (void)cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

sf_status sf_pipeline_destroy(sf_pipeline* pl) {
  if (!pl) return SF_ERR_INVALID_ARG;
  sf_status st = SF_OK;
  {
    DeviceGuard guard(pl->device);
    if (cudaStreamSynchronize(pl->in) != cudaSuccess || cudaStreamSynchronize(pl->compute) != cudaSuccess ||
        cudaStreamSynchronize(pl->out) != cudaSuccess) {
      (void)cudaGetLastError();
      st = SF_ERR_CUDA;
    }
    release(pl);
  }
  return st;
}

}  // extern "C"
