// libsf C ABI: argument validation, workspace layout and stage orchestration.
// Every computational step runs in this library's own CUDA kernels.
#include <string.h>

#include <atomic>
#include <mutex>

#include "sf_fused.cuh"
#include "sf_internal.cuh"

using namespace sf;

namespace sf {

namespace {
std::atomic<uint64_t> g_launches{0};
struct TraceState {
  void* const* events = nullptr;
  int32_t n_events = 0;
  int32_t next = 0;
  int32_t* stage_out = nullptr;
  int32_t records = 0;
  bool armed = false;
  bool open = false;
} g_trace;
}  // namespace

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

void trace_begin(int stage, cudaStream_t s) {
  TraceState& t = g_trace;
  if (!t.armed || t.open || t.next + 2 > t.n_events) return;
  if (cudaEventRecord((cudaEvent_t)t.events[t.next], s) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  t.stage_out[t.records] = stage;
  t.open = true;
}

void trace_end(cudaStream_t s) {
  TraceState& t = g_trace;
  if (!t.open) return;
  if (cudaEventRecord((cudaEvent_t)t.events[t.next + 1], s) != cudaSuccess) (void)cudaGetLastError();
  t.next += 2;
  t.records++;
  t.open = false;
}

}  // namespace sf

namespace {

#define SF_TRY_CUDA(expr)                 \
  do {                                    \
    if ((expr) != cudaSuccess) {          \
      (void)cudaGetLastError();           \
      return SF_ERR_CUDA;                 \
    }                                     \
  } while (0)

sf_status check_size(int32_t W, int32_t H) {
  if (W <= 0 || H <= 0) return SF_ERR_INVALID_ARG;
  if ((int64_t)W * H > (int64_t)1 << 26) return SF_ERR_UNSUPPORTED;  // 64 Mpx
  if (W > 32767 || H > 32767) return SF_ERR_UNSUPPORTED;
  return SF_OK;
}

sf_status check_census(int32_t cw, int32_t ch, int32_t W, int32_t H) {
  if (cw <= 0 || ch <= 0 || (cw % 2) == 0 || (ch % 2) == 0) return SF_ERR_INVALID_ARG;
  if (cw * ch - 1 > 64) return SF_ERR_INVALID_ARG;
  if (W < cw || H < ch) return SF_ERR_INVALID_ARG;
  return SF_OK;
}

sf_status check_params(const sf_sgm_params* p, int32_t W, int32_t H) {
  if (!p) return SF_ERR_INVALID_ARG;
  sf_status st = check_census(p->census_w, p->census_h, W, H);
  if (st != SF_OK) return st;
  if (p->D < 1 || p->D > SF_MAX_DISPARITY) return SF_ERR_INVALID_ARG;
  if (p->P2 < p->P1) return SF_ERR_INVALID_ARG;
  const int cmax = p->census_w * p->census_h - 1;
  if (cmax + (int)p->P2 > 255) return SF_ERR_UNSUPPORTED;
  if (p->path_mask & ~0xffu) return SF_ERR_INVALID_ARG;
  if (p->subpixel != 0 && p->subpixel != 1) return SF_ERR_INVALID_ARG;
  if (p->lr_tol < 0) return SF_ERR_INVALID_ARG;
  return SF_OK;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Workspace of sf_sgm_full / sf_scene_flow, carved with 256-byte alignment.
struct Workspace {
  size_t cost, agg, dL, dR, dsub, disp0, disp1, total;
  Workspace(int W, int H, int D) {
    const size_t N = (size_t)W * H;
    size_t o = 0;
    cost = o; o = align_up(o + N * D, 256);
    agg = o; o = align_up(o + N * D * sizeof(uint16_t), 256);
    dL = o; o = align_up(o + N * sizeof(int16_t), 256);
    dR = o; o = align_up(o + N * sizeof(int16_t), 256);
    dsub = o; o = align_up(o + N * sizeof(float), 256);
    disp0 = o; o = align_up(o + N * sizeof(float), 256);
    disp1 = o; o = align_up(o + N * sizeof(float), 256);
    total = o;
  }
};

// Staging area that sf_scene_flow_host appends after the regular workspace.
struct HostStaging {
  size_t img[4], flow, s4, motion, point, valid, total;
  HostStaging(int W, int H, size_t base) {
    const size_t N = (size_t)W * H;
    size_t o = base;
    for (int k = 0; k < 4; k++) { img[k] = o; o = align_up(o + N, 256); }
    flow = o; o = align_up(o + N * 2 * sizeof(float), 256);
    s4 = o; o = align_up(o + N * 4 * sizeof(float), 256);
    motion = o; o = align_up(o + N * 3 * sizeof(float), 256);
    point = o; o = align_up(o + N * 3 * sizeof(float), 256);
    valid = o; o = align_up(o + N, 256);
    total = o;
  }
};

sf_status sgm_full_impl(const uint8_t* left, const uint8_t* right, int W, int H, int pitch,
                        const sf_sgm_params* p, int16_t* dL_out, int16_t* dR_out,
                        uint8_t* valid_out, float* disp_out, uint8_t* ws, cudaStream_t s) {
  Workspace lay(W, H, p->D);
  uint8_t* cost = ws + lay.cost;
  uint16_t* agg = reinterpret_cast<uint16_t*>(ws + lay.agg);
  int16_t* dL = dL_out ? dL_out : reinterpret_cast<int16_t*>(ws + lay.dL);
  int16_t* dR = dR_out ? dR_out : reinterpret_cast<int16_t*>(ws + lay.dR);
  float* dsub = reinterpret_cast<float*>(ws + lay.dsub);
  uint8_t* valid = valid_out;
  // left image as reference
  SF_TRY_CUDA(launch_cost_volume(left, right, W, H, pitch, p->census_w, p->census_h, p->D, 0, cost, s));
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg, s));
  SF_TRY_CUDA(launch_select(agg, W, H, p->D, p->subpixel, dL, dsub, s));
  // right image as reference
  SF_TRY_CUDA(launch_cost_volume(right, left, W, H, pitch, p->census_w, p->census_h, p->D, 1, cost, s));
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg, s));
  SF_TRY_CUDA(launch_select(agg, W, H, p->D, 0, dR, nullptr, s));
  if (!valid) valid = reinterpret_cast<uint8_t*>(ws + lay.cost);  // cost is dead by now
  SF_TRY_CUDA(launch_lr_check(dL, dR, dsub, W, H, p->lr_tol, valid, disp_out, s));
  return SF_OK;
}

bool g_use_fused = true;

// Whether the fused stereo kernels handle this request (otherwise the staged
// kernels above run): a whole image row of distances must fit one CTA's
// shared memory.
bool fused_eligible(int W, int H, const sf_sgm_params* p) {
  (void)H;
  if (!g_use_fused) return false;
  return fused::cost_pair_smem(W, p->D) <= 227u * 1024u;
}

// Workspace of the fused path for `npairs` stereo pairs (2 passes each).
struct FusedLayout {
  size_t census, cost, hvol, sdown, bs, flags, err, dint, dsub, valid, disp, total;
  FusedLayout(int W, int H, int D, int npairs) {
    const size_t N = (size_t)W * H;
    const int Dp = fused::padded_d(D), npass = 2 * npairs;
    const int J = (W + fused::kTW - 1) / fused::kTW;
    size_t o = 0;
    census = o; o = align_up(o + (size_t)npass * N * sizeof(uint64_t), 256);
    cost = o; o = align_up(o + (size_t)npass * N * Dp, 256);
    hvol = o; o = align_up(o + (size_t)npass * 2 * N * Dp, 256);
    sdown = o; o = align_up(o + fused::sdown_bytes(W, H, D, npass), 256);
    bs = o; o = align_up(o + fused::bs_bytes(W, D, npass), 256);
    flags = o; o = align_up(o + (size_t)2 * (npass * J + 1) * sizeof(int), 256);
    err = o; o = align_up(o + 256, 256);
    dint = o; o = align_up(o + (size_t)npass * N * sizeof(int16_t), 256);
    dsub = o; o = align_up(o + (size_t)npairs * N * sizeof(float), 256);
    valid = o; o = align_up(o + (size_t)npairs * N, 256);
    disp = o; o = align_up(o + (size_t)npairs * N * sizeof(float), 256);
    total = o;
  }
};

constexpr long long kSpinLimit = 1ll << 24;   // bounded neighbour wait (~1 s)

// Side stream on which the horizontal-path kernel overlaps the down sweep
// (one per device, created on first use; fork and join through events so the
// pattern also works under CUDA graph capture of the caller's stream).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_side_mu;
SideStream g_side[64];

cudaError_t side_stream(SideStream** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  SideStream& ss = g_side[dev];
  if (!ss.s) {
    if ((e = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *out = &ss;
  return cudaSuccess;
}

// Band sweeps + horizontal paths for `npass` cost volumes already in place.
sf_status run_aggregation(int W, int H, const sf_sgm_params* p, int npass, uint8_t* ws,
                          const FusedLayout& lay, const fused::PassIO* io_up, cudaStream_t s) {
  const size_t N = (size_t)W * H;
  const int Dp = fused::padded_d(p->D);
  const int J = (W + fused::kTW - 1) / fused::kTW;
  uint8_t* cost = ws + lay.cost;
  uint8_t* hvol = ws + lay.hvol;
  fused::HLineArgs ha{};
  ha.W = W; ha.H = H; ha.D = p->D; ha.Dp = Dp; ha.npass = npass; ha.P1 = p->P1; ha.P2 = p->P2;
  ha.path_mask = p->path_mask;
  ha.err = reinterpret_cast<int*>(ws + lay.err);
  for (int k = 0; k < npass; k++) {
    ha.cost[k] = io_up[k].cost ? io_up[k].cost : cost + (size_t)k * N * Dp;
    ha.hfwd[k] = hvol + (size_t)(2 * k) * N * Dp;
    ha.hbwd[k] = hvol + (size_t)(2 * k + 1) * N * Dp;
  }
  SF_TRY_CUDA(cudaMemsetAsync(ws + lay.err, 0, sizeof(int), s));
  // the horizontal paths run beside the down sweep; the up sweep joins them
  std::lock_guard<std::mutex> guard(g_side_mu);
  SideStream* side = nullptr;
  SF_TRY_CUDA(side_stream(&side));
  SF_TRY_CUDA(cudaEventRecord(side->fork, s));
  SF_TRY_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0));
  SF_TRY_CUDA(fused::launch_hline(ha, side->s));
  SF_TRY_CUDA(cudaEventRecord(side->join, side->s));
  int* flags = reinterpret_cast<int*>(ws + lay.flags);
  SF_TRY_CUDA(cudaMemsetAsync(flags, 0, (size_t)2 * (npass * J + 1) * sizeof(int), s));
  fused::SweepArgs sa{};
  sa.W = W; sa.H = H; sa.D = p->D; sa.Dp = Dp; sa.P1 = p->P1; sa.P2 = p->P2; sa.J = J;
  sa.nb = (H + fused::band_rows(p->D) - 1) / fused::band_rows(p->D); sa.items = npass * J; sa.subpixel = p->subpixel;
  sa.path_mask = p->path_mask;
  sa.en_h0 = (p->path_mask >> 0) & 1u;
  sa.en_h1 = (p->path_mask >> 1) & 1u;
  sa.sdown = reinterpret_cast<uint32_t*>(ws + lay.sdown);
  sa.bs = ws + lay.bs;
  sa.err = reinterpret_cast<int*>(ws + lay.err);
  sa.spin_limit = kSpinLimit;
  for (int k = 0; k < npass; k++) {
    sa.io[k].cost = ha.cost[k];
    sa.io[k].hfwd = ha.hfwd[k];
    sa.io[k].hbwd = ha.hbwd[k];
  }
  sa.flags = flags;
  sa.task_counter = flags + 2 * npass * J;
  SF_TRY_CUDA(fused::launch_sweep(sa, false, s));
  for (int k = 0; k < npass; k++) {
    sa.io[k].dint = io_up[k].dint;
    sa.io[k].dsub = io_up[k].dsub;
    sa.io[k].S = io_up[k].S;
  }
  sa.flags = flags + npass * J;
  sa.task_counter = flags + 2 * npass * J + 1;
  SF_TRY_CUDA(cudaStreamWaitEvent(s, side->join, 0));
  SF_TRY_CUDA(fused::launch_sweep(sa, true, s));
  return SF_OK;
}

// Fused SGM for `npairs` stereo pairs: census, one distance computation per
// pair, both reference passes, the left-right check.
sf_status run_fused_pairs(const uint8_t* const* left, const uint8_t* const* right, int npairs,
                          int W, int H, int pitch, const sf_sgm_params* p, int16_t* const* dL_out,
                          int16_t* const* dR_out, uint8_t* const* valid_out, float* const* disp_out,
                          uint8_t* ws, cudaStream_t s) {
  FusedLayout lay(W, H, p->D, npairs);
  const size_t N = (size_t)W * H;
  const int Dp = fused::padded_d(p->D), npass = 2 * npairs;
  const int cmax = p->census_w * p->census_h - 1;
  uint64_t* census = reinterpret_cast<uint64_t*>(ws + lay.census);
  uint8_t* cost = ws + lay.cost;
  for (int k = 0; k < npairs; k++) {
    SF_TRY_CUDA(launch_census(left[k], W, H, pitch, p->census_w, p->census_h, census + (2 * k) * N, s));
    SF_TRY_CUDA(launch_census(right[k], W, H, pitch, p->census_w, p->census_h, census + (2 * k + 1) * N, s));
  }
  for (int k = 0; k < npairs; k++)
    SF_TRY_CUDA(fused::launch_cost_pair(census + (2 * k) * N, census + (2 * k + 1) * N, W, H, p->D, Dp,
                                        cmax, cost + (size_t)(2 * k) * N * Dp,
                                        cost + (size_t)(2 * k + 1) * N * Dp, s));
  int16_t* dint = reinterpret_cast<int16_t*>(ws + lay.dint);
  float* dsub = reinterpret_cast<float*>(ws + lay.dsub);
  fused::PassIO io[fused::kMaxPass] = {};
  for (int k = 0; k < npairs; k++) {
    io[2 * k].dint = (dL_out && dL_out[k]) ? dL_out[k] : dint + (size_t)(2 * k) * N;
    io[2 * k].dsub = dsub + (size_t)k * N;
    io[2 * k + 1].dint = (dR_out && dR_out[k]) ? dR_out[k] : dint + (size_t)(2 * k + 1) * N;
  }
  sf_status st = run_aggregation(W, H, p, npass, ws, lay, io, s);
  if (st != SF_OK) return st;
  for (int k = 0; k < npairs; k++) {
    uint8_t* valid = (valid_out && valid_out[k]) ? valid_out[k] : ws + lay.valid + (size_t)k * N;
    SF_TRY_CUDA(launch_lr_check(io[2 * k].dint, io[2 * k + 1].dint, io[2 * k].dsub, W, H, p->lr_tol,
                                valid, disp_out[k], s));
  }
  return SF_OK;
}

size_t workspace_bytes(int W, int H, const sf_sgm_params* p, int npairs) {
  if (fused_eligible(W, H, p)) return std::max(FusedLayout(W, H, p->D, npairs).total, Workspace(W, H, p->D).total);
  return Workspace(W, H, p->D).total;
}

}  // namespace

extern "C" {

void sf_default_params(sf_sgm_params* p) {
  if (!p) return;
  p->census_w = 9;
  p->census_h = 7;
  p->P1 = 7;
  p->P2 = 86;
  p->path_mask = 0xffu;
  p->D = 128;
  p->subpixel = 1;
  p->lr_tol = 1;
}

const char* sf_status_string(sf_status s) {
  switch (s) {
    case SF_OK: return "SF_OK";
    case SF_ERR_INVALID_ARG: return "SF_ERR_INVALID_ARG";
    case SF_ERR_UNSUPPORTED: return "SF_ERR_UNSUPPORTED";
    case SF_ERR_CUDA: return "SF_ERR_CUDA";
    case SF_ERR_TIMEOUT: return "SF_ERR_TIMEOUT";
  }
  return "SF_ERR_UNKNOWN";
}

sf_status sf_census(const uint8_t* img, int32_t W, int32_t H, int32_t pitch, int32_t census_w,
                    int32_t census_h, uint64_t* census_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!img || !census_out || pitch < W) return SF_ERR_INVALID_ARG;
  if ((st = check_census(census_w, census_h, W, H)) != SF_OK) return st;
  if (!aligned(census_out, 8)) return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_census(img, W, H, pitch, census_w, census_h, census_out, (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_cost_volume(const uint8_t* ref, const uint8_t* other, int32_t W, int32_t H,
                         int32_t pitch, const sf_sgm_params* p, int32_t ref_is_right,
                         uint8_t* cost_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!ref || !other || !cost_out || pitch < W) return SF_ERR_INVALID_ARG;
  if (ref_is_right != 0 && ref_is_right != 1) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  SF_TRY_CUDA(launch_cost_volume(ref, other, W, H, pitch, p->census_w, p->census_h, p->D,
                                 ref_is_right, cost_out, (cudaStream_t)stream));
  return SF_OK;
}

size_t sf_aggregate_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p) {
  if (check_size(W, H) != SF_OK || !p || p->D < 1 || p->D > SF_MAX_DISPARITY) return 0;
  if (p->D % 16 != 0) return 0;   // staged kernels, no workspace
  return FusedLayout(W, H, p->D, 1).total;
}

sf_status sf_sgm_aggregate(const uint8_t* cost, int32_t W, int32_t H, const sf_sgm_params* p,
                           uint16_t* agg_out, void* workspace, size_t ws_bytes, void* stream) {
  (void)workspace; (void)ws_bytes;
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!cost || !agg_out) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (!aligned(agg_out, 2)) return SF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // fused sweeps when the volume is 16-disparity aligned and a workspace of
  // sf_aggregate_workspace_size() bytes is given; staged kernels otherwise
  if (g_use_fused && p->D % 16 == 0 && aligned(cost, 16) && workspace && aligned(workspace, 256) &&
      ws_bytes >= FusedLayout(W, H, p->D, 1).total) {
    FusedLayout lay(W, H, p->D, 1);
    fused::PassIO io[fused::kMaxPass] = {};
    io[0].cost = cost;
    io[0].S = agg_out;
    return run_aggregation(W, H, p, 1, (uint8_t*)workspace, lay, io, s);
  }
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg_out, s));
  return SF_OK;
}

sf_status sf_disparity_select(const uint16_t* agg, int32_t W, int32_t H, int32_t D,
                              int32_t subpixel, int16_t* disp_int_out, float* disp_sub_out,
                              void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!agg || !disp_int_out) return SF_ERR_INVALID_ARG;
  if (D < 1 || D > SF_MAX_DISPARITY || (subpixel != 0 && subpixel != 1)) return SF_ERR_INVALID_ARG;
  if (!aligned(agg, 2) || !aligned(disp_int_out, 2) || !aligned(disp_sub_out, 4))
    return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_select(agg, W, H, D, subpixel, disp_int_out, disp_sub_out, (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_lr_check(const int16_t* dL, const int16_t* dR, const float* dL_sub, int32_t W,
                      int32_t H, int32_t tol, uint8_t* valid_out, float* disp_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!dL || !dR || !dL_sub || !valid_out || !disp_out || tol < 0) return SF_ERR_INVALID_ARG;
  if (!aligned(dL, 2) || !aligned(dR, 2) || !aligned(dL_sub, 4) || !aligned(disp_out, 4))
    return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_lr_check(dL, dR, dL_sub, W, H, tol, valid_out, disp_out, (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_combine_sceneflow(const float* D0, const float* D1, const float* flow, int32_t W,
                               int32_t H, const sf_camera* cam, float* s4_out, float* motion_out,
                               float* point_out, uint8_t* valid_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!D0 || !D1 || !flow || !cam || !s4_out || !valid_out) return SF_ERR_INVALID_ARG;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  if (!aligned(D0, 4) || !aligned(D1, 4) || !aligned(flow, 8) || !aligned(s4_out, 16) ||
      !aligned(motion_out, 4) || !aligned(point_out, 4))
    return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_combine(D0, D1, flow, W, H, cam->f, cam->B, cam->cx, cam->cy, s4_out,
                             motion_out, point_out, valid_out, (cudaStream_t)stream));
  return SF_OK;
}

size_t sf_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p) {
  if (check_size(W, H) != SF_OK || !p || p->D < 1 || p->D > SF_MAX_DISPARITY) return 0;
  return workspace_bytes(W, H, p, 2);
}

sf_status sf_sgm_full(const uint8_t* left, const uint8_t* right, int32_t W, int32_t H,
                      int32_t pitch, const sf_sgm_params* p, int16_t* dL_out, int16_t* dR_out,
                      uint8_t* valid_out, float* disp_out, void* workspace, size_t ws_bytes,
                      void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!left || !right || !disp_out || !workspace || pitch < W) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (ws_bytes < workspace_bytes(W, H, p, 1) || !aligned(workspace, 256)) return SF_ERR_INVALID_ARG;
  if (!aligned(dL_out, 2) || !aligned(dR_out, 2) || !aligned(disp_out, 4)) return SF_ERR_INVALID_ARG;
  if (fused_eligible(W, H, p))
    return run_fused_pairs(&left, &right, 1, W, H, pitch, p, &dL_out, &dR_out, &valid_out, &disp_out,
                           (uint8_t*)workspace, (cudaStream_t)stream);
  return sgm_full_impl(left, right, W, H, pitch, p, dL_out, dR_out, valid_out, disp_out,
                       (uint8_t*)workspace, (cudaStream_t)stream);
}

sf_status sf_scene_flow(const uint8_t* left_t, const uint8_t* right_t, const uint8_t* left_t1,
                        const uint8_t* right_t1, int32_t pitch, const float* flow, int32_t W,
                        int32_t H, const sf_sgm_params* p, const sf_camera* cam, float* s4_out,
                        float* motion_out, float* point_out, uint8_t* valid_out, float* D0_out,
                        float* D1_out, void* workspace, size_t ws_bytes, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!left_t || !right_t || !left_t1 || !right_t1 || !flow || !cam || !s4_out || !valid_out ||
      !workspace || pitch < W)
    return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  if (ws_bytes < workspace_bytes(W, H, p, 2) || !aligned(workspace, 256)) return SF_ERR_INVALID_ARG;
  if (!aligned(flow, 8) || !aligned(s4_out, 16) || !aligned(motion_out, 4) ||
      !aligned(point_out, 4) || !aligned(D0_out, 4) || !aligned(D1_out, 4))
    return SF_ERR_INVALID_ARG;
  uint8_t* ws = (uint8_t*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  float* D0;
  float* D1;
  if (fused_eligible(W, H, p)) {
    FusedLayout fl(W, H, p->D, 2);
    D0 = D0_out ? D0_out : reinterpret_cast<float*>(ws + fl.disp);
    D1 = D1_out ? D1_out : reinterpret_cast<float*>(ws + fl.disp) + (size_t)W * H;
    const uint8_t* L[2] = {left_t, left_t1};
    const uint8_t* R[2] = {right_t, right_t1};
    float* disp[2] = {D0, D1};
    if ((st = run_fused_pairs(L, R, 2, W, H, pitch, p, nullptr, nullptr, nullptr, disp, ws, s)) != SF_OK)
      return st;
  } else {
    Workspace lay(W, H, p->D);
    D0 = D0_out ? D0_out : reinterpret_cast<float*>(ws + lay.disp0);
    D1 = D1_out ? D1_out : reinterpret_cast<float*>(ws + lay.disp1);
    if ((st = sgm_full_impl(left_t, right_t, W, H, pitch, p, nullptr, nullptr, nullptr, D0, ws, s)) != SF_OK)
      return st;
    if ((st = sgm_full_impl(left_t1, right_t1, W, H, pitch, p, nullptr, nullptr, nullptr, D1, ws, s)) != SF_OK)
      return st;
  }
  SF_TRY_CUDA(launch_combine(D0, D1, flow, W, H, cam->f, cam->B, cam->cx, cam->cy, s4_out,
                             motion_out, point_out, valid_out, s));
  return SF_OK;
}

size_t sf_scene_flow_host_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p) {
  const size_t base = sf_workspace_size(W, H, p);
  if (base == 0) return 0;
  return HostStaging(W, H, base).total;
}

sf_status sf_scene_flow_host(const uint8_t* left_t, const uint8_t* right_t,
                             const uint8_t* left_t1, const uint8_t* right_t1, const float* flow,
                             int32_t W, int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                             float* s4_out, float* motion_out, float* point_out,
                             uint8_t* valid_out, void* dev_workspace, size_t ws_bytes,
                             void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!left_t || !right_t || !left_t1 || !right_t1 || !flow || !cam || !s4_out || !valid_out ||
      !dev_workspace)
    return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  const size_t base = workspace_bytes(W, H, p, 2);
  HostStaging hs(W, H, base);
  if (ws_bytes < hs.total || !aligned(dev_workspace, 256)) return SF_ERR_INVALID_ARG;
  uint8_t* ws = (uint8_t*)dev_workspace;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)W * H;
  const uint8_t* imgs[4] = {left_t, right_t, left_t1, right_t1};
  for (int k = 0; k < 4; k++)
    SF_TRY_CUDA(cudaMemcpyAsync(ws + hs.img[k], imgs[k], N, cudaMemcpyHostToDevice, s));
  SF_TRY_CUDA(cudaMemcpyAsync(ws + hs.flow, flow, N * 2 * sizeof(float), cudaMemcpyHostToDevice, s));
  float* d_motion = motion_out ? reinterpret_cast<float*>(ws + hs.motion) : nullptr;
  float* d_point = point_out ? reinterpret_cast<float*>(ws + hs.point) : nullptr;
  st = sf_scene_flow(ws + hs.img[0], ws + hs.img[1], ws + hs.img[2], ws + hs.img[3], W,
                     reinterpret_cast<const float*>(ws + hs.flow), W, H, p, cam,
                     reinterpret_cast<float*>(ws + hs.s4), d_motion, d_point, ws + hs.valid,
                     nullptr, nullptr, ws, base, stream);
  if (st != SF_OK) return st;
  SF_TRY_CUDA(cudaMemcpyAsync(s4_out, ws + hs.s4, N * 4 * sizeof(float), cudaMemcpyDeviceToHost, s));
  SF_TRY_CUDA(cudaMemcpyAsync(valid_out, ws + hs.valid, N, cudaMemcpyDeviceToHost, s));
  if (motion_out)
    SF_TRY_CUDA(cudaMemcpyAsync(motion_out, d_motion, N * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (point_out)
    SF_TRY_CUDA(cudaMemcpyAsync(point_out, d_point, N * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
  SF_TRY_CUDA(cudaStreamSynchronize(s));
  return SF_OK;
}

sf_status sf_trace_arm(void* const* events, int32_t n_events, int32_t* stage_out) {
  if (!events || !stage_out || n_events < 2) return SF_ERR_INVALID_ARG;
  g_trace = TraceState();
  g_trace.events = events;
  g_trace.n_events = n_events;
  g_trace.stage_out = stage_out;
  g_trace.armed = true;
  return SF_OK;
}

int32_t sf_trace_disarm(void) {
  const int32_t n = g_trace.records;
  g_trace = TraceState();
  return n;
}

uint64_t sf_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

sf_status sf_set_fused(int32_t enable) {
  if (enable != 0 && enable != 1) return SF_ERR_INVALID_ARG;
  g_use_fused = enable != 0;
  return SF_OK;
}

sf_status sf_check_workspace(const void* workspace, int32_t W, int32_t H, const sf_sgm_params* p,
                             int32_t npairs, void* stream) {
  if (!workspace || !p || check_size(W, H) != SF_OK || (npairs != 1 && npairs != 2))
    return SF_ERR_INVALID_ARG;
  if (!fused_eligible(W, H, p)) return SF_OK;
  FusedLayout lay(W, H, p->D, npairs);
  int err = 0;
  cudaStream_t s = (cudaStream_t)stream;
  SF_TRY_CUDA(cudaMemcpyAsync(&err, (const uint8_t*)workspace + lay.err, sizeof(int),
                              cudaMemcpyDeviceToHost, s));
  SF_TRY_CUDA(cudaStreamSynchronize(s));
  return err ? SF_ERR_TIMEOUT : SF_OK;
}

}  // extern "C"
