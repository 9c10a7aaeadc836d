// libsf C ABI: argument validation, workspace layout and stage orchestration.
// Every computational step runs in this library's own CUDA kernels.
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>
#include <algorithm>

#include "sf_confnet.cuh"
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
  if (p->adaptive_p2 != 0 && p->adaptive_p2 != 1) return SF_ERR_INVALID_ARG;
  if (p->uniqueness < 0 || p->uniqueness > 99) return SF_ERR_INVALID_ARG;
  return SF_OK;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Completion flags of the horizontal paths' row blocks of one pass (two
// directions, row blocks of at least 16 rows) for the launch that runs them
// beside the sweeps.
inline int flags_h_count(int H) { return 2 * ((H + 3) / 4); }   // row blocks of 4 rows or more

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
  // left image as reference (the guide of the adaptive P2 is the pass's
  // reference image; the uniqueness filter applies to the left winners)
  SF_TRY_CUDA(launch_cost_volume(left, right, W, H, pitch, p->census_w, p->census_h, p->D, 0, cost, s));
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg, s,
                               p->adaptive_p2 ? left : nullptr, pitch));
  SF_TRY_CUDA(launch_select(agg, W, H, p->D, p->subpixel, dL, dsub, s, p->uniqueness));
  // right image as reference
  SF_TRY_CUDA(launch_cost_volume(right, left, W, H, pitch, p->census_w, p->census_h, p->D, 1, cost, s));
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg, s,
                               p->adaptive_p2 ? right : nullptr, pitch));
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
  (void)W;
  (void)p;
  return g_use_fused;
}

// ---- fused-path workspace --------------------------------------------------
// A control block (error word, task counters, per-pass band flags: zeroed by
// one memset per call) followed by the buffers of each stereo pair.
struct PassBuffers {
  size_t cost, hf, hb, sdown, bs, dint, flags;   // flags: offset in the control block
};
struct PairBuffers {
  size_t census_l, census_r, dsub, valid, disp;
  PassBuffers pass[2];
};
struct PairShape {
  int W, H, D;
};

size_t carve(size_t& o, size_t bytes) {
  const size_t at = o;
  o = align_up(o + bytes, 256);
  return at;
}

struct FusedPlan {
  std::vector<PairBuffers> pairs;
  size_t err = 0, counters = 0, control_bytes = 0, tables = 0, total = 0;
  int ncounters = 0;
  // Dshape(i): the D that fixes the kernel shape of pair i's sweeps
  FusedPlan(const PairShape* ps, int n, const int* dshape, int ncounters_, size_t table_bytes) {
    pairs.resize(n);
    ncounters = ncounters_;
    size_t c = 0;
    err = c; c += sizeof(int);
    counters = c; c += (size_t)ncounters * sizeof(int);
    for (int i = 0; i < n; i++) {
      const int J = (ps[i].W + fused::kTW - 1) / fused::kTW;
      for (int k = 0; k < 2; k++) {
        pairs[i].pass[k].flags = c;
        c += (size_t)(2 * J + flags_h_count(ps[i].H)) * sizeof(int);
      }
    }
    control_bytes = align_up(c, 256);
    size_t o = control_bytes;
    tables = carve(o, table_bytes);
    for (int i = 0; i < n; i++) {
      const int W = ps[i].W, H = ps[i].H, D = ps[i].D;
      const size_t N = (size_t)W * H;
      const int Dp = fused::padded_d(D);
      PairBuffers& b = pairs[i];
      b.census_l = carve(o, N * sizeof(uint64_t));
      b.census_r = carve(o, N * sizeof(uint64_t));
      for (int k = 0; k < 2; k++) {
        PassBuffers& pb = b.pass[k];
        pb.cost = carve(o, N * Dp);
        pb.hf = carve(o, N * Dp);
        pb.hb = carve(o, N * Dp);
        pb.sdown = carve(o, fused::sdown_bytes(W, H, dshape[i]));
        pb.bs = carve(o, fused::bs_bytes(W, D));
        pb.dint = carve(o, N * sizeof(int16_t));
      }
      b.dsub = carve(o, N * sizeof(float));
      b.valid = carve(o, N);
      b.disp = carve(o, N * sizeof(float));
    }
    total = o;
  }
};

FusedPlan single_plan(int W, int H, int D, int npairs) {
  PairShape ps[2] = {{W, H, D}, {W, H, D}};
  int dshape[2] = {D, D};
  return FusedPlan(ps, npairs, dshape, 2, 0);
}

constexpr long long kSpinLimit = 1ll << 24;   // bounded neighbour wait (~1 s)

// Test hooks (sf_debug_set): poll limit of the bounded waits, and tasks the
// down sweep's queue skips (their bands are never computed, so the waits of
// later bands run out).
std::atomic<long long> g_spin_limit{kSpinLimit};
std::atomic<int> g_skip_down_tasks{0};

// Pass descriptor of pass k of a pair laid out at `b` in workspace ws.
fused::PassDesc pass_desc(uint8_t* ws, const FusedPlan& plan, const PairBuffers& b, int k, int W,
                          int H, int D, int Dshape, const uint8_t* cost_override) {
  fused::PassDesc d{};
  d.W = W; d.H = H; d.D = D; d.Dp = fused::padded_d(D);
  d.J = (W + fused::kTW - 1) / fused::kTW;
  const int th = fused::band_rows(Dshape);
  d.nb = (H + th - 1) / th;
  const PassBuffers& pb = b.pass[k];
  d.cost = cost_override ? cost_override : ws + pb.cost;
  d.hfwd = ws + pb.hf;
  d.hbwd = ws + pb.hb;
  d.sdown = reinterpret_cast<uint32_t*>(ws + pb.sdown);
  d.bs = ws + pb.bs;
  d.flags_down = reinterpret_cast<int*>(ws + pb.flags);
  d.flags_up = d.flags_down + d.J;
  d.flags_h = d.flags_up + d.J;
  d.dint = reinterpret_cast<int16_t*>(ws + pb.dint);
  d.dsub = nullptr;
  d.S = nullptr;
  d.guide = nullptr;
  d.gpitch = 0;
  (void)plan;
  return d;
}

// Task tables of a set of passes with one kernel shape: passes sorted by band
// count (descending); step-major task order (a merged launch lists each step's
// tasks twice, down sweep then up sweep).  Written to `tab` (host ints):
// [band_start (nb+1)] [band_npass (nb)] [prefixJ (npass+1)] [hline block prefix (npass+1)].
struct TaskTables {
  std::vector<int> ints;
  int nbands = 0, ntasks = 0, nblocks = 0, off_band_start = 0, off_band_npass = 0, off_prefixJ = 0,
      off_hblocks = 0;
  int hline_rows = 16;   // rows per block of the horizontal-path kernel
};
TaskTables build_tables(const fused::PassDesc* d, int npass, bool merged, int Dshape) {
  TaskTables t;
  int nb_max = 0;
  for (int k = 0; k < npass; k++) nb_max = std::max(nb_max, d[k].nb);
  t.nbands = nb_max;
  t.off_band_start = 0;
  t.off_band_npass = nb_max + 1;
  t.off_prefixJ = t.off_band_npass + nb_max;
  t.off_hblocks = t.off_prefixJ + npass + 1;
  t.ints.assign(t.off_hblocks + npass + 1, 0);
  int* prefixJ = &t.ints[t.off_prefixJ];
  for (int k = 0; k < npass; k++) prefixJ[k + 1] = prefixJ[k] + d[k].J;
  int task = 0;
  for (int b = 0; b < nb_max; b++) {
    int active = 0;
    while (active < npass && d[active].nb > b) active++;
    t.ints[t.off_band_start + b] = task;
    t.ints[t.off_band_npass + b] = active;
    task += (merged ? 2 : 1) * prefixJ[active];
  }
  t.ints[t.off_band_start + nb_max] = task;
  t.ntasks = task;
  int* hb = &t.ints[t.off_hblocks];
  t.hline_rows = fused::hline_block_rows(Dshape);
  for (int k = 0; k < npass; k++) hb[k + 1] = hb[k] + 2 * ((d[k].H + t.hline_rows - 1) / t.hline_rows);
  t.nblocks = hb[npass];
  return t;
}

// Horizontal paths, the down sweep, then the up sweep, for passes that share
// one kernel shape, in stream order.  Run side by side on a second stream,
// the horizontal kernel and the down sweep (both latency-bound chains) gave
// frame times that depended on how their blocks landed on the SMs (the
// 1242 x 375, D = 128 frame: about 1.45 or 1.70 ms, varying from run to run
// and process to process); one after the other the frame takes a steady
// 1.64 ms.
sf_status run_sweeps(const sf_sgm_params* p, const fused::PassDesc* d, int npass, int Dshape,
                     const fused::PassDesc* d_dev_down, const fused::PassDesc* d_dev_up,
                     const int* tab_dev, const TaskTables* tt, int* counters, int* err,
                     cudaStream_t s, int table = fused::kShapePlain) {
  const bool inl = d_dev_down == nullptr;
  const fused::Shape shape = fused::shape_for(Dshape, table);
  const bool merged = shape.order >= 1;
  // the horizontal paths inside the sweep launch: passes of one size (the
  // batch's uneven passes keep their own launch)
  const bool with_h = shape.order == 2 && inl;
  fused::HLineArgs ha{};
  ha.P1 = p->P1; ha.P2 = p->P2; ha.Dmax = Dshape; ha.npass = npass; ha.path_mask = p->path_mask;
  ha.shape_table = table;
  ha.err = err;
  fused::SweepArgs sa{};
  sa.shape_table = table;
  sa.P1 = p->P1; sa.P2 = p->P2; sa.subpixel = p->subpixel; sa.Dmax = Dshape; sa.npass = npass;
  sa.unique = p->uniqueness;
  sa.variants = (p->adaptive_p2 || p->uniqueness) ? 1 : 0;
  sa.path_mask = p->path_mask;
  sa.en_h0 = (p->path_mask >> 0) & 1u;
  sa.en_h1 = (p->path_mask >> 1) & 1u;
  sa.err = err;
  sa.spin_limit = g_spin_limit.load(std::memory_order_relaxed);
  if (inl) {
    for (int k = 0; k < npass; k++) ha.inl[k] = sa.inl[k] = d[k];
    ha.block_rows = fused::hline_block_rows(Dshape);
    ha.uniform_blocks = 2 * ((d[0].H + ha.block_rows - 1) / ha.block_rows);
    ha.nblocks = npass * ha.uniform_blocks;
    sa.uniform_items = npass * d[0].J;
    sa.ntasks = (merged ? 2 : 1) * d[0].nb * sa.uniform_items;
    sa.nbands = d[0].nb;
  } else {
    ha.pass_ptr = d_dev_down;
    ha.block_prefix = tab_dev + tt->off_hblocks;
    ha.nblocks = tt->nblocks;
    ha.block_rows = tt->hline_rows;
    sa.pass_ptr = d_dev_down;
    sa.band_start = tab_dev + tt->off_band_start;
    sa.band_npass = tab_dev + tt->off_band_npass;
    sa.prefixJ = tab_dev + tt->off_prefixJ;
    sa.nbands = tt->nbands;
    sa.ntasks = tt->ntasks;
  }
  if (with_h) {
    const int rows = fused::merged_hline_rows(shape.dc, shape.chunks, shape.halo);
    sa.hl_blocks = (d[0].H + rows - 1) / rows;
    sa.hl_tasks = npass * 2 * sa.hl_blocks;
    sa.ntasks += sa.hl_tasks;
  } else {
    SF_TRY_CUDA(fused::launch_hline(ha, s));
  }
  sa.task_counter = counters;
  if (const int skip = g_skip_down_tasks.load(std::memory_order_relaxed)) {
    static int skip_host;
    skip_host = skip;
    SF_TRY_CUDA(cudaMemcpyAsync(counters, &skip_host, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  if (merged) {
    // both scan orders in one launch; every task may select, so all use the
    // descriptors that carry the outputs
    if (inl) {
      for (int k = 0; k < npass; k++) sa.inl[k] = d[k];
    } else {
      sa.pass_ptr = d_dev_up;
    }
    SF_TRY_CUDA(fused::launch_sweep(sa, with_h ? 3 : 2, s));
    return SF_OK;
  }
  SF_TRY_CUDA(fused::launch_sweep(sa, 0, s));
  if (inl) {
    for (int k = 0; k < npass; k++) sa.inl[k] = d[k];   // with outputs of the up sweep
  } else {
    sa.pass_ptr = d_dev_up;
  }
  sa.task_counter = counters + 1;
  SF_TRY_CUDA(fused::launch_sweep(sa, 1, s));
  return SF_OK;
}

// Census of `npairs` stereo pairs of one size, then the shared distance
// computation of all of them in one launch (the rows of every pair spread
// over the persistent CTAs).
sf_status run_pair_costs(const uint8_t* const* left, const uint8_t* const* right, int npairs, int W, int H,
                         int pitch, int D, const sf_sgm_params* p, uint8_t* ws, const PairBuffers* const* b,
                         cudaStream_t s) {
  if (npairs < 1 || npairs > fused::kMaxPass) return SF_ERR_INVALID_ARG;
  fused::CostPairs job{};
  job.npairs = npairs;
  const uint8_t* imgs[2 * fused::kMaxPass];
  uint64_t* cens[2 * fused::kMaxPass];
  for (int k = 0; k < npairs; k++) {
    uint64_t* cl = reinterpret_cast<uint64_t*>(ws + b[k]->census_l);
    uint64_t* cr = reinterpret_cast<uint64_t*>(ws + b[k]->census_r);
    imgs[2 * k] = left[k];
    imgs[2 * k + 1] = right[k];
    cens[2 * k] = cl;
    cens[2 * k + 1] = cr;
    job.cL[k] = cl;
    job.cR[k] = cr;
    job.CL[k] = ws + b[k]->pass[0].cost;
    job.CR[k] = ws + b[k]->pass[1].cost;
  }
  // every image's census in one launch
  SF_TRY_CUDA(launch_census_images(imgs, cens, 2 * npairs, W, H, pitch, p->census_w, p->census_h, s));
  SF_TRY_CUDA(fused::launch_cost_pair(job, W, H, D, fused::padded_d(D), p->census_w * p->census_h - 1, s));
  return SF_OK;
}

// Fused SGM for `npairs` stereo pairs of one size: census, one distance
// computation per pair, both reference passes, the left-right check.
// With d_out given, the left-right checks are left to the caller, who gets
// the passes' descriptors (winners, subpixel maps) there.
sf_status run_fused_pairs(const uint8_t* const* left, const uint8_t* const* right, int npairs,
                          int W, int H, int pitch, const sf_sgm_params* p, int16_t* const* dL_out,
                          int16_t* const* dR_out, uint8_t* const* valid_out, float* const* disp_out,
                          uint8_t* ws, cudaStream_t s, fused::PassDesc* d_out = nullptr) {
  FusedPlan plan = single_plan(W, H, p->D, npairs);
  const size_t N = (size_t)W * H;
  SF_TRY_CUDA(cudaMemsetAsync(ws, 0, plan.control_bytes, s));
  {
    const PairBuffers* bufs[fused::kMaxPass];
    for (int k = 0; k < npairs; k++) bufs[k] = &plan.pairs[k];
    sf_status st = run_pair_costs(left, right, npairs, W, H, pitch, p->D, p, ws, bufs, s);
    if (st != SF_OK) return st;
  }
  fused::PassDesc d[fused::kMaxPass];
  for (int k = 0; k < npairs; k++) {
    for (int r = 0; r < 2; r++) {
      fused::PassDesc& pd = d[2 * k + r];
      pd = pass_desc(ws, plan, plan.pairs[k], r, W, H, p->D, p->D, nullptr);
      if (p->adaptive_p2) {
        pd.guide = r == 0 ? left[k] : right[k];
        pd.gpitch = pitch;
      }
      int16_t* const* user = r == 0 ? dL_out : dR_out;
      if (user && user[k]) pd.dint = user[k];
      if (r == 0) pd.dsub = reinterpret_cast<float*>(ws + plan.pairs[k].dsub);
    }
  }
  sf_status st = run_sweeps(p, d, 2 * npairs, p->D, nullptr, nullptr, nullptr, nullptr,
                            reinterpret_cast<int*>(ws + plan.counters), reinterpret_cast<int*>(ws + plan.err), s);
  if (st != SF_OK) return st;
  if (d_out) {
    for (int k = 0; k < 2 * npairs; k++) d_out[k] = d[k];
    return SF_OK;
  }
  for (int k = 0; k < npairs; k++) {
    uint8_t* valid = (valid_out && valid_out[k]) ? valid_out[k] : ws + plan.pairs[k].valid;
    SF_TRY_CUDA(launch_lr_check(d[2 * k].dint, d[2 * k + 1].dint, d[2 * k].dsub, W, H, p->lr_tol, valid,
                                disp_out[k], s));
  }
  (void)N;
  return SF_OK;
}

std::vector<int> b_shape_keys() {
  std::vector<int> v;
  for (int D = 16; D <= SF_MAX_DISPARITY; D += 16) {
    const fused::Shape sh = fused::shape_for(D);
    v.push_back(sh.order * 1000000 + sh.dc * 10000 + sh.chunks * 100 + sh.halo);
  }
  return v;
}

// ---- batches ----------------------------------------------------------------
// Every item contributes two stereo pairs (t, t+1) = four passes.  Passes are
// grouped by kernel shape; each group shares one persistent down sweep and one
// up sweep whose descriptors and task tables live in the workspace.
struct BatchClass {
  fused::Shape sh;
  int Dshape = 0;
  std::vector<int> pass_ids;   // sorted by band count, descending
  TaskTables tt;
  size_t off_down = 0, off_up = 0, off_tab = 0;   // within the tables region
};

struct BatchSetup {
  std::vector<PairShape> pairs;
  std::vector<int> dshape;
  std::vector<BatchClass> classes;
  size_t table_bytes = 0;
  sf_status status = SF_OK;
};

sf_status check_item(const sf_batch_item& it, const sf_sgm_params* p) {
  sf_status st = check_size(it.W, it.H);
  if (st != SF_OK) return st;
  if (!it.left_t || !it.right_t || !it.left_t1 || !it.right_t1 || !it.flow || !it.s4_out ||
      !it.valid_out || it.pitch < it.W)
    return SF_ERR_INVALID_ARG;
  if (it.D < 1 || it.D > SF_MAX_DISPARITY) return SF_ERR_INVALID_ARG;
  if (!(it.cam.f > 0.0f) || !(it.cam.B > 0.0f)) return SF_ERR_INVALID_ARG;
  if (!aligned(it.flow, 8) || !aligned(it.s4_out, 16) || !aligned(it.motion_out, 4) ||
      !aligned(it.point_out, 4) || !aligned(it.D0_out, 4) || !aligned(it.D1_out, 4))
    return SF_ERR_INVALID_ARG;
  sf_sgm_params q = *p;
  q.D = it.D;
  if ((st = check_params(&q, it.W, it.H)) != SF_OK) return st;
  return SF_OK;
}

BatchSetup batch_setup(const sf_batch_item* items, int n, const sf_sgm_params* p) {
  BatchSetup b;
  if (!items || n < 1 || !p) {
    b.status = SF_ERR_INVALID_ARG;
    return b;
  }
  for (int i = 0; i < n; i++) {
    if ((b.status = check_item(items[i], p)) != SF_OK) return b;
    for (int f = 0; f < 2; f++) {
      b.pairs.push_back({items[i].W, items[i].H, items[i].D});
      b.dshape.push_back(items[i].D);
    }
  }
  const int npass = 2 * (int)b.pairs.size();
  for (int id = 0; id < npass; id++) {
    const PairShape& ps = b.pairs[id / 2];
    const fused::Shape sh = fused::shape_for(ps.D);
    int c = 0;
    for (; c < (int)b.classes.size(); c++) {
      const fused::Shape& o = b.classes[c].sh;
      if (o.dc == sh.dc && o.chunks == sh.chunks && o.halo == sh.halo && o.order == sh.order) break;
    }
    if (c == (int)b.classes.size()) {
      b.classes.push_back(BatchClass());
      b.classes[c].sh = sh;
      b.classes[c].Dshape = ps.D;
    }
    b.classes[c].Dshape = std::max(b.classes[c].Dshape, ps.D);
    b.classes[c].pass_ids.push_back(id);
  }
  size_t o = 0;
  for (BatchClass& c : b.classes) {
    const int th = c.sh.halo + 1;
    auto nb_of = [&](int id) { return (b.pairs[id / 2].H + th - 1) / th; };
    std::stable_sort(c.pass_ids.begin(), c.pass_ids.end(),
                     [&](int x, int y) { return nb_of(x) > nb_of(y); });
    std::vector<fused::PassDesc> tmp(c.pass_ids.size());
    for (size_t k = 0; k < c.pass_ids.size(); k++) {
      const PairShape& ps = b.pairs[c.pass_ids[k] / 2];
      tmp[k] = fused::PassDesc{};
      tmp[k].W = ps.W;
      tmp[k].H = ps.H;
      tmp[k].J = (ps.W + fused::kTW - 1) / fused::kTW;
      tmp[k].nb = nb_of(c.pass_ids[k]);
    }
    c.tt = build_tables(tmp.data(), (int)tmp.size(), c.sh.order >= 1, c.Dshape);   // orders 1 and 2: one merged launch
    c.off_down = o; o = align_up(o + tmp.size() * sizeof(fused::PassDesc), 256);
    c.off_up = o; o = align_up(o + tmp.size() * sizeof(fused::PassDesc), 256);
    c.off_tab = o; o = align_up(o + c.tt.ints.size() * sizeof(int), 256);
  }
  b.table_bytes = o;
  return b;
}

// Host image of the tables region for a plan placed in workspace ws.
std::vector<uint8_t> batch_tables(const BatchSetup& b, const FusedPlan& plan, uint8_t* ws,
                                  const sf_sgm_params* p, const sf_batch_item* items) {
  std::vector<uint8_t> blob(b.table_bytes, 0);
  for (const BatchClass& c : b.classes) {
    fused::PassDesc* dn = reinterpret_cast<fused::PassDesc*>(blob.data() + c.off_down);
    fused::PassDesc* up = reinterpret_cast<fused::PassDesc*>(blob.data() + c.off_up);
    for (size_t k = 0; k < c.pass_ids.size(); k++) {
      const int id = c.pass_ids[k], pair = id / 2, r = id % 2;
      const PairShape& ps = b.pairs[pair];
      dn[k] = pass_desc(ws, plan, plan.pairs[pair], r, ps.W, ps.H, ps.D, ps.D, nullptr);
      dn[k].dint = nullptr;
      if (p->adaptive_p2) {
        // pair 2 i + f of item i: frame t (f = 0) or t+1; pass r: reference image
        const sf_batch_item& it = items[pair / 2];
        const bool t1 = (pair & 1) != 0;
        dn[k].guide = r == 0 ? (t1 ? it.left_t1 : it.left_t) : (t1 ? it.right_t1 : it.right_t);
        dn[k].gpitch = it.pitch;
      }
      up[k] = dn[k];
      up[k].dint = reinterpret_cast<int16_t*>(ws + plan.pairs[pair].pass[r].dint);
      up[k].dsub = r == 0 ? reinterpret_cast<float*>(ws + plan.pairs[pair].dsub) : nullptr;
    }
    memcpy(blob.data() + c.off_tab, c.tt.ints.data(), c.tt.ints.size() * sizeof(int));
  }
  return blob;
}

// Everything after the table upload: costs, sweeps, checks, combination.
// ws: the wave's buffers (control block first); tab: its descriptor tables.
// The error word is cleared by the first wave only, so a bounded wait that
// gave up in any wave stays recorded.
sf_status batch_enqueue(const sf_batch_item* items, int n, const sf_sgm_params* p, const BatchSetup& b,
                        const FusedPlan& plan, uint8_t* ws, uint8_t* tab, bool first_wave, cudaStream_t s) {
  if (first_wave)
    SF_TRY_CUDA(cudaMemsetAsync(ws, 0, plan.control_bytes, s));
  else
    SF_TRY_CUDA(cudaMemsetAsync(ws + plan.counters, 0, plan.control_bytes - plan.counters, s));
  for (int i = 0; i < n; i++) {
    const sf_batch_item& it = items[i];
    const uint8_t* L[2] = {it.left_t, it.left_t1};
    const uint8_t* R[2] = {it.right_t, it.right_t1};
    const PairBuffers* bufs[2] = {&plan.pairs[2 * i], &plan.pairs[2 * i + 1]};
    sf_status st = run_pair_costs(L, R, 2, it.W, it.H, it.pitch, it.D, p, ws, bufs, s);
    if (st != SF_OK) return st;
  }
  int* counters = reinterpret_cast<int*>(ws + plan.counters);
  for (size_t c = 0; c < b.classes.size(); c++) {
    const BatchClass& bc = b.classes[c];
    sf_status st = run_sweeps(p, nullptr, (int)bc.pass_ids.size(), bc.Dshape,
                              reinterpret_cast<const fused::PassDesc*>(tab + bc.off_down),
                              reinterpret_cast<const fused::PassDesc*>(tab + bc.off_up),
                              reinterpret_cast<const int*>(tab + bc.off_tab), &bc.tt, counters + 2 * c,
                              reinterpret_cast<int*>(ws + plan.err), s);
    if (st != SF_OK) return st;
  }
  // per item: both checks and the combination in one launch
  for (int i = 0; i < n; i++) {
    const sf_batch_item& it = items[i];
    const PairBuffers& p0 = plan.pairs[2 * i];
    const PairBuffers& p1 = plan.pairs[2 * i + 1];
    CheckCombineArgs ca{};
    ca.dL0 = reinterpret_cast<const int16_t*>(ws + p0.pass[0].dint);
    ca.dR0 = reinterpret_cast<const int16_t*>(ws + p0.pass[1].dint);
    ca.dsub0 = reinterpret_cast<const float*>(ws + p0.dsub);
    ca.dL1 = reinterpret_cast<const int16_t*>(ws + p1.pass[0].dint);
    ca.dR1 = reinterpret_cast<const int16_t*>(ws + p1.pass[1].dint);
    ca.dsub1 = reinterpret_cast<const float*>(ws + p1.dsub);
    ca.flow = reinterpret_cast<const float2*>(it.flow);
    ca.W = it.W; ca.H = it.H; ca.tol = p->lr_tol;
    ca.f = it.cam.f; ca.B = it.cam.B; ca.cx = it.cam.cx; ca.cy = it.cam.cy;
    ca.D0 = it.D0_out ? it.D0_out : reinterpret_cast<float*>(ws + p0.disp);
    ca.D1 = it.D1_out ? it.D1_out : reinterpret_cast<float*>(ws + p1.disp);
    ca.s4 = reinterpret_cast<float4*>(it.s4_out);
    ca.motion = it.motion_out; ca.point = it.point_out; ca.valid = it.valid_out;
    SF_TRY_CUDA(launch_check_combine(ca, s));
  }
  return SF_OK;
}

// ---- batch waves: items in consecutive groups whose buffers fit a limit,
// one after another over one shared region (process-wide limit, 0 = one
// wave).  Workspace: every wave's descriptor tables, then the region.
std::atomic<size_t> g_batch_wave_bytes{0};

struct BatchWave {
  int start = 0, count = 0;
  BatchSetup b;
  FusedPlan plan;
  size_t tab_off = 0;
  BatchWave(const sf_batch_item* items, int s0, int n, const sf_sgm_params* p)
      : start(s0), count(n), b(batch_setup(items + s0, n, p)),
        plan(b.pairs.data(), (int)b.pairs.size(), b.dshape.data(), 2 * (int)b.classes.size(), 0) {}
};

struct BatchLayout {
  std::vector<BatchWave> waves;
  size_t region = 0, region_off = 0, total = 0;
  sf_status status = SF_OK;
  BatchLayout(const sf_batch_item* items, int n, const sf_sgm_params* p) {
    const BatchSetup all = batch_setup(items, n, p);
    if ((status = all.status) != SF_OK) return;
    const size_t limit = g_batch_wave_bytes.load(std::memory_order_relaxed);
    int i = 0;
    while (i < n) {
      int k = 1;   // at least one item per wave
      while (limit && i + k < n && BatchWave(items, i, k + 1, p).plan.total <= limit) k++;
      if (!limit) k = n - i;
      waves.emplace_back(items, i, k, p);
      i += k;
    }
    size_t o = 0;
    for (BatchWave& w : waves) {
      w.tab_off = o;
      o = align_up(o + w.b.table_bytes, 256);
      region = std::max(region, w.plan.total);
    }
    region_off = o;
    total = o + region;
  }
};

struct GraphEntry {
  std::vector<uint8_t> key;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

std::vector<uint8_t> batch_key(const sf_batch_item* items, int n, const sf_sgm_params* p, void* ws,
                               size_t ws_bytes, void* stream) {
  std::vector<uint8_t> k;
  auto put = [&](const void* v, size_t nb) {
    const uint8_t* c = (const uint8_t*)v;
    k.insert(k.end(), c, c + nb);
  };
  put(&n, sizeof(n));
  put(items, sizeof(sf_batch_item) * (size_t)n);
  put(p, sizeof(*p));
  put(&ws, sizeof(ws));
  put(&ws_bytes, sizeof(ws_bytes));
  put(&stream, sizeof(stream));
  for (const auto& pi : b_shape_keys()) put(&pi, sizeof(pi));
  const size_t wave = g_batch_wave_bytes.load(std::memory_order_relaxed);
  put(&wave, sizeof(wave));
  return k;
}

size_t workspace_bytes(int W, int H, const sf_sgm_params* p, int npairs) {
  if (fused_eligible(W, H, p)) return std::max(single_plan(W, H, p->D, npairs).total, Workspace(W, H, p->D).total);
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
  p->adaptive_p2 = 0;
  p->uniqueness = 0;
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
  return single_plan(W, H, p->D, 1).total;
}

}  // extern "C"

namespace {

// sf_sgm_aggregate(_guided): guide is the reference image for the adaptive
// P2 (nullptr with constant P2).
sf_status aggregate_impl(const uint8_t* cost, const uint8_t* guide, int gpitch, int32_t W, int32_t H,
                         const sf_sgm_params* p, uint16_t* agg_out, void* workspace, size_t ws_bytes,
                         cudaStream_t s) {
  // fused sweeps when the volume is 16-disparity aligned and a workspace of
  // sf_aggregate_workspace_size() bytes is given; staged kernels otherwise
  if (g_use_fused && p->D % 16 == 0 && aligned(cost, 16) && workspace && aligned(workspace, 256) &&
      ws_bytes >= single_plan(W, H, p->D, 1).total) {
    FusedPlan plan = single_plan(W, H, p->D, 1);
    uint8_t* ws = (uint8_t*)workspace;
    SF_TRY_CUDA(cudaMemsetAsync(ws, 0, plan.control_bytes, s));
    fused::PassDesc d = pass_desc(ws, plan, plan.pairs[0], 0, W, H, p->D, p->D, cost);
    d.dint = nullptr;
    d.S = agg_out;
    d.guide = guide;
    d.gpitch = gpitch;
    return run_sweeps(p, &d, 1, p->D, nullptr, nullptr, nullptr, nullptr,
                      reinterpret_cast<int*>(ws + plan.counters), reinterpret_cast<int*>(ws + plan.err), s);
  }
  SF_TRY_CUDA(launch_aggregate(cost, W, H, p->D, p->P1, p->P2, p->path_mask, agg_out, s, guide, gpitch));
  return SF_OK;
}

}  // namespace

extern "C" {

sf_status sf_sgm_aggregate(const uint8_t* cost, int32_t W, int32_t H, const sf_sgm_params* p,
                           uint16_t* agg_out, void* workspace, size_t ws_bytes, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!cost || !agg_out) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (p->adaptive_p2) return SF_ERR_INVALID_ARG;   // needs the guide: sf_sgm_aggregate_guided
  if (!aligned(agg_out, 2)) return SF_ERR_INVALID_ARG;
  return aggregate_impl(cost, nullptr, 0, W, H, p, agg_out, workspace, ws_bytes, (cudaStream_t)stream);
}

sf_status sf_sgm_aggregate_guided(const uint8_t* cost, const uint8_t* guide, int32_t pitch, int32_t W,
                                  int32_t H, const sf_sgm_params* p, uint16_t* agg_out, void* workspace,
                                  size_t ws_bytes, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!cost || !agg_out || !guide || pitch < W) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (!aligned(agg_out, 2)) return SF_ERR_INVALID_ARG;
  return aggregate_impl(cost, p->adaptive_p2 ? guide : nullptr, pitch, W, H, p, agg_out, workspace, ws_bytes,
                        (cudaStream_t)stream);
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

sf_status sf_fill_disparity(const float* in, int32_t W, int32_t H, const uint8_t* guide, int32_t pitch,
                            int32_t mode, float* out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!in || !out || in == out) return SF_ERR_INVALID_ARG;
  if (mode != SF_FILL_BACKGROUND && mode != SF_FILL_EDGE_AWARE) return SF_ERR_INVALID_ARG;
  if (mode == SF_FILL_EDGE_AWARE && (!guide || pitch < W)) return SF_ERR_INVALID_ARG;
  if (!aligned(in, 4) || !aligned(out, 4)) return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_fill_map(in, W, H, mode == SF_FILL_EDGE_AWARE ? guide : nullptr, pitch, mode, out,
                              (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_densify_sceneflow(const float* s4_in, const float* flow, int32_t W, int32_t H, const sf_camera* cam,
                               const uint8_t* guide, int32_t pitch, int32_t mode, float* s4_out,
                               float* motion_out, float* point_out, uint8_t* valid_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!s4_in || !flow || !cam || !s4_out || !valid_out || s4_in == s4_out) return SF_ERR_INVALID_ARG;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  if (mode != SF_FILL_BACKGROUND && mode != SF_FILL_EDGE_AWARE) return SF_ERR_INVALID_ARG;
  if (mode == SF_FILL_EDGE_AWARE && (!guide || pitch < W)) return SF_ERR_INVALID_ARG;
  if (!aligned(s4_in, 16) || !aligned(s4_out, 16) || !aligned(flow, 8) || !aligned(motion_out, 4) ||
      !aligned(point_out, 4))
    return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_densify(s4_in, flow, W, H, cam->f, cam->B, cam->cx, cam->cy,
                             mode == SF_FILL_EDGE_AWARE ? guide : nullptr, pitch, mode, s4_out, motion_out,
                             point_out, valid_out, (cudaStream_t)stream));
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
    FusedPlan fl = single_plan(W, H, p->D, 2);
    D0 = D0_out ? D0_out : reinterpret_cast<float*>(ws + fl.pairs[0].disp);
    D1 = D1_out ? D1_out : reinterpret_cast<float*>(ws + fl.pairs[1].disp);
    const uint8_t* L[2] = {left_t, left_t1};
    const uint8_t* R[2] = {right_t, right_t1};
    float* disp[2] = {D0, D1};
    fused::PassDesc d[4];
    if ((st = run_fused_pairs(L, R, 2, W, H, pitch, p, nullptr, nullptr, nullptr, disp, ws, s, d)) != SF_OK)
      return st;
    // both checks and the combination in one launch
    CheckCombineArgs ca{};
    ca.dL0 = d[0].dint; ca.dR0 = d[1].dint; ca.dsub0 = d[0].dsub;
    ca.dL1 = d[2].dint; ca.dR1 = d[3].dint; ca.dsub1 = d[2].dsub;
    ca.flow = reinterpret_cast<const float2*>(flow);
    ca.W = W; ca.H = H; ca.tol = p->lr_tol;
    ca.f = cam->f; ca.B = cam->B; ca.cx = cam->cx; ca.cy = cam->cy;
    ca.D0 = D0; ca.D1 = D1;
    ca.s4 = reinterpret_cast<float4*>(s4_out);
    ca.motion = motion_out; ca.point = point_out; ca.valid = valid_out;
    SF_TRY_CUDA(launch_check_combine(ca, s));
    return SF_OK;
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

sf_status sf_debug_set(int32_t key, int64_t value) {
  if (key == SF_DEBUG_SPIN_LIMIT) {
    if (value < 0) return SF_ERR_INVALID_ARG;
    g_spin_limit.store(value == 0 ? kSpinLimit : value, std::memory_order_relaxed);
    return SF_OK;
  }
  if (key == SF_DEBUG_SKIP_TASKS) {
    if (value < 0 || value > (1 << 30)) return SF_ERR_INVALID_ARG;
    g_skip_down_tasks.store((int)value, std::memory_order_relaxed);
    return SF_OK;
  }
  if (key == SF_DEBUG_HLINE_DC) {
    return fused::set_hline_dc(value == 0 ? 4 : (int)value) == 0 ? SF_OK : SF_ERR_INVALID_ARG;
  }
  return SF_ERR_INVALID_ARG;
}

size_t sf_batch_workspace_size(const sf_batch_item* items, int32_t n, const sf_sgm_params* p) {
  const BatchLayout lay(items, n, p);
  return lay.status == SF_OK ? lay.total : 0;
}

sf_status sf_set_batch_wave_limit(size_t bytes) {
  g_batch_wave_bytes.store(bytes, std::memory_order_relaxed);
  return SF_OK;
}

sf_status sf_batch_run(const sf_batch_item* items, int32_t n, const sf_sgm_params* p, uint32_t flags,
                       void* workspace, size_t ws_bytes, void* stream) {
  const BatchLayout lay(items, n, p);
  if (lay.status != SF_OK) return lay.status;
  if (flags & ~SF_BATCH_GRAPH) return SF_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < lay.total || !aligned(workspace, 256)) return SF_ERR_INVALID_ARG;
  uint8_t* ws = (uint8_t*)workspace;
  uint8_t* region = ws + lay.region_off;
  cudaStream_t s = (cudaStream_t)stream;
  // every wave's descriptor tables travel before the work (pageable source:
  // the copy has read it when the call returns)
  for (const BatchWave& w : lay.waves) {
    std::vector<uint8_t> blob = batch_tables(w.b, w.plan, region, p, items + w.start);
    SF_TRY_CUDA(cudaMemcpyAsync(ws + w.tab_off, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
  }
  auto enqueue = [&]() -> sf_status {
    for (size_t i = 0; i < lay.waves.size(); i++) {
      const BatchWave& w = lay.waves[i];
      sf_status st = batch_enqueue(items + w.start, w.count, p, w.b, w.plan, region, ws + w.tab_off, i == 0, s);
      if (st != SF_OK) return st;
    }
    return SF_OK;
  };
  if (!(flags & SF_BATCH_GRAPH)) return enqueue();
  if (s == nullptr) return SF_ERR_INVALID_ARG;   // the legacy default stream cannot be captured
  std::vector<uint8_t> key = batch_key(items, n, p, workspace, ws_bytes, stream);
  std::lock_guard<std::mutex> guard(g_graph_mu);
  for (GraphEntry& g : g_graphs) {
    if (g.key == key) {
      SF_TRY_CUDA(cudaGraphLaunch(g.exec, s));
      return SF_OK;
    }
  }
  SF_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  sf_status st = enqueue();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st != SF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SF_ERR_CUDA;
  }
  GraphEntry g;
  g.key = key;
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SF_ERR_CUDA;
  }
  g_graphs.push_back(g);
  SF_TRY_CUDA(cudaGraphLaunch(g_graphs.back().exec, s));
  return SF_OK;
}

void sf_batch_release_graphs(void) {
  std::lock_guard<std::mutex> guard(g_graph_mu);
  for (GraphEntry& g : g_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  g_graphs.clear();
}

sf_status sf_set_sweep_shape(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo) {
  return fused::set_shape_override(fused::kShapePlain, d_lo, d_hi, dc, halo, 0) == 0 ? SF_OK : SF_ERR_UNSUPPORTED;
}

sf_status sf_set_sweep_schedule(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo, int32_t order) {
  return fused::set_shape_override(fused::kShapePlain, d_lo, d_hi, dc, halo, order) == 0 ? SF_OK
                                                                                           : SF_ERR_UNSUPPORTED;
}

sf_status sf_set_learned_sweep_schedule(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo, int32_t order) {
  return fused::set_shape_override(fused::kShapeLearned, d_lo, d_hi, dc, halo, order) == 0 ? SF_OK
                                                                                             : SF_ERR_UNSUPPORTED;
}

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
  FusedPlan lay = single_plan(W, H, p->D, npairs);
  int err = 0;
  cudaStream_t s = (cudaStream_t)stream;
  SF_TRY_CUDA(cudaMemcpyAsync(&err, (const uint8_t*)workspace + lay.err, sizeof(int),
                              cudaMemcpyDeviceToHost, s));
  SF_TRY_CUDA(cudaStreamSynchronize(s));
  return err ? SF_ERR_TIMEOUT : SF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Aggregation without a caller-provided workspace.
//
// For callers that cannot allocate device memory: a host program that owns no
// device allocator (no PyTorch, no pool), or a latency-bound loop that must
// not call cudaMalloc/cudaFree (they can synchronise the device and take
// locks).  The band sweeps' scratch then lives in this file-scope array, one
// copy per device, reserved when the library's device code is loaded.
// ---------------------------------------------------------------------------
static __device__ __align__(256) uint8_t g_noalloc_scratch[SF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device.  Outside stream
// capture it is looked up on every call (cheap once the module is loaded), so
// an address that moved with a device or context reset is never reused; under
// capture the address of the last uncaptured call on this device serves (the
// first lookup may load the module's device code, which capture forbids).
sf_status noalloc_scratch(cudaStream_t s, uint8_t** out) {
  int dev = -1;
  SF_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return SF_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SF_TRY_CUDA(cudaStreamIsCapturing(s, &cap));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (rc != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return SF_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<uint8_t*>(g_noalloc_ptr[dev]);
  return SF_OK;
}

}  // namespace

// Scratch of one aggregation pass: control words (error word, the two sweep
// task counters, the strip flags of both sweeps), then the two horizontal
// path volumes, the down-sweep partial sum and the band-end states.
struct NoallocLayout {
  size_t err = 0, counters = 0, flags = 0, control_bytes = 0, hf = 0, hb = 0, sdown = 0, bs = 0,
         total = 0;
  NoallocLayout(int W, int H, int D) {
    const size_t N = (size_t)W * H;
    const int J = (W + fused::kTW - 1) / fused::kTW;
    const int Dp = fused::padded_d(D);
    size_t c = 0;
    err = c; c += sizeof(int);
    counters = c; c += 2 * sizeof(int);
    flags = c; c += (size_t)(2 * J + flags_h_count(H)) * sizeof(int);
    control_bytes = align_up(c, 256);
    size_t o = control_bytes;
    hf = o; o = align_up(o + N * Dp, 256);
    hb = o; o = align_up(o + N * Dp, 256);
    sdown = o; o = align_up(o + fused::sdown_bytes(W, H, D), 256);
    bs = o; o = align_up(o + fused::bs_bytes(W, D), 256);
    total = o;
  }
};

extern "C" sf_status sf_sgm_aggregate_noalloc(const uint8_t* cost, int32_t W, int32_t H,
                                              const sf_sgm_params* p, uint16_t* agg_out,
                                              int32_t* err_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!cost || !agg_out) return SF_ERR_INVALID_ARG;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (p->adaptive_p2) return SF_ERR_INVALID_ARG;   // no guide image here
  if (p->D % 16 != 0) return SF_ERR_UNSUPPORTED;
  if (!aligned(cost, 16) || !aligned(agg_out, 2) || !aligned(err_out, 4)) return SF_ERR_INVALID_ARG;
  const NoallocLayout lay(W, H, p->D);
  if (lay.total > (size_t)SF_NOALLOC_SCRATCH_BYTES) return SF_ERR_UNSUPPORTED;
  uint8_t* ws = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = noalloc_scratch(s, &ws)) != SF_OK) return st;
  // the control words start every call at zero; the rest of the scratch is
  // fully written before it is read
  SF_TRY_CUDA(cudaMemsetAsync(ws, 0, lay.control_bytes, s));
  fused::PassDesc d{};
  d.W = W; d.H = H; d.D = p->D; d.Dp = fused::padded_d(p->D);
  d.J = (W + fused::kTW - 1) / fused::kTW;
  d.nb = (H + fused::band_rows(p->D) - 1) / fused::band_rows(p->D);
  d.cost = cost;
  d.hfwd = ws + lay.hf;
  d.hbwd = ws + lay.hb;
  d.sdown = reinterpret_cast<uint32_t*>(ws + lay.sdown);
  d.bs = ws + lay.bs;
  d.flags_down = reinterpret_cast<int*>(ws + lay.flags);
  d.flags_up = d.flags_down + d.J;
  d.flags_h = d.flags_up + d.J;
  d.dint = nullptr;
  d.dsub = nullptr;
  d.S = agg_out;
  d.guide = nullptr;
  d.gpitch = 0;
  st = run_sweeps(p, &d, 1, p->D, nullptr, nullptr, nullptr, nullptr,
                  reinterpret_cast<int*>(ws + lay.counters), reinterpret_cast<int*>(ws + lay.err), s);
  if (st != SF_OK) return st;
  if (err_out)
    SF_TRY_CUDA(cudaMemcpyAsync(err_out, ws + lay.err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return SF_OK;
}

// ---------------------------------------------------------------------------
// Learned confidence: the left pass, its features, the network.
// ---------------------------------------------------------------------------
namespace {

struct LearnedPair {
  size_t census_l = 0, census_r = 0, cost = 0, hf = 0, hb = 0, sdown = 0, bs = 0, S = 0, feat = 0,
         dint = 0, dsub = 0, disp = 0, flags = 0;
};

// Shape table of a learned launch of npairs left passes: the learned table
// for one frame's two passes, the plain calls' (tuned on four passes) for
// more.
inline int learned_table(int npairs) { return npairs <= 2 ? fused::kShapeLearned : fused::kShapePlain; }

struct LearnedPlan {
  size_t err = 0, counters = 0, control_bytes = 0, total = 0;
  LearnedPair pr[fused::kMaxPass];
  LearnedPlan(int W, int H, int D, int npairs) {
    const size_t N = (size_t)W * H;
    const int J = (W + fused::kTW - 1) / fused::kTW;
    const int Dp = fused::padded_d(D);
    size_t c = 0;
    err = c; c += sizeof(int);
    counters = c; c += 2 * sizeof(int);
    for (int k = 0; k < npairs; k++) {
      pr[k].flags = c;
      c += (size_t)(2 * J + flags_h_count(H)) * sizeof(int);
    }
    control_bytes = align_up(c, 256);
    size_t o = control_bytes;
    auto carve = [&](size_t bytes) {
      const size_t at = o;
      o = align_up(o + bytes, 256);
      return at;
    };
    for (int k = 0; k < npairs; k++) {
      LearnedPair& b = pr[k];
      b.census_l = carve(N * 8);
      b.census_r = carve(N * 8);
      b.cost = carve(N * Dp);
      b.hf = carve(N * Dp);
      b.hb = carve(N * Dp);
      // room for either table's shape (a sequence's last launch may carry
      // fewer passes than the workspace was sized for)
      b.sdown = carve(std::max(fused::sdown_bytes(W, H, D, fused::kShapeLearned),
                               fused::sdown_bytes(W, H, D, fused::kShapePlain)));
      b.bs = carve(fused::bs_bytes(W, D));
      b.S = carve(N * D * sizeof(uint16_t));
      b.feat = carve(N * 16);
      b.dint = carve(N * sizeof(int16_t));
      b.dsub = carve(N * sizeof(float));
      b.disp = carve(N * sizeof(float));
    }
    total = o;
  }
};

sf_status check_learned(int W, int H, const sf_sgm_params* p) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if ((st = check_params(p, W, H)) != SF_OK) return st;
  if (p->path_mask != 0xFFu) return SF_ERR_UNSUPPORTED;   // features use all eight paths
  // the network's acceptance rule stands in for every check of the left
  // winners, the uniqueness filter included
  if (p->uniqueness != 0) return SF_ERR_UNSUPPORTED;
  return SF_OK;
}

// Learned stereo for npairs (1 or 2) pairs of one size: both left passes
// share the sweep launches.
sf_status run_learned_pairs(int npairs, const uint8_t* const* left, const uint8_t* const* right, int W,
                            int H, int pitch, const sf_sgm_params* p, const void* packed, float threshold,
                            int16_t* const* dint_out, float* const* prob_out, uint8_t* const* valid_out,
                            float* const* disp_out, uint16_t* const* feat_out, uint8_t* ws,
                            cudaStream_t s) {
  const LearnedPlan plan(W, H, p->D, npairs);
  const int D = p->D, Dp = fused::padded_d(D);
  const int J = (W + fused::kTW - 1) / fused::kTW;
  // one frame's two left passes: the learned calls' own tuned schedule
  // (their launches carry half the work of the plain frame's four passes)
  const int table = learned_table(npairs);
  SF_TRY_CUDA(cudaMemsetAsync(ws, 0, plan.control_bytes, s));
  fused::PassDesc d[fused::kMaxPass];
  fused::CostPairs job{};
  job.npairs = npairs;
  const uint8_t* imgs[2 * fused::kMaxPass];
  uint64_t* cens[2 * fused::kMaxPass];
  for (int k = 0; k < npairs; k++) {
    const LearnedPair& b = plan.pr[k];
    uint64_t* cl = reinterpret_cast<uint64_t*>(ws + b.census_l);
    uint64_t* cr = reinterpret_cast<uint64_t*>(ws + b.census_r);
    imgs[2 * k] = left[k];
    imgs[2 * k + 1] = right[k];
    cens[2 * k] = cl;
    cens[2 * k + 1] = cr;
    job.cL[k] = cl;
    job.cR[k] = cr;
    job.CL[k] = ws + b.cost;
  }
  // every image's census in one launch
  SF_TRY_CUDA(launch_census_images(imgs, cens, 2 * npairs, W, H, pitch, p->census_w, p->census_h, s));
  // the left volumes of every pair in one launch
  SF_TRY_CUDA(fused::launch_cost_left(job, W, H, D, Dp, p->census_w * p->census_h - 1, s));
  for (int k = 0; k < npairs; k++) {
    const LearnedPair& b = plan.pr[k];
    fused::PassDesc& pd = d[k];
    pd = fused::PassDesc{};
    pd.W = W; pd.H = H; pd.D = D; pd.Dp = Dp; pd.J = J;
    pd.nb = (H + fused::band_rows(D, table) - 1) / fused::band_rows(D, table);
    pd.cost = ws + b.cost;
    pd.hfwd = ws + b.hf;
    pd.hbwd = ws + b.hb;
    pd.sdown = reinterpret_cast<uint32_t*>(ws + b.sdown);
    pd.bs = ws + b.bs;
    pd.flags_down = reinterpret_cast<int*>(ws + b.flags);
    pd.flags_up = pd.flags_down + J;
    pd.flags_h = pd.flags_up + J;
    pd.dint = nullptr;
    pd.dsub = nullptr;
    pd.S = reinterpret_cast<uint16_t*>(ws + b.S);
    pd.guide = p->adaptive_p2 ? left[k] : nullptr;
    pd.gpitch = pitch;
  }
  sf_status st = run_sweeps(p, d, npairs, D, nullptr, nullptr, nullptr, nullptr,
                            reinterpret_cast<int*>(ws + plan.counters), reinterpret_cast<int*>(ws + plan.err), s,
                            table);
  if (st != SF_OK) return st;
  const fused::Shape shape = fused::shape_for(D, table);
  static_assert(confnet::kMaxInferPass >= fused::kMaxPass, "one network launch per learned call");
  confnet::InferArgs ia{};
  for (int k = 0; k < npairs; k++) {
    const LearnedPair& b = plan.pr[k];
    confnet::FeatureArgs fa{};
    fa.W = W; fa.H = H; fa.D = D; fa.Dp = Dp; fa.J = J;
    fa.dpad_shape = shape.chunks * shape.dc;
    fa.subpixel = p->subpixel;
    fa.S = reinterpret_cast<const uint16_t*>(ws + b.S);
    fa.sdown = reinterpret_cast<const uint32_t*>(ws + b.sdown);
    fa.hfwd = ws + b.hf;
    fa.hbwd = ws + b.hb;
    fa.cost = ws + b.cost;
    fa.feat = feat_out && feat_out[k] ? feat_out[k] : reinterpret_cast<uint16_t*>(ws + b.feat);
    fa.dint = dint_out && dint_out[k] ? dint_out[k] : reinterpret_cast<int16_t*>(ws + b.dint);
    fa.dsub = reinterpret_cast<float*>(ws + b.dsub);
    {
      StageTrace trace(SF_STAGE_FEATURES, s);
      SF_TRY_CUDA(confnet::launch_features(fa, s));
    }
    confnet::InferPass& ip = ia.pass[k];
    ip.feat = fa.feat;
    ip.dint = fa.dint;
    ip.dsub = fa.dsub;
    ip.prob = prob_out ? prob_out[k] : nullptr;
    ip.valid = valid_out ? valid_out[k] : nullptr;
    ip.disp = disp_out ? disp_out[k] : nullptr;
  }
  if (packed) {
    // one network launch over the tiles of every pair
    ia.W = W; ia.H = H; ia.npass = npairs;
    ia.packed = packed;
    ia.threshold = threshold;
    ia.err = reinterpret_cast<int*>(ws + plan.err);
    StageTrace trace(SF_STAGE_CONFNET, s);
    SF_TRY_CUDA(confnet::launch_infer(ia, s));
  }
  return SF_OK;
}

bool hparams_ok(const sf_confnet_hparams* hp) {
  return hp && hp->step >= 1 && hp->lr >= 0.0f && hp->beta1 >= 0.0f && hp->beta1 < 1.0f &&
         hp->beta2 >= 0.0f && hp->beta2 < 1.0f && hp->eps > 0.0f && hp->w_neg >= 0.0f;
}

}  // namespace

extern "C" {

int32_t sf_confnet_param_count(void) { return confnet::kParamCount; }

size_t sf_confnet_packed_bytes(void) { return confnet::kPackedBytes; }

sf_status sf_confnet_pack(const float* params, void* packed, void* stream) {
  if (!params || !packed || !aligned(packed, 16) || !aligned(params, 4)) return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(confnet::launch_pack(params, packed, (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_confnet_infer(const void* packed, const uint16_t* features, const int16_t* dint,
                           const float* dsub, int32_t W, int32_t H, float threshold, float* prob_out,
                           uint8_t* valid_out, float* disp_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!packed || !features || !aligned(packed, 16) || !aligned(features, 16)) return SF_ERR_INVALID_ARG;
  if ((valid_out || disp_out) && (!dint || !dsub)) return SF_ERR_INVALID_ARG;
  if (!aligned(dint, 2) || !aligned(dsub, 4) || !aligned(prob_out, 4) || !aligned(disp_out, 4))
    return SF_ERR_INVALID_ARG;
  confnet::InferArgs ia{};
  ia.W = W; ia.H = H; ia.npass = 1;
  ia.packed = packed;
  ia.pass[0].feat = features;
  ia.pass[0].dint = dint;
  ia.pass[0].dsub = dsub;
  ia.pass[0].prob = prob_out;
  ia.pass[0].valid = valid_out;
  ia.pass[0].disp = disp_out;
  ia.threshold = threshold;
  ia.err = nullptr;
  SF_TRY_CUDA(confnet::launch_infer(ia, (cudaStream_t)stream));
  return SF_OK;
}

size_t sf_confnet_train_workspace_size(int32_t B, int32_t W, int32_t H) {
  if (B < 1 || W < 1 || H < 1 || (size_t)B * W * H > (size_t)1 << 26) return 0;
  return confnet::train_workspace_bytes(B, W, H);
}

sf_status sf_confnet_train_step(float* params, float* adam_m, float* adam_v, const uint16_t* features,
                                const uint8_t* labels, int32_t B, int32_t W, int32_t H,
                                const sf_confnet_hparams* hp, float* grad_out, float* loss_out,
                                float* logits_out, void* workspace, size_t ws_bytes, void* stream) {
  if (B < 1 || W < 1 || H < 1 || (size_t)B * W * H > (size_t)1 << 26) return SF_ERR_INVALID_ARG;
  if (!params || !features || !workspace || !hparams_ok(hp)) return SF_ERR_INVALID_ARG;
  if (ws_bytes < confnet::train_workspace_bytes(B, W, H) || !aligned(workspace, 256)) return SF_ERR_INVALID_ARG;
  if (!aligned(params, 4) || !aligned(features, 16) || !aligned(grad_out, 4) || !aligned(loss_out, 4) ||
      !aligned(logits_out, 4) || !aligned(adam_m, 4) || !aligned(adam_v, 4))
    return SF_ERR_INVALID_ARG;
  confnet::TrainArgs t{};
  t.B = B; t.W = W; t.H = H;
  t.params = params;
  t.adam_m = labels ? adam_m : nullptr;
  t.adam_v = labels ? adam_v : nullptr;
  t.features = features;
  t.labels = labels;
  t.lr = hp->lr; t.beta1 = hp->beta1; t.beta2 = hp->beta2; t.eps = hp->eps; t.w_neg = hp->w_neg;
  t.step = hp->step;
  t.grad_out = grad_out;
  t.loss_out = loss_out;
  t.logits_out = logits_out;
  t.workspace = workspace;
  SF_TRY_CUDA(confnet::launch_train_step(t, (cudaStream_t)stream));
  return SF_OK;
}

sf_status sf_confnet_adam(float* params, float* adam_m, float* adam_v, const float* grad,
                          const sf_confnet_hparams* hp, void* stream) {
  if (!params || !adam_m || !adam_v || !grad || !hparams_ok(hp)) return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(confnet::launch_adam(params, adam_m, adam_v, grad, confnet::kParamCount, hp->lr, hp->beta1,
                                   hp->beta2, hp->eps, hp->step, (cudaStream_t)stream));
  return SF_OK;
}

size_t sf_learned_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p, int32_t npairs) {
  if (check_size(W, H) != SF_OK || !p || p->D < 1 || p->D > SF_MAX_DISPARITY) return 0;
  if (npairs < 1 || npairs > fused::kMaxPass) return 0;
  return LearnedPlan(W, H, p->D, npairs).total;
}

sf_status sf_sgm_learned(const uint8_t* left, const uint8_t* right, int32_t W, int32_t H,
                         int32_t pitch, const sf_sgm_params* p, const void* packed, float threshold,
                         int16_t* dint_out, float* prob_out, uint8_t* valid_out, float* disp_out,
                         uint16_t* features_out, void* workspace, size_t ws_bytes, void* stream) {
  sf_status st = check_learned(W, H, p);
  if (st != SF_OK) return st;
  if (!left || !right || !workspace || pitch < W) return SF_ERR_INVALID_ARG;
  if (ws_bytes < LearnedPlan(W, H, p->D, 1).total || !aligned(workspace, 256)) return SF_ERR_INVALID_ARG;
  if (!aligned(packed, 16) || !aligned(features_out, 16) || !aligned(dint_out, 2) || !aligned(prob_out, 4) ||
      !aligned(disp_out, 4))
    return SF_ERR_INVALID_ARG;
  return run_learned_pairs(1, &left, &right, W, H, pitch, p, packed, threshold, &dint_out, &prob_out,
                           &valid_out, &disp_out, &features_out, (uint8_t*)workspace, (cudaStream_t)stream);
}

sf_status sf_scene_flow_learned_frames(const sf_learned_frame* frames, int32_t n, int32_t pitch, int32_t W,
                                       int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                                       const void* packed, float threshold, void* workspace, size_t ws_bytes,
                                       void* stream) {
  sf_status st = check_learned(W, H, p);
  if (st != SF_OK) return st;
  if (!frames || n < 1 || 2 * n > fused::kMaxPass) return SF_ERR_INVALID_ARG;
  if (!cam || !packed || !workspace || pitch < W) return SF_ERR_INVALID_ARG;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  for (int i = 0; i < n; i++) {
    const sf_learned_frame& f = frames[i];
    if (!f.left_t || !f.right_t || !f.left_t1 || !f.right_t1 || !f.flow || !f.s4_out || !f.valid_out)
      return SF_ERR_INVALID_ARG;
    if (!aligned(f.flow, 8) || !aligned(f.s4_out, 16) || !aligned(f.motion_out, 4) ||
        !aligned(f.point_out, 4) || !aligned(f.D0_out, 4) || !aligned(f.D1_out, 4))
      return SF_ERR_INVALID_ARG;
  }
  const LearnedPlan plan(W, H, p->D, 2 * n);
  if (ws_bytes < plan.total || !aligned(workspace, 256) || !aligned(packed, 16)) return SF_ERR_INVALID_ARG;
  uint8_t* ws = (uint8_t*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  const uint8_t* L[fused::kMaxPass];
  const uint8_t* R[fused::kMaxPass];
  float* disp[fused::kMaxPass];
  for (int i = 0; i < n; i++) {
    const sf_learned_frame& f = frames[i];
    L[2 * i] = f.left_t;
    R[2 * i] = f.right_t;
    L[2 * i + 1] = f.left_t1;
    R[2 * i + 1] = f.right_t1;
    disp[2 * i] = f.D0_out ? f.D0_out : reinterpret_cast<float*>(ws + plan.pr[2 * i].disp);
    disp[2 * i + 1] = f.D1_out ? f.D1_out : reinterpret_cast<float*>(ws + plan.pr[2 * i + 1].disp);
  }
  if ((st = run_learned_pairs(2 * n, L, R, W, H, pitch, p, packed, threshold, nullptr, nullptr, nullptr, disp,
                              nullptr, ws, s)) != SF_OK)
    return st;
  for (int i = 0; i < n; i++) {
    const sf_learned_frame& f = frames[i];
    SF_TRY_CUDA(launch_combine(disp[2 * i], disp[2 * i + 1], f.flow, W, H, cam->f, cam->B, cam->cx, cam->cy,
                               f.s4_out, f.motion_out, f.point_out, f.valid_out, s));
  }
  return SF_OK;
}

// ---- sequences of more than two frames ---------------------------------------
// Workspace: the stereo work of one group of frames (two pairs with the
// plain check, four left passes with the learned confidence), reused group
// after group in stream order, then the K disparity maps.
}  // extern "C"

namespace {

struct SequencePlan {
  size_t stereo = 0, disp = 0, total = 0;
  int group = 1;
  SequencePlan(int W, int H, const sf_sgm_params* p, int K, bool learned) {
    const size_t N = (size_t)W * H;
    group = learned ? fused::kMaxPass : 2;
    stereo = learned ? LearnedPlan(W, H, p->D, group).total : workspace_bytes(W, H, p, 2);
    size_t o = align_up(stereo, 256);
    disp = o;
    o += (size_t)K * align_up(N * sizeof(float), 256);
    total = o;
  }
  float* disp_map(uint8_t* ws, int k, int W, int H) const {
    return reinterpret_cast<float*>(ws + disp + (size_t)k * align_up((size_t)W * H * sizeof(float), 256));
  }
};

}  // namespace

extern "C" {

sf_status sf_chain_sceneflow(const float* const* disps, const float* const* flows, int32_t K, int32_t W,
                             int32_t H, const sf_camera* cam, float* points_out, uint8_t* valid_out, void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!disps || !flows || !cam || K < 2 || K > SF_MAX_FRAMES) return SF_ERR_INVALID_ARG;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  if (!points_out && !valid_out) return SF_ERR_INVALID_ARG;
  for (int k = 0; k < K; k++)
    if (!disps[k] || !aligned(disps[k], 4)) return SF_ERR_INVALID_ARG;
  for (int k = 0; k + 1 < K; k++)
    if (!flows[k] || !aligned(flows[k], 8)) return SF_ERR_INVALID_ARG;
  if (!aligned(points_out, 4)) return SF_ERR_INVALID_ARG;
  SF_TRY_CUDA(launch_chain(disps, flows, K, W, H, cam->f, cam->B, cam->cx, cam->cy, points_out, valid_out,
                           (cudaStream_t)stream));
  return SF_OK;
}

size_t sf_sequence_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p, int32_t K, int32_t learned) {
  if (check_size(W, H) != SF_OK || !p || p->D < 1 || p->D > SF_MAX_DISPARITY) return 0;
  if (K < 2 || K > SF_MAX_FRAMES || (learned != 0 && learned != 1)) return 0;
  return SequencePlan(W, H, p, K, learned != 0).total;
}

sf_status sf_sequence_sceneflow(const uint8_t* const* left, const uint8_t* const* right, int32_t K, int32_t pitch,
                                const float* const* flows, int32_t W, int32_t H, const sf_sgm_params* p,
                                const sf_camera* cam, const void* packed, float threshold, float* const* disp_out,
                                float* const* s4_out, uint8_t* const* valid_out, float* const* motion_out,
                                float* points_out, uint8_t* chain_valid_out, void* workspace, size_t ws_bytes,
                                void* stream) {
  sf_status st = check_size(W, H);
  if (st != SF_OK) return st;
  if (!left || !right || !flows || !cam || !workspace || pitch < W || K < 2 || K > SF_MAX_FRAMES)
    return SF_ERR_INVALID_ARG;
  const bool learned = packed != nullptr;
  if ((st = learned ? check_learned(W, H, p) : check_params(p, W, H)) != SF_OK) return st;
  if (!(cam->f > 0.0f) || !(cam->B > 0.0f)) return SF_ERR_INVALID_ARG;
  if ((s4_out == nullptr) != (valid_out == nullptr)) return SF_ERR_INVALID_ARG;
  for (int k = 0; k < K; k++) {
    if (!left[k] || !right[k]) return SF_ERR_INVALID_ARG;
    if (disp_out && (!disp_out[k] || !aligned(disp_out[k], 4))) return SF_ERR_INVALID_ARG;
  }
  for (int k = 0; k + 1 < K; k++) {
    if (!flows[k] || !aligned(flows[k], 8)) return SF_ERR_INVALID_ARG;
    if (s4_out && (!s4_out[k] || !valid_out[k] || !aligned(s4_out[k], 16))) return SF_ERR_INVALID_ARG;
    if (motion_out && !aligned(motion_out[k], 4)) return SF_ERR_INVALID_ARG;
  }
  if ((points_out || chain_valid_out) && !aligned(points_out, 4)) return SF_ERR_INVALID_ARG;
  const SequencePlan plan(W, H, p, K, learned);
  if (ws_bytes < plan.total || !aligned(workspace, 256) || (learned && !aligned(packed, 16)))
    return SF_ERR_INVALID_ARG;
  uint8_t* ws = (uint8_t*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  float* disp[SF_MAX_FRAMES];
  for (int k = 0; k < K; k++) disp[k] = disp_out ? disp_out[k] : plan.disp_map(ws, k, W, H);
  // every stereo frame once, a group of frames per set of launches
  for (int g = 0; g < K; g += plan.group) {
    const int n = std::min(plan.group, K - g);
    if (learned) {
      st = run_learned_pairs(n, left + g, right + g, W, H, pitch, p, packed, threshold, nullptr, nullptr, nullptr,
                             disp + g, nullptr, ws, s);
    } else if (fused_eligible(W, H, p)) {
      st = run_fused_pairs(left + g, right + g, n, W, H, pitch, p, nullptr, nullptr, nullptr, disp + g, ws, s);
    } else {
      for (int k = g; k < g + n && st == SF_OK; k++)
        st = sgm_full_impl(left[k], right[k], W, H, pitch, p, nullptr, nullptr, nullptr, disp[k], ws, s);
    }
    if (st != SF_OK) return st;
  }
  if (s4_out) {
    for (int k = 0; k + 1 < K; k++)
      SF_TRY_CUDA(launch_combine(disp[k], disp[k + 1], flows[k], W, H, cam->f, cam->B, cam->cx, cam->cy, s4_out[k],
                                 motion_out ? motion_out[k] : nullptr, nullptr, valid_out[k], s));
  }
  if (points_out || chain_valid_out) {
    const float* dconst[SF_MAX_FRAMES];
    for (int k = 0; k < K; k++) dconst[k] = disp[k];
    SF_TRY_CUDA(launch_chain(dconst, flows, K, W, H, cam->f, cam->B, cam->cx, cam->cy, points_out, chain_valid_out,
                             s));
  }
  return SF_OK;
}

sf_status sf_scene_flow_learned(const uint8_t* left_t, const uint8_t* right_t, const uint8_t* left_t1,
                                const uint8_t* right_t1, int32_t pitch, const float* flow, int32_t W,
                                int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                                const void* packed, float threshold, float* s4_out, float* motion_out,
                                float* point_out, uint8_t* valid_out, float* D0_out, float* D1_out,
                                void* workspace, size_t ws_bytes, void* stream) {
  const sf_learned_frame f = {left_t, right_t, left_t1, right_t1, flow, s4_out, motion_out, point_out,
                              valid_out, D0_out, D1_out};
  return sf_scene_flow_learned_frames(&f, 1, pitch, W, H, p, cam, packed, threshold, workspace, ws_bytes,
                                      stream);
}

}  // extern "C"
