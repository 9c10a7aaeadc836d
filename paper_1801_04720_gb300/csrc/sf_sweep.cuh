// The band sweeps of the fused SGM path (template and launch dispatch),
// shared by the translation units that instantiate them: sgm_sweep.cu (the
// plain SGM) and sgm_sweep_var.cu (with the SGM variants compiled in), so
// the build compiles the two halves in parallel.  See sgm_fused.cu for the
// stages around them.
#pragma once

#include <algorithm>

#include "sf_fused.cuh"
#include "sgm_common.cuh"

// Sweep shapes this build provides: (disparities per thread, chunks, halo).
#define SF_SWEEP_SHAPES(X)                                                                   \
  X(8, 2, 16) X(8, 4, 16) X(8, 8, 16) X(8, 16, 16) X(8, 2, 8) X(8, 4, 8) X(8, 8, 8)        \
  X(8, 16, 8) X(16, 4, 8) X(16, 8, 8) X(16, 16, 8) X(16, 4, 16) X(16, 8, 16)

namespace sf {
namespace fused {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Penalty table of the intensity-adaptive P2 (the SGM cited in Sec. 3.1):
// entry g = P2 / g rounded down, at least P1, for an intensity step g > 0,
// and P2 for g = 0.  Filled by the whole block before its first barrier.
__device__ __forceinline__ void fill_p2_table(uint16_t* lut, int P1, int P2) {
  for (int g = threadIdx.x; g < 256; g += blockDim.x) lut[g] = (uint16_t)(g == 0 ? P2 : max(P1, P2 / g));
}
__device__ __forceinline__ uint32_t absdiff_u8(uint32_t a, uint32_t b) { return a > b ? a - b : b - a; }

// ---------------------------------------------------------------------------
// horizontal paths (+1,0) and (-1,0): one block of rows of one pass
// ---------------------------------------------------------------------------
constexpr long long kMbarSpin = 1ll << 22;     // bounded mbarrier wait

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          (unsigned)__cvta_generic_to_shared(dst)),
      "l"(src), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The rows [ybase, ybase + 2 pairs) of pass pd in direction dir (0: (+1,0),
// 1: (-1,0)), by the whole block: thread t = lp * CHUNKS + q owns line pair
// lp (two rows per u16x2 register) and disparities [q DC, q DC + DC).
// Column chunks of the cost volume (the block's rows x CW columns x Dp bytes)
// arrive by bulk asynchronous copies into two shared buffers of tile_bytes,
// their completion tracked by bars[2]; the serial walk along x reads them
// from shared memory and writes L_r as a uint8 volume.  The mbarriers are
// initialised by the caller and may serve several calls: ph[b] counts the
// phases bars[b] has completed, and is advanced here.  Every thread of the
// block calls this; s_lut holds the adaptive-P2 table when pd.guide is set
// (ADAPTIVE builds only).  Returns false when a copy never completed (err
// is then set and the block must stop).
template <int DC, int CHUNKS, bool ADAPTIVE>
__device__ __forceinline__ bool hline_rows_body(const PassDesc& pd, int dir, int ybase, int pairs, int P1, int P2,
                                           uint8_t* tiles, int tile_bytes, uint64_t* bars, int* s_fail,
                                           const uint16_t* s_lut, int* ph, int* err) {
  using V = typename ByteVec<DC>::T;
  const int W = pd.W, H = pd.H, Dp = pd.Dp;
  const uint8_t* C = pd.cost;
  uint8_t* out = dir == 0 ? pd.hfwd : pd.hbwd;
  const int t = threadIdx.x;
  const int lp = t / CHUNKS;
  const int q = t - lp * CHUNKS;
  const int rows = 2 * pairs;
  const int nrows = min(rows, H - ybase);
  const int r0 = 2 * lp, r1 = min(2 * lp + 1, nrows - 1);
  const bool row_ok = r0 < nrows;
  const int d0 = q * DC;
  const bool live = d0 < Dp;                 // chunks past the padded depth hold no data
  const bool io = live && row_ok;
  const bool two = r1 != r0;
  const int D = pd.D;
  const bool pad = d0 + DC > D;
  const bool q_first = q == 0, q_last = q == CHUNKS - 1;
  const uint32_t p1x2 = P1 * 0x10001u, p2x2 = P2 * 0x10001u;
  const int CW = max(1, tile_bytes / (rows * Dp));   // columns per chunk
  const int nchunks = (W + CW - 1) / CW;
  auto chunk_x0 = [&](int c) { return dir == 0 ? c * CW : max(0, W - (c + 1) * CW); };
  auto chunk_w = [&](int c) { return dir == 0 ? min(CW, W - c * CW) : (W - c * CW) - chunk_x0(c); };
  auto issue = [&](int c) {                  // one thread: all rows of chunk c
    uint8_t* dst = tiles + (c & 1) * tile_bytes;
    const int xs = chunk_x0(c), cw = chunk_w(c);
    const unsigned bytes = (unsigned)(cw * Dp);
    fence_proxy_async();
    mbar_arrive_tx(&bars[c & 1], bytes * (unsigned)nrows);
    for (int r = 0; r < nrows; r++)
      bulk_g2s(dst + (size_t)r * CW * Dp, C + ((size_t)(ybase + r) * W + xs) * Dp, bytes, &bars[c & 1]);
  };
  if (t == 0) *s_fail = 0;
  __syncthreads();   // barriers initialised, shared memory free, s_fail cleared
  if (t == 0) issue(0);
  uint32_t L[DC], Cr[DC], N[DC];
#pragma unroll
  for (int i = 0; i < DC; i++) L[i] = 0;
  uint32_t m = 0;
  // adaptive P2: the guide pixels of both rows at the walk's current column
  // (rows past the block's last row read its last row; their lanes are not
  // stored) and the previous column's values
  const bool adaptive = ADAPTIVE && pd.guide != nullptr;
  const int gstep = dir == 0 ? 1 : -1;
  const uint8_t* ga = nullptr;
  const uint8_t* gb = nullptr;
  uint32_t gprev0 = 0, gprev1 = 0;
  if (adaptive) {
    const int xstart = dir == 0 ? 0 : W - 1;
    ga = pd.guide + (size_t)(ybase + min(r0, nrows - 1)) * pd.gpitch + xstart;
    gb = pd.guide + (size_t)(ybase + r1) * pd.gpitch + xstart;
  }
  // one step along the line: costs from the tile, the update, the outputs.
  // (A line's first step has L = 0 and m = 0, so its update is C whatever
  // the end values at d = 0 and d = Dp-1.)
  const int step = dir == 0 ? Dp : -Dp;
  auto line_step = [&](const uint8_t*& ta, const uint8_t*& tb, uint8_t*& oa, uint8_t*& ob, const uint32_t* Lp,
                       uint32_t* Ln) {
    V va = ByteVec<DC>::zero(), vb = va;
    if (io) {
      va = *reinterpret_cast<const V*>(ta);
      vb = *reinterpret_cast<const V*>(tb);
    }
    ta += step;
    tb += step;
    bytes_to_pairs<DC>(va, vb, Cr);
    if (pad) {
#pragma unroll
      for (int i = 0; i < DC; i++)
        if (d0 + i >= D) Cr[i] = kPadCost2;
    }
    uint32_t left = __shfl_up_sync(0xffffffffu, Lp[DC - 1], 1, CHUNKS);
    uint32_t right = __shfl_down_sync(0xffffffffu, Lp[0], 1, CHUNKS);
    if (q_first) left = kInf2;
    if (q_last) right = kInf2;
    uint32_t p2s = p2x2;
    if (ADAPTIVE && adaptive) {
      // (a line's first step gets a meaningless penalty: its update is C)
      const uint32_t i0 = __ldg(ga), i1 = __ldg(gb);
      ga += gstep;
      gb += gstep;
      p2s = (uint32_t)s_lut[absdiff_u8(i0, gprev0)] | ((uint32_t)s_lut[absdiff_u8(i1, gprev1)] << 16);
      gprev0 = i0;
      gprev1 = i1;
    }
    sgm_update<DC>(Lp, Cr, left, right, m, p1x2, p2s, Ln);
    m = group_min2<CHUNKS>(tree_min<DC>(Ln));
    if (io) {
      V wa, wb;
      pairs_to_bytes<DC>(Ln, wa, wb);
      store_cs(reinterpret_cast<V*>(oa), wa);
      if (two) store_cs(reinterpret_cast<V*>(ob), wb);
    }
    oa += step;
    ob += step;
  };
  // Chunk c is the (c >> 1)-th phase of this call on bars[c & 1], i.e. phase
  // ph[c & 1] + (c >> 1) overall; waiting on that phase's parity returns once
  // it has completed.
  auto parity = [&](int c) { return (unsigned)((ph[c & 1] + (c >> 1)) & 1); };
  int c = 0;
  for (; c < nchunks; c++) {
    if (t == 0 && c + 1 < nchunks) issue(c + 1);
    const unsigned par = parity(c);
    // bounded wait for chunk c by one thread; every thread then reads the
    // verdict after the same barrier, so all of them leave or stay together
    if (t == 0) {
      long long spins = 0;
      while (!mbar_try_wait(&bars[c & 1], par)) {
        if (++spins > kMbarSpin) {
          *s_fail = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (*s_fail) break;
    // the phase has completed: each thread observes it itself (returns at
    // once), which orders the copied bytes before its reads
    {
      long long spins = 0;
      while (!mbar_try_wait(&bars[c & 1], par) && ++spins < kMbarSpin) {
      }
    }
    const int xs = chunk_x0(c), cw = chunk_w(c);
    const int cx0 = dir == 0 ? 0 : cw - 1;   // first column of the walk in this chunk
    const uint8_t* tile = tiles + (c & 1) * tile_bytes;
    const uint8_t* ta = tile + (r0 * CW + cx0) * Dp + d0;
    const uint8_t* tb = tile + (r1 * CW + cx0) * Dp + d0;
    uint8_t* oa = out + ((size_t)(ybase + r0) * W + xs + cx0) * Dp + d0;
    uint8_t* ob = out + ((size_t)(ybase + r1) * W + xs + cx0) * Dp + d0;
    int u = 0;
    // two steps per trip: the states alternate between L and N (no copies)
    for (; u + 1 < cw; u += 2) {
      line_step(ta, tb, oa, ob, L, N);
      line_step(ta, tb, oa, ob, N, L);
    }
    if (u < cw) {
      line_step(ta, tb, oa, ob, L, N);
#pragma unroll
      for (int i = 0; i < DC; i++) L[i] = N[i];
    }
    __syncthreads();   // buffer c&1 is free for chunk c+2
  }
  const bool ok = *s_fail == 0;
  if (!ok) {
    // chunk c never completed: record it, then let the copies still in
    // flight land before the block leaves its shared memory (bounded).  In
    // flight: chunk c and, if it was issued, chunk c + 1; every earlier chunk
    // was waited for.  Each is awaited on the parity of its own phase.
    if (t == 0) {
      atomicExch(err, 1);
      const int last = min(c + 1, nchunks - 1);
      for (int cc = c; cc <= last; cc++) {
        long long spins = 0;
        while (!mbar_try_wait(&bars[cc & 1], parity(cc)) && ++spins < kMbarSpin) {
        }
      }
    }
    __syncthreads();
    return false;
  }
  ph[0] += (nchunks + 1) >> 1;
  ph[1] += nchunks >> 1;
  return true;
}

// hline_rows_body inlined into the standalone kernel, and called out of
// line from the merged sweep kernel (whose own registers it would otherwise
// crowd).
template <int DC, int CHUNKS, bool ADAPTIVE>
__device__ __forceinline__ bool hline_rows(const PassDesc& pd, int dir, int ybase, int pairs, int P1, int P2,
                                           uint8_t* tiles, int tile_bytes, uint64_t* bars, int* s_fail,
                                           const uint16_t* s_lut, int* ph, int* err) {
  return hline_rows_body<DC, CHUNKS, ADAPTIVE>(pd, dir, ybase, pairs, P1, P2, tiles, tile_bytes, bars, s_fail, s_lut,
                                               ph, err);
}
template <int DC, int CHUNKS, bool ADAPTIVE>
__device__ __noinline__ bool hline_rows_call(const PassDesc& pd, int dir, int ybase, int pairs, int P1, int P2,
                                             uint8_t* tiles, int tile_bytes, uint64_t* bars, int* s_fail,
                                             const uint16_t* s_lut, int* ph, int* err) {
  return hline_rows_body<DC, CHUNKS, ADAPTIVE>(pd, dir, ybase, pairs, P1, P2, tiles, tile_bytes, bars, s_fail, s_lut,
                                               ph, err);
}

// ---------------------------------------------------------------------------
// 3./4. band sweeps
// ---------------------------------------------------------------------------
// Thread layout: t = pair * CHUNKS + q.  Pairs 0..15 own columns
// (x0 + c, x0 + 16 + c) and carry all three paths.  FL = the diagonal path fed
// from column x-1 ((+1,+1) down, (+1,-1) up), FR = the one fed from column
// x+1 ((-1,+1) down, (-1,-1) up).  FL enters the strip from the left, so the
// left halo pairs (x0 - HALO + h, x0 - HALO/2 + h) carry FL only; the right
// halo pairs (x1 + h, x1 + HALO/2 + h) carry FR only.  Halo pairs whose
// columns can no longer reach the strip before the band ends skip the update.

// Task index -> (pass, step in processing order, strip, scan order).  Tasks are
// step-major; with one shape for every pass the split is arithmetic,
// otherwise passes are sorted by band count (descending) and the tables give
// each step's first task and the prefix of strip counts.  A merged launch
// (both scan orders in one queue) lists, per step, the tasks of the down
// sweep and then those of the up sweep (scan 1).
template <bool MERGED>
__device__ __forceinline__ void decode_task(const SweepArgs& a, int task, int& p, int& bi, int& j, int& scan) {
  scan = 0;
  if (a.uniform_items > 0) {
    const int per = MERGED ? 2 * a.uniform_items : a.uniform_items;
    bi = task / per;
    int it = task - bi * per;
    if (MERGED && it >= a.uniform_items) {
      scan = 1;
      it -= a.uniform_items;
    }
    const int J = a.inl[0].J;
    p = it / J;
    j = it - p * J;
    return;
  }
  int lo = 0, hi = a.nbands - 1;   // last step whose first task <= task
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.band_start[mid] <= task) lo = mid; else hi = mid - 1;
  }
  bi = lo;
  int off = task - a.band_start[bi];
  if (MERGED) {
    const int nact = a.prefixJ[a.band_npass[bi]];
    if (off >= nact) {
      scan = 1;
      off -= nact;
    }
  }
  int plo = 0, phi = a.band_npass[bi] - 1;   // last pass whose strip prefix <= off
  while (plo < phi) {
    const int mid = (plo + phi + 1) >> 1;
    if (a.prefixJ[mid] <= off) plo = mid; else phi = mid - 1;
  }
  p = plo;
  j = off - a.prefixJ[p];
}

template <int N>
__device__ __forceinline__ void load_u4(uint32_t* r, const uint4* src, int stride) {
#pragma unroll
  for (int w = 0; w < N / 4; w++) {
    const uint4 v = src[w * stride];
    r[4 * w] = v.x; r[4 * w + 1] = v.y; r[4 * w + 2] = v.z; r[4 * w + 3] = v.w;
  }
}

template <int N>
__device__ __forceinline__ void store_u4(uint4* dst, int stride, const uint32_t* r) {
#pragma unroll
  for (int w = 0; w < N / 4; w++) dst[w * stride] = make_uint4(r[4 * w], r[4 * w + 1], r[4 * w + 2], r[4 * w + 3]);
}

// Launch modes of the band sweeps: the down sweep alone, the up sweep alone
// (it reads the down sweep's partial sums and selects), or both scan orders
// in one launch.  In the merged launch each band of a strip is reached twice,
// once by each scan order: the first arrival stores its three paths' partial
// sum, the second adds it, the horizontal paths and its own three paths, and
// selects.  With M = ceil(nb / 2), the down sweep arrives first at bands
// 0 .. M-1 and the up sweep at bands M .. nb-1, so both run at once from
// opposite ends and the work in flight doubles.
constexpr int kModeDown = 0, kModeUp = 1, kModeMerged = 2;
// kModeMergedH: kModeMerged whose queue starts with the horizontal paths'
// row blocks (hline_rows, 2 (16 + HALO) rows each), each publishing a flag
// that the second arrivals at its rows wait for, so those latency-bound
// walks overlap the first half of the sweeps instead of preceding them.
constexpr int kModeMergedH = 3;

template <int DC, int CHUNKS, int HALO, int MODE>
struct SweepCfg {
  static constexpr bool SEC = MODE != kModeDown;   // second arrivals possible
  static constexpr bool MERGED = MODE == kModeMerged || MODE == kModeMergedH;
  static constexpr int NP = 16 + HALO;      // column pairs per task
  static constexpr int NT = NP * CHUNKS;    // threads
  static constexpr int NO = 16 * CHUNKS;    // threads of owned pairs
  static constexpr int TH = HALO + 1;       // band rows
  static constexpr int RING = SEC ? 2 : 3;  // prefetch depth in rows
  static constexpr int XW = DC / 4 + 4;     // uint4 slots per owned thread per row (second arrival)
  // halo threads per owned column pair for the winner selection
  static constexpr int select_threads() { return (HALO * CHUNKS) / 16 > 0 ? (HALO * CHUNKS) / 16 : 1; }
  static constexpr bool select_by_halo() {
    return SEC && CHUNKS >= 2 && (HALO * CHUNKS) / 16 >= 1 && select_threads() <= 32 &&
           (CHUNKS % select_threads()) == 0;
  }
  static constexpr size_t smem_bytes() {
    return (size_t)2 * 2 * (DC / 4) * NT * 16     // diagonal hand-over
           + (size_t)2 * 2 * NP * 4                // pair minima
           + (size_t)2 * (DC / 4) * NO * 16        // aggregated-cost rows for selection
           + (size_t)RING * 2 * NT * DC            // cost ring
           + (SEC ? (size_t)RING * XW * NO * 16 : 0);
  }
};

// Registers: a separate down or up launch runs one CTA per SM with nothing
// beside it, so it may use the whole register file (at most 168 a thread;
// the 16-disparity shapes keep 168); a merged launch aims at two CTAs per SM.
constexpr int sweep_max_regs(int nt, int ctas) {
  const int budget = 65536 / (nt * ctas);
  return budget > 168 ? 168 : (budget / 8) * 8;
}

// two CTAs per SM for a merged launch where that leaves a thread at least
// 128 registers, else one
constexpr int merged_ctas(int nt) { return 65536 / (2 * nt) >= 128 ? 2 : 1; }

// VAR: the SGM variants (intensity-adaptive P2, uniqueness filter) are
// compiled in; without them the kernel carries none of their registers.
template <int DC, int CHUNKS, int HALO, int MODE, bool VAR>
__global__ void __launch_bounds__((16 + HALO) * CHUNKS, 1)
    __maxnreg__(MODE >= kModeMerged ? sweep_max_regs((16 + HALO) * CHUNKS, merged_ctas((16 + HALO) * CHUNKS))
                                    : (DC == 16 ? 168 : sweep_max_regs((16 + HALO) * CHUNKS, 1)))
    sweep_kernel(const __grid_constant__ SweepArgs a) {
  using Cfg = SweepCfg<DC, CHUNKS, HALO, MODE>;
  using V = typename ByteVec<DC>::T;
  constexpr int NP = Cfg::NP, NT = Cfg::NT, NO = Cfg::NO, TH = Cfg::TH, RING = Cfg::RING;
  constexpr int XW = Cfg::XW, G = DC / 4;
  // winner selection by the halo warps (they carry one path, the owned
  // warps three plus the sums): SEL_P threads per owned column pair
  constexpr int SEL_P = Cfg::select_threads();
  constexpr bool HALO_SELECT = Cfg::select_by_halo();
  static_assert(HALO_SELECT || !Cfg::SEC, "launches with second arrivals select by the halo threads");
  extern __shared__ __align__(16) uint8_t smem[];
  // diagonal hand-over buffers, [parity][register group][thread] uint4
  // (consecutive threads hit consecutive 16-byte words: no bank conflicts)
  uint4* xfl = reinterpret_cast<uint4*>(smem);
  uint4* xfr = xfl + 2 * G * NT;
  uint32_t* mfl = reinterpret_cast<uint32_t*>(xfr + 2 * G * NT);   // [parity][pair]
  uint32_t* mfr = mfl + 2 * NP;
  uint4* srow = reinterpret_cast<uint4*>(mfr + 2 * NP);            // [parity][group][owned thread]
  V* ringc = reinterpret_cast<V*>(srow + 2 * G * NO);              // [slot][lo/hi][thread]
  uint4* ringx = reinterpret_cast<uint4*>(ringc + RING * 2 * NT);  // [slot][XW][owned thread]
  __shared__ int s_abort;
  __shared__ int s_task;
  __shared__ uint16_t s_lut[256];   // adaptive P2 by intensity step
  constexpr bool MERGED = Cfg::MERGED;
  constexpr bool HL = MODE == kModeMergedH;
  constexpr int HL_ROWS = merged_hline_rows(DC, CHUNKS, HALO);   // rows per horizontal-path task
  __shared__ __align__(8) uint64_t hbars[2];   // horizontal-path tiles (HL)
  __shared__ int s_hfail;
  int hph[2] = {0, 0};

  const int t = threadIdx.x;
  const int pr = t / CHUNKS;
  const int q = t - pr * CHUNKS;
  const bool owned = pr < 16;
  const int d0 = q * DC;
  const uint32_t p1x2 = a.P1 * 0x10001u, p2x2 = a.P2 * 0x10001u;
  static_assert(CHUNKS >= 2, "owned pairs fill whole warps");
  constexpr int HH = HALO / 2;             // pairs per halo side
  constexpr int LH0 = 16, RH0 = 16 + HH;    // first left / right halo pair
  const int role = owned ? 0 : (pr < RH0 ? 1 : 2);   // 0 owned, 1 left halo, 2 right halo
  // lanes of this thread's role in its warp: owned pairs fill whole warps;
  // a warp may hold pairs of both halo sides (whole pairs of CHUNKS lanes),
  // and each side runs its own code with its own shuffles
  const unsigned role_mask = __ballot_sync(0xffffffffu, owned) * (role == 0) +
                             __ballot_sync(0xffffffffu, role == 1) * (role == 1) +
                             __ballot_sync(0xffffffffu, role == 2) * (role == 2);
  const int hh = role == 1 ? pr - LH0 : pr - RH0;
  // hand-over sources: FL from column x-1, FR from column x+1.  Whole
  // registers move between pairs except at the seams of the layout, where
  // prmt joins one lane of each of two pairs.
  int fl_src = pr, fl_src2 = -1, fr_src = pr, fr_src2 = -1;
  uint32_t fl_sel = 0, fr_sel = 0;
  if (role == 0) {
    if (pr > 0) fl_src = pr - 1;
    else { fl_src = RH0 - 1; fl_src2 = 15; fl_sel = 0x5432u; }    // (x0-1, x0+15)
    if (pr < 15) fr_src = pr + 1;
    else { fr_src = 0; fr_src2 = RH0; fr_sel = 0x5432u; }         // (x0+16, x1)
  } else if (role == 1) {
    if (hh > 0) fl_src = pr - 1;
    else { fl_src = pr; fl_src2 = RH0 - 1; fl_sel = 0x5410u; }    // (-, x0-HALO/2-1)
  } else {
    if (hh < HH - 1) fr_src = pr + 1;
    else { fr_src = RH0; fr_src2 = pr; fr_sel = 0x7632u; }        // (x1+HALO/2, -)
  }
  if (t == 0) s_abort = 0;
  if (HL && t == 0) {
    mbar_init(&hbars[0], 1);
    mbar_init(&hbars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (VAR) fill_p2_table(s_lut, a.P1, a.P2);
  __syncthreads();

  // Tasks (band, pass, strip) in band-major order from a global counter: any
  // CTA takes the next one, so a slow SM delays nobody but itself.  A task
  // waits (bounded) for the previous band of its own strip and of both
  // neighbour strips; those tasks were handed out earlier.  A CTA claims its
  // next task as soon as its current one has passed its waits (the counter's
  // round trip then overlaps the band); a claimed task that is not running
  // yet belongs to a CTA whose current task comes earlier in the queue and
  // only waits on still earlier tasks, so by induction over the queue every
  // claimed task runs.
  const int ntasks = a.ntasks;
  if (t == 0) s_task = atomicAdd(a.task_counter, 1);
  for (;;) {
    __syncthreads();   // the claim is visible; every thread has left the previous task
    int task = s_task;
    if (task >= ntasks) break;
    if (HL) {
      if (task < a.hl_tasks) {
        // a block of rows of the horizontal paths (2 hl_blocks per pass)
        const int per = 2 * a.hl_blocks;
        const int hp = task / per, hrem = task - hp * per;
        const int dir = hrem / a.hl_blocks, rb = hrem - dir * a.hl_blocks;
        const PassDesc hd = a.pass_ptr ? a.pass_ptr[hp] : a.inl[hp];
        if ((a.path_mask >> dir) & 1u) {
          constexpr int kTile = (int)((Cfg::smem_bytes() / 2) & ~(size_t)127);
          // a warp per line pair above 64 disparities (4 a lane up to 128,
          // 8 above), as the standalone walk; else the sweep's own layout
          constexpr bool kWarp = HL_ROWS != 2 * NP;
          constexpr int kHDC = DC * CHUNKS > 128 ? 8 : 4;
          bool hok;
          if constexpr (kWarp)
            hok = hline_rows_call<kHDC, 32, VAR>(hd, dir, rb * HL_ROWS, HL_ROWS / 2, a.P1, a.P2, smem, kTile, hbars,
                                                 &s_hfail, s_lut, hph, a.err);
          else
            hok = hline_rows_call<DC, CHUNKS, VAR>(hd, dir, rb * HL_ROWS, NP, a.P1, a.P2, smem, kTile, hbars,
                                                   &s_hfail, s_lut, hph, a.err);
          if (!hok) return;
        }
        __syncthreads();   // every thread's stores before the release
        if (t == 0) {
          st_release(hd.flags_h + dir * a.hl_blocks + rb, 1);
          s_task = atomicAdd(a.task_counter, 1);   // every thread read this task's index before the barrier
        }
        continue;
      }
      task -= a.hl_tasks;
    }
    int p, bi, j, scan;   // scan: 0 down sweep, 1 up sweep (merged launch)
    decode_task<MERGED>(a, task, p, bi, j, scan);
    const PassDesc pd = a.pass_ptr ? a.pass_ptr[p] : a.inl[p];   // by value: fields in registers
    const int W = pd.W, H = pd.H, Dp = pd.Dp, J = pd.J, D = pd.D;
    // scan order of this task (up: bottom to top) and whether it is the
    // second arrival at its band (adds the other order's partial sum and the
    // horizontal paths, and selects) or the first (stores its partial sum)
    const bool up = MODE == kModeUp || (MERGED && scan == 1);
    const int band = up ? (pd.nb - 1 - bi) : bi;
    const int meet = (pd.nb + 1) >> 1;
    const bool second = MODE == kModeUp ? true
                                        : (MODE == kModeDown ? false : (up ? band < meet : band >= meet));
    const bool en_v = (a.path_mask >> (up ? 3 : 2)) & 1u;
    const bool en_fl = (a.path_mask >> (up ? 6 : 4)) & 1u;
    const bool en_fr = (a.path_mask >> (up ? 5 : 7)) & 1u;
    const bool en_all = en_v && en_fl && en_fr;
    const bool pad = d0 + DC > D;
    const bool s_vec = second && pd.S && D % 8 == 0 && (reinterpret_cast<uintptr_t>(pd.S) & 15u) == 0;
    const bool live = d0 < Dp;   // chunks past the padded depth hold no data
    const int ytop = band * TH;
    const int nrows = min(TH, H - ytop);
    const int x0 = j * kTW;
    int* const flags = up ? pd.flags_up : pd.flags_down;
    // ---- columns of this thread's pair ----
    int xlo, xhi;
    if (role == 0) {
      xlo = x0 + pr;
      xhi = x0 + 16 + pr;
    } else if (role == 1) {
      xlo = x0 - HALO + hh;
      xhi = x0 - HH + hh;
    } else {
      xlo = x0 + kTW + hh;
      xhi = x0 + kTW + HH + hh;
    }
    const bool lo_in = live && xlo >= 0 && xlo < W, hi_in = live && xhi >= 0 && xhi < W;
    // this thread's S_down tiles (down sweep): row y at sd_out + y * sd_row
    uint4* const sd_out = reinterpret_cast<uint4*>(pd.sdown) + ((size_t)(j * 16 + pr) * CHUNKS + q) * G;
    const size_t sd_row = (size_t)J * 16 * CHUNKS * G;
    // ---- prefetch ring: the first rows' inputs are requested before the
    // neighbour wait (they do not depend on it) ----
    // parts: 1 the costs, 2 the other order's partial sums, 4 the
    // horizontal volumes (the last two for a second arrival's owned pairs)
    auto issue_row = [&](int r, int parts) {
      const bool ok = r < nrows;
      const int yy = up ? ytop + nrows - 1 - r : ytop + r;
      if (parts & 1) {
        V* cs = ringc + (r % RING) * 2 * NT + t;
        const uint8_t* rowc = pd.cost + (size_t)yy * W * Dp + d0;
        cp_async<DC>(cs, ok && lo_in ? rowc + (size_t)xlo * Dp : pd.cost, ok && lo_in);
        cp_async<DC>(cs + NT, ok && hi_in ? rowc + (size_t)xhi * Dp : pd.cost, ok && hi_in);
      }
      if (Cfg::SEC && second && owned) {
        uint4* xs = ringx + (r % RING) * XW * NO + t;
        if (parts & 2) {
          const uint4* sd = sd_out + (ok ? (size_t)yy * sd_row : 0);
#pragma unroll
          for (int w = 0; w < G; w++) cp_async<16>(xs + w * NO, sd + w, ok);
        }
        if (parts & 4) {
          const size_t ol = ((size_t)yy * W + xlo) * Dp + d0, oh = ((size_t)yy * W + xhi) * Dp + d0;
          const bool fl = ok && lo_in, fh = ok && hi_in;
          cp_async<DC>(xs + (G + 0) * NO, fl && a.en_h0 ? pd.hfwd + ol : pd.hfwd, fl && a.en_h0);
          cp_async<DC>(xs + (G + 1) * NO, fh && a.en_h0 ? pd.hfwd + oh : pd.hfwd, fh && a.en_h0);
          cp_async<DC>(xs + (G + 2) * NO, fl && a.en_h1 ? pd.hbwd + ol : pd.hbwd, fl && a.en_h1);
          cp_async<DC>(xs + (G + 3) * NO, fh && a.en_h1 ? pd.hbwd + oh : pd.hbwd, fh && a.en_h1);
        }
      }
      cp_async_commit();
    };
    // A second arrival of a merged launch reads the other order's partial
    // sums, which exist only after its wait: its first rows' costs (and,
    // when the horizontal paths ran in an earlier launch, their volumes) are
    // requested before the wait, the partial sums after it.  The extra
    // commit group is older than every later row's, so the ring's
    // wait_group count still covers each row.
    const bool early = !(MERGED && second);
    const int pre = early ? 7 : (HL ? 1 : 1 | 4);
#pragma unroll
    for (int r = 0; r < RING - 1; r++) issue_row(r, pre);
    // ---- wait for the previous band of this strip and its neighbours, and
    // (second arrival of a merged launch) for the other scan order's pass
    // over this band of this strip: the first warp's lanes poll one flag
    // each, so the flags' round trips overlap (at most 3 + 1 + 6 flags) ----
    if (t < 32) {
      const int* fp = nullptr;
      int tgt = 0, idx = 0;
      auto add = [&](const int* f, int target) {
        if (idx == t) {
          fp = f;
          tgt = target;
        }
        idx++;
      };
      if (bi > 0) {
        for (int n = j - 1; n <= j + 1; n++)
          if (n >= 0 && n < J) add(flags + n, bi);
      }
      if (MERGED && second) add((up ? pd.flags_down : pd.flags_up) + j, up ? band + 1 : pd.nb - band);
      if (HL && second) {
        // the horizontal paths of this band's rows
        const int hr0 = ytop / HL_ROWS, hr1 = (ytop + nrows - 1) / HL_ROWS;
        for (int dir = 0; dir < 2; dir++)
          for (int rb = hr0; rb <= hr1; rb++) add(pd.flags_h + dir * a.hl_blocks + rb, 1);
      }
      if (fp) {
        long long spins = 0;
        while (ld_acquire(fp) < tgt) {
          if (++spins > a.spin_limit || *((volatile int*)a.err) != 0) {
            atomicExch(a.err, 1);
            s_abort = 1;
            break;
          }
          if (spins > 64) __nanosleep(32);
        }
      }
    }
    __syncthreads();
    if (s_abort) {
      cp_async_wait<0>();
      return;
    }
    // claim the next task now (every thread read this one's index before
    // the barrier above); the last thread, a halo lane, holds the answer in
    // a register until the band ends, so no warp waits for the round trip
    int next_task = 0;
    if (t == NT - 1) next_task = atomicAdd(a.task_counter, 1);
    if (!early) {
#pragma unroll
      for (int r = 0; r < RING - 1; r++) issue_row(r, 7 & ~pre);
    }

    // lanes whose predecessor column lies outside the image start a path
    const uint32_t fl_keep = ((xlo - 1 >= 0) ? 0x0000ffffu : 0u) | ((xhi - 1 >= 0) ? 0xffff0000u : 0u);
    const uint32_t fr_keep = ((xlo + 1 < W) ? 0x0000ffffu : 0u) | ((xhi + 1 < W) ? 0xffff0000u : 0u);
    // band-end states [order][parity][3][W][Dp]: each scan order of a merged
    // launch has its own (a separate up launch reuses the down sweep's)
    uint8_t* const bs0 = pd.bs + (MERGED && up ? (size_t)6 * W * Dp : 0);
    const uint8_t* bsv = bs0 + ((size_t)(((bi + 1) & 1)) * 3 + 0) * W * Dp;
    const uint8_t* bsl = bsv + (size_t)W * Dp;
    const uint8_t* bsr = bsl + (size_t)W * Dp;
    uint8_t* wsv = bs0 + ((size_t)((bi & 1)) * 3 + 0) * W * Dp;
    uint8_t* wsl = wsv + (size_t)W * Dp;
    uint8_t* wsr = wsl + (size_t)W * Dp;

    uint32_t Lv[DC], Lf[DC], Lr[DC], Cc[DC];
    uint32_t mv = 0, mf = 0, mr = 0;
    // ---- predecessor states at the band boundary ----
    {
      const bool have = bi > 0;
      auto load_pair = [&](const uint8_t* base, int cl, int ch, uint32_t* r, uint32_t keep) {
        V va = ByteVec<DC>::zero(), vb = va;
        if (live && have && (keep & 0xffffu) && cl >= 0 && cl < W)
          va = __ldcg(reinterpret_cast<const V*>(base + (size_t)cl * Dp + d0));
        if (live && have && (keep & 0xffff0000u) && ch >= 0 && ch < W)
          vb = __ldcg(reinterpret_cast<const V*>(base + (size_t)ch * Dp + d0));
        bytes_to_pairs_u8<DC>(va, vb, r);
        if (pad) {
#pragma unroll
          for (int i = 0; i < DC; i++)
            if (d0 + i >= D) r[i] = (have ? kPadCost2 : 0u) & keep;
        }
      };
#pragma unroll
      for (int i = 0; i < DC; i++) Lv[i] = Lf[i] = Lr[i] = 0;
      if (role == 0) {
        load_pair(bsv, xlo, xhi, Lv, 0xffffffffu);
        load_pair(bsl, xlo - 1, xhi - 1, Lf, fl_keep);
        load_pair(bsr, xlo + 1, xhi + 1, Lr, fr_keep);
        const uint32_t av = group_min2<CHUNKS>(tree_min<DC>(Lv), role_mask);
        const uint32_t af = group_min2<CHUNKS>(tree_min<DC>(Lf), role_mask);
        const uint32_t ar = group_min2<CHUNKS>(tree_min<DC>(Lr), role_mask);
        mv = have ? av : 0u;
        mf = have ? (af & fl_keep) : 0u;
        mr = have ? (ar & fr_keep) : 0u;
      } else if (role == 1) {
        load_pair(bsl, xlo - 1, xhi - 1, Lf, fl_keep);
        const uint32_t af = group_min2<CHUNKS>(tree_min<DC>(Lf), role_mask);
        mf = have ? (af & fl_keep) : 0u;
      } else {
        load_pair(bsr, xlo + 1, xhi + 1, Lr, fr_keep);
        const uint32_t ar = group_min2<CHUNKS>(tree_min<DC>(Lr), role_mask);
        mr = have ? (ar & fr_keep) : 0u;
      }
    }

    // winner-take-all + parabolic subpixel of row kk, done by the halo
    // threads from the aggregated costs the owned threads left in shared
    // memory: SEL_P threads per owned column pair, packed u16x2 minima over
    // both columns at once.  Padding disparities hold 0xffff there, above
    // every aggregated cost (at most 8 x 255).
    auto select_row = [&](int kk) {
      if (!HALO_SELECT || owned || !pd.dint || !second) return;
      constexpr int PT = SEL_P, CPT = CHUNKS / SEL_P;
      const int yk = up ? ytop + nrows - 1 - kk : ytop + kk;
      const int ht = t - NO;
      const int cp = ht / PT, sub = ht - cp * PT;
      const uint4* rw = srow + (kk & 1) * G * NO + cp * CHUNKS + sub * CPT;
      // the minimal S of each column, over this thread's chunks, then over
      // the pair's threads
      uint32_t g = 0xffffffffu;
#pragma unroll
      for (int jj = 0; jj < CPT; jj++) {
#pragma unroll
        for (int w = 0; w < G; w++) {
          const uint4 v4 = rw[w * NO + jj];
          g = vmin2(g, vmin2(vmin2(v4.x, v4.y), vmin2(v4.z, v4.w)));
        }
      }
#pragma unroll
      for (int o = 1; o < PT; o <<= 1) g = vmin2(g, __shfl_xor_sync(0xffffffffu, g, o, PT));
      // the first disparity reaching it: key = (S > min) * 256 + d per
      // column (S - min >= 0 lane-wise, so the subtraction borrows nothing)
      uint32_t key = 0xffffffffu;
#pragma unroll
      for (int jj = 0; jj < CPT; jj++) {
        const uint32_t db = (uint32_t)((sub * CPT + jj) * DC) * 0x10001u;
#pragma unroll
        for (int w = 0; w < G; w++) {
          const uint4 v4 = rw[w * NO + jj];
          const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int e = 0; e < 4; e++)
            key = vmin2(key, vmin2(vv[e] - g, 0x10001u) * 256u + db + (uint32_t)(4 * w + e) * 0x10001u);
        }
      }
#pragma unroll
      for (int o = 1; o < PT; o <<= 1) key = vmin2(key, __shfl_xor_sync(0xffffffffu, key, o, PT));
      // uniqueness: the smallest S two or more disparities away from d*
      uint32_t s2 = 0xffffffffu;
      if (VAR && a.unique && pd.dsub) {
        const int dl = (int)(key & 0xffu), dh = (int)((key >> 16) & 0xffu);
#pragma unroll
        for (int jj = 0; jj < CPT; jj++) {
#pragma unroll
          for (int w = 0; w < G; w++) {
            const uint4 v4 = rw[w * NO + jj];
            const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const int d = (sub * CPT + jj) * DC + 4 * w + e;
              const uint32_t ex = ((d >= dl - 1 && d <= dl + 1) ? 0x0000ffffu : 0u) |
                                  ((d >= dh - 1 && d <= dh + 1) ? 0xffff0000u : 0u);
              s2 = vmin2(s2, vv[e] | ex);
            }
          }
        }
#pragma unroll
        for (int o = 1; o < PT; o <<= 1) s2 = vmin2(s2, __shfl_xor_sync(0xffffffffu, s2, o, PT));
      }
      // thread 0 of the pair writes the low column, thread 1 the high one
      const uint32_t* sw = reinterpret_cast<const uint32_t*>(srow + (kk & 1) * G * NO);
      for (int l = sub; l < 2; l += PT) {
        const int x = x0 + cp + 16 * l;
        if (x >= W) continue;
        const int sh = 16 * l;
        auto s_at = [&](int d) {
          const int qq = d / DC, ii = d - qq * DC;
          return (sw[((ii >> 2) * NO + cp * CHUNKS + qq) * 4 + (ii & 3)] >> sh) & 0xffffu;
        };
        const int ds = (int)((key >> sh) & 0xffu);
        const int sv = (int)((g >> sh) & 0xffffu);
        float v = (float)ds;
        if (a.subpixel && ds > 0 && ds < D - 1) {
          const int am = (int)s_at(ds - 1) - sv;
          const int bp = (int)s_at(ds + 1) - sv;
          v = __fadd_rn((float)ds, __fdiv_rn((float)(am - bp), (float)(2 * (am + bp))));
        }
        if (VAR && 100 * (int)((s2 >> sh) & 0xffffu) < (100 + a.unique) * sv) v = __int_as_float(0x7fc00000);
        pd.dint[(size_t)yk * W + x] = (int16_t)ds;
        if (pd.dsub) pd.dsub[(size_t)yk * W + x] = v;
      }
    };

    // neighbour disparities d0-1 and d0+DC of one path: from the adjacent
    // chunks of the pair, or "none" (kInf2) past d = 0 and d = Dp-1.  A lane
    // without a predecessor (first row, or its column just entered the
    // image) has L = 0 and m = 0, so its update is C whatever these values.
    const bool q_first = q == 0, q_last = q == CHUNKS - 1;
    auto neighbours = [&](const uint32_t* L, uint32_t& lo, uint32_t& hi) {
      lo = __shfl_up_sync(role_mask, L[DC - 1], 1, CHUNKS);
      hi = __shfl_down_sync(role_mask, L[0], 1, CHUNKS);
      if (q_first) lo = kInf2;
      if (q_last) hi = kInf2;
    };

    for (int k = 0; k < nrows; k++) {
      const int y = up ? ytop + nrows - 1 - k : ytop + k;
      issue_row(k + RING - 1, 7);
      cp_async_wait<RING - 1>();
      {
        const V* cs = ringc + (k % RING) * 2 * NT + t;
        bytes_to_pairs<DC>(cs[0], cs[NT], Cc);
      }
      if (pad) {
#pragma unroll
        for (int i = 0; i < DC; i++)
          if (d0 + i >= D) Cc[i] = kPadCost2;
      }
      const int par = k & 1;
      const bool more = k + 1 < nrows;
      // adaptive P2 of the step into row y, per path (the predecessor is
      // (x, y-1) / (x-1, y-1) / (x+1, y-1) going down, y+1 going up), both
      // lanes; columns and rows are clamped into the image: a lane whose
      // predecessor is outside restarts and ignores its penalty
      uint32_t p2v = p2x2, p2f = p2x2, p2r = p2x2;
      if (VAR && pd.guide) {
        const int yq = min(max(up ? y + 1 : y - 1, 0), H - 1);
        const uint8_t* gc = pd.guide + (size_t)y * pd.gpitch;
        const uint8_t* gq = pd.guide + (size_t)yq * pd.gpitch;
        const int cl = min(max(xlo, 0), W - 1), ch = min(max(xhi, 0), W - 1);
        const uint32_t il = __ldg(gc + cl), ih = __ldg(gc + ch);
        auto pen = [&](int dx) {
          const uint32_t ql = __ldg(gq + min(max(xlo + dx, 0), W - 1));
          const uint32_t qh = __ldg(gq + min(max(xhi + dx, 0), W - 1));
          return (uint32_t)s_lut[absdiff_u8(il, ql)] | ((uint32_t)s_lut[absdiff_u8(ih, qh)] << 16);
        };
        if (role == 0) p2v = pen(0);
        if (role != 2) p2f = pen(-1);
        if (role != 1) p2r = pen(+1);
      }
      if (role == 0) {
        // ---- owned pairs: all three paths ----
        uint32_t Nv[DC], Nf[DC], Nr[DC];
        uint32_t lv, rv, lf, rf, lr, rr;
        neighbours(Lv, lv, rv);
        neighbours(Lf, lf, rf);
        neighbours(Lr, lr, rr);
        sgm_update<DC>(Lv, Cc, lv, rv, mv, p1x2, p2v, Nv);
        sgm_update<DC>(Lf, Cc, lf, rf, mf, p1x2, p2f, Nf);
        sgm_update<DC>(Lr, Cc, lr, rr, mr, p1x2, p2r, Nr);
        mv = group_min2<CHUNKS>(tree_min<DC>(Nv), role_mask);
        mf = group_min2<CHUNKS>(tree_min<DC>(Nf), role_mask);
        mr = group_min2<CHUNKS>(tree_min<DC>(Nr), role_mask);
        // diagonal hand-over to the next row (written early)
        if (more) {
          store_u4<DC>(xfl + par * G * NT + t, NT, Nf);
          store_u4<DC>(xfr + par * G * NT + t, NT, Nr);
          if (q == 0) {
            mfl[par * NP + pr] = mf;
            mfr[par * NP + pr] = mr;
          }
        }
        // ---- accumulate and emit ----
        uint32_t S[DC];
        if (en_all) {
#pragma unroll
          for (int i = 0; i < DC; i++) S[i] = Nv[i] + Nf[i] + Nr[i];
        } else {
#pragma unroll
          for (int i = 0; i < DC; i++)
            S[i] = (en_v ? Nv[i] : 0u) + (en_fl ? Nf[i] : 0u) + (en_fr ? Nr[i] : 0u);
        }
        if (!Cfg::SEC || !second) {
          store_u4<DC>(sd_out + (size_t)y * sd_row, 1, S);
        } else {
          // add the down sweep and the horizontal paths
          uint32_t sdv[DC], hf[DC], hb[DC];
          const uint4* xs = ringx + (k % RING) * XW * NO + t;
          load_u4<DC>(sdv, xs, NO);
          bytes_to_pairs_u8<DC>(*reinterpret_cast<const V*>(xs + G * NO),
                                *reinterpret_cast<const V*>(xs + (G + 1) * NO), hf);
          bytes_to_pairs_u8<DC>(*reinterpret_cast<const V*>(xs + (G + 2) * NO),
                                *reinterpret_cast<const V*>(xs + (G + 3) * NO), hb);
#pragma unroll
          for (int i = 0; i < DC; i++) S[i] += sdv[i] + hf[i] + hb[i];
          if (pad) {
#pragma unroll
            for (int i = 0; i < DC; i++)
              if (d0 + i >= D) S[i] = 0xffffffffu;
          }
          if (pd.S) {
            // full aggregated cost, [H][W][D] uint16: eight disparities per
            // 16-byte store where the rows allow it
            if (s_vec && !pad) {
#pragma unroll
              for (int w = 0; w < DC / 8; w++) {
                const uint32_t* s8 = S + 8 * w;
                const uint4 lo4 = make_uint4(prmt(s8[0], s8[1], 0x5410u), prmt(s8[2], s8[3], 0x5410u),
                                             prmt(s8[4], s8[5], 0x5410u), prmt(s8[6], s8[7], 0x5410u));
                const uint4 hi4 = make_uint4(prmt(s8[0], s8[1], 0x7632u), prmt(s8[2], s8[3], 0x7632u),
                                             prmt(s8[4], s8[5], 0x7632u), prmt(s8[6], s8[7], 0x7632u));
                if (lo_in) *reinterpret_cast<uint4*>(pd.S + ((size_t)y * W + xlo) * D + d0 + 8 * w) = lo4;
                if (hi_in) *reinterpret_cast<uint4*>(pd.S + ((size_t)y * W + xhi) * D + d0 + 8 * w) = hi4;
              }
            } else {
#pragma unroll
              for (int i = 0; i < DC; i++) {
                if (d0 + i < D) {
                  if (lo_in) pd.S[((size_t)y * W + xlo) * D + d0 + i] = (uint16_t)(S[i] & 0xffffu);
                  if (hi_in) pd.S[((size_t)y * W + xhi) * D + d0 + i] = (uint16_t)(S[i] >> 16);
                }
              }
            }
          }
          if (pd.dint) {
            // the halo warps select the winners of this row after the barrier
            store_u4<DC>(srow + (k & 1) * G * NO + t, NO, S);
          }
        }
#pragma unroll
        for (int i = 0; i < DC; i++) Lv[i] = Nv[i];
        if (!more) {
          // band end: publish the states of the owned columns
          V va, vb;
          pairs_to_bytes<DC>(Nv, va, vb);
          if (lo_in) *reinterpret_cast<V*>(wsv + (size_t)xlo * Dp + d0) = va;
          if (hi_in) *reinterpret_cast<V*>(wsv + (size_t)xhi * Dp + d0) = vb;
          pairs_to_bytes<DC>(Nf, va, vb);
          if (lo_in) *reinterpret_cast<V*>(wsl + (size_t)xlo * Dp + d0) = va;
          if (hi_in) *reinterpret_cast<V*>(wsl + (size_t)xhi * Dp + d0) = vb;
          pairs_to_bytes<DC>(Nr, va, vb);
          if (lo_in) *reinterpret_cast<V*>(wsr + (size_t)xlo * Dp + d0) = va;
          if (hi_in) *reinterpret_cast<V*>(wsr + (size_t)xhi * Dp + d0) = vb;
        }
      } else if (role == 1) {
        // ---- left halo: the path entering from x-1 only, while one of the
        // pair's columns can still reach the strip ----
        if (more) {
          uint32_t Nf[DC];
          uint32_t lf, rf;
          neighbours(Lf, lf, rf);
          const bool act = hh + HH >= k;
          if (act) {
            sgm_update<DC>(Lf, Cc, lf, rf, mf, p1x2, p2f, Nf);
          } else {
#pragma unroll
            for (int i = 0; i < DC; i++) Nf[i] = Lf[i];
          }
          mf = group_min2<CHUNKS>(act ? tree_min<DC>(Nf) : 0u, role_mask);
          store_u4<DC>(xfl + par * G * NT + t, NT, Nf);
          if (q == 0) mfl[par * NP + pr] = mf;
        }
      } else {
        // ---- right halo: the path entering from x+1 only ----
        if (more) {
          uint32_t Nr[DC];
          uint32_t lr, rr;
          neighbours(Lr, lr, rr);
          const bool act = hh <= HALO - 1 - k;
          if (act) {
            sgm_update<DC>(Lr, Cc, lr, rr, mr, p1x2, p2r, Nr);
          } else {
#pragma unroll
            for (int i = 0; i < DC; i++) Nr[i] = Lr[i];
          }
          mr = group_min2<CHUNKS>(act ? tree_min<DC>(Nr) : 0u, role_mask);
          store_u4<DC>(xfr + par * G * NT + t, NT, Nr);
          if (q == 0) mfr[par * NP + pr] = mr;
        }
      }
      if (!more) break;
      __syncthreads();
      if (role != 2) {
        const uint4* b = xfl + par * G * NT;
        if (fl_src2 < 0) {
          load_u4<DC>(Lf, b + fl_src * CHUNKS + q, NT);
          mf = mfl[par * NP + fl_src];
        } else {
          uint32_t s1[DC], s2[DC];
          load_u4<DC>(s1, b + fl_src * CHUNKS + q, NT);
          load_u4<DC>(s2, b + fl_src2 * CHUNKS + q, NT);
#pragma unroll
          for (int i = 0; i < DC; i++) Lf[i] = prmt(s1[i], s2[i], fl_sel);
          mf = prmt(mfl[par * NP + fl_src], mfl[par * NP + fl_src2], fl_sel);
        }
      }
      if (role != 1) {
        const uint4* b = xfr + par * G * NT;
        if (fr_src2 < 0) {
          load_u4<DC>(Lr, b + fr_src * CHUNKS + q, NT);
          mr = mfr[par * NP + fr_src];
        } else {
          uint32_t s1[DC], s2[DC];
          load_u4<DC>(s1, b + fr_src * CHUNKS + q, NT);
          load_u4<DC>(s2, b + fr_src2 * CHUNKS + q, NT);
#pragma unroll
          for (int i = 0; i < DC; i++) Lr[i] = prmt(s1[i], s2[i], fr_sel);
          mr = prmt(mfr[par * NP + fr_src], mfr[par * NP + fr_src2], fr_sel);
        }
      }
      // a lane whose predecessor column is outside the image restarts
      if (fl_keep != 0xffffffffu) {
#pragma unroll
        for (int i = 0; i < DC; i++) Lf[i] &= fl_keep;
        mf &= fl_keep;
      }
      if (fr_keep != 0xffffffffu) {
#pragma unroll
        for (int i = 0; i < DC; i++) Lr[i] &= fr_keep;
        mr &= fr_keep;
      }
      select_row(k);   // halo threads; row k's costs are complete after the barrier
    }
    // ---- publish progress: the barrier orders every thread's band-end
    // stores before thread 0's release (cumulativity); the exchange buffers
    // and prefetch ring are free for the next task afterwards ----
    cp_async_wait<0>();
    __syncthreads();
    if (t == 0) st_release(flags + j, bi + 1);
    if (t == NT - 1) s_task = next_task;   // read after the barrier at the top of the loop
    select_row(nrows - 1);   // the last row of the band (its costs are in place)
  }
}

template <int DC, int CHUNKS, int HALO, int MODE, bool VAR>
cudaError_t sweep_dispatch(const SweepArgs& a, cudaStream_t s) {
  using Cfg = SweepCfg<DC, CHUNKS, HALO, MODE>;
  auto kern = sweep_kernel<DC, CHUNKS, HALO, MODE, VAR>;
  const size_t smem = Cfg::smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  // one wave of CTAs; tasks come from a queue and are claimed only by
  // running CTAs, each of which finishes its current (earlier) task before
  // the one it claimed, so no co-residency guarantee is needed
  const int grid = std::max(1, std::min(a.ntasks, per_sm * sms));
  kern<<<grid, Cfg::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, bool VAR>
cudaError_t sweep_select(const SweepArgs& a, cudaStream_t s) {
  const Shape sh = shape_for(a.Dmax, a.shape_table);
#define SF_CASE(DC_, CH_, HA_) \
  if (sh.dc == DC_ && sh.chunks == CH_ && sh.halo == HA_) return sweep_dispatch<DC_, CH_, HA_, MODE, VAR>(a, s);
  SF_SWEEP_SHAPES(SF_CASE)
#undef SF_CASE
  return cudaErrorInvalidConfiguration;
}

// One launch of the sweeps in launch mode `mode` (0 down, 1 up, 2 merged).
template <bool VAR>
cudaError_t sweep_launch(const SweepArgs& a, int mode, cudaStream_t s) {
  switch (mode) {
    case kModeDown: return sweep_select<kModeDown, VAR>(a, s);
    case kModeUp: return sweep_select<kModeUp, VAR>(a, s);
    case kModeMergedH: return sweep_select<kModeMergedH, VAR>(a, s);
    default: return sweep_select<kModeMerged, VAR>(a, s);
  }
}

}  // namespace

}  // namespace fused
}  // namespace sf
