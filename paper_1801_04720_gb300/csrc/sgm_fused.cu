// Fused SGM stereo for the scene-flow hot path (Sec. 3.1 of arXiv 1801.04720:
// SGM with eight paths and a left-right check), GB300 layout.
//
// Stages for one stereo pair (left image L, right image R):
//   1. cost_pair_kernel: every Hamming distance between census strings of the
//      same image row with 0 <= xL - xR < D is computed ONCE (one row per CTA,
//      held in shared memory) and written twice: as the left-reference volume
//      C_L[y][x][d] = H(cL(x), cR(x-d)) and the right-reference volume
//      C_R[y][x][d] = H(cR(x), cL(x+d)).  POPC runs at a quarter of the
//      integer rate, so sharing the distances between both passes halves it.
//      Rows whose W x (Dp + 16) bytes exceed one CTA's shared memory take
//      cost_tiled_kernel instead: one launch per reference image, x-tiles.
//      The learned path needs C_L alone: the same kernel then writes each
//      row's distances straight to C_L, without the shared-memory band.
//   2. hline_kernel: the two horizontal paths (+1,0) and (-1,0), each row an
//      independent line; two rows share a register (u16x2 lanes).  Writes
//      L_r as uint8 volumes.  Runs before the down sweep.
//   3. sweep_kernel<DOWN>: paths (0,+1), (+1,+1), (-1,+1) walking the image
//      top to bottom in bands of halo+1 rows.  A task is one band of one
//      32-column strip of one pass; the diagonal paths enter a strip from its
//      neighbours, so the band is computed on a trapezoid with `halo` extra
//      columns per side, started from the neighbours' band-end states (global
//      memory, published with release/acquire flags; waits are bounded).
//      Writes the partial sum S_down in a tile layout.
//   4. sweep_kernel<UP>: paths (0,-1), (-1,-1), (+1,-1) bottom to top, adds
//      S_down and both horizontal paths, and fuses winner-take-all and the
//      parabolic subpixel step (or writes the full aggregated cost).
//   3+4. sweep_kernel<MERGED>: both scan orders in one launch, meeting in
//      the middle: each band is finished (sums and selection) by whichever
//      order reaches it second, so twice as many band tasks can run at once.
// Tasks come from a band-major queue, so the sweep time is the band chain
// (bands x per-band latency); each task is spread over many threads to keep
// that latency short.  All arithmetic is exact integer math in 16-bit lanes
// (L_r <= cmax + P2, S <= 8 (cmax + P2) < 2^16).
#include "sf_sweep.cuh"



namespace sf {
namespace fused {

namespace {


// ---------------------------------------------------------------------------
// 1. cost volumes of a stereo pair
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024, 1)
    cost_pair_kernel(const CostPairs job, int W, int H, int D, int Dp, int cmax) {
  extern __shared__ __align__(16) uint8_t smem[];
  // per census buffer (two, the next row's arriving while this row is
  // computed): the left census row, then the right one split by index mod 4
  // (srt[j & 3][j >> 2]) so that lanes reading cR(x - 4 lane - k) hit
  // consecutive words.  Then the distances H(cL(x), cR(x-d)) as rows
  // [W][Ds]; 4 padding bytes per row spread the diagonal reads of the
  // right-reference pass over the banks.  With CR == nullptr (the left
  // volume only) each row's distances go straight to C_L and no band is used.
  // One launch walks the rows of every pair of the job (row r: pair r / H),
  // so the persistent CTAs share them evenly.
  const bool left_only = job.CR[0] == nullptr;
  const int nrows = job.npairs * H;
  const int Q = (W + 3) >> 2;
  const int cw = W + 4 * Q;   // 8-byte words per census buffer
  uint64_t* cbuf = reinterpret_cast<uint64_t*>(smem);
  uint8_t* band = reinterpret_cast<uint8_t*>(cbuf + 2 * cw);
  const int Ds = Dp + 4;
  const int groups = Dp >> 2;   // 4 disparities per lane and step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto fetch = [&](int row, int buf) {
    const int k = row / H, y = row - k * H;
    const uint64_t* cL = job.cL[k];
    const uint64_t* cR = job.cR[k];
    uint64_t* sl = cbuf + buf * cw;
    uint64_t* srt = sl + W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
      cp_async<8>(sl + i, cL + (size_t)y * W + i, true);
      cp_async<8>(srt + (i & 3) * Q + (i >> 2), cR + (size_t)y * W + i, true);
    }
    cp_async_commit();
  };
  int buf = 0;
  if (blockIdx.x < nrows) fetch(blockIdx.x, 0);
  for (int row = blockIdx.x; row < nrows; row += gridDim.x, buf ^= 1) {
    const int pk = row / H, y = row - pk * H;
    uint8_t* const CL = job.CL[pk];
    uint8_t* const CR = job.CR[pk];
    cp_async_wait<0>();
    __syncthreads();   // this row's census is in; the band is free
    if (row + (int)gridDim.x < nrows) fetch(row + gridDim.x, buf ^ 1);
    const uint64_t* sl = cbuf + buf * cw;
    const uint64_t* srt = sl + W;
    // right pixel j = x - 4g - k sits at srt[(x-k) & 3][((x-k) >> 2) - g]; a
    // warp's columns step by nw (a multiple of 4), which leaves (x-k) & 3
    // unchanged and adds nw / 4 to (x-k) >> 2
    int base[4];
#pragma unroll
    for (int k = 0; k < 4; k++) base[k] = ((warp - k) & 3) * Q + ((warp - k) >> 2);
    for (int x = warp; x < W; x += nw) {
      const uint64_t a = sl[x];
      uint32_t* dst = left_only ? reinterpret_cast<uint32_t*>(CL + ((size_t)y * W + x) * Dp)
                                : reinterpret_cast<uint32_t*>(band + x * Ds);
      // every candidate of this column exists (warp-uniform): no checks
      const bool full = D == Dp && x >= Dp - 1;
      for (int g = lane; g < groups; g += 32) {
        const int d0 = 4 * g;
        uint32_t packed = 0;
        if (full) {
#pragma unroll
          for (int k = 0; k < 4; k++) packed |= (uint32_t)__popcll(a ^ srt[base[k] - g]) << (8 * k);
        } else {
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const bool ok = d0 + k < D && d0 + k <= x;
            // (index 0 where there is no candidate: every address stays in the row)
            const uint64_t b = srt[ok ? base[k] - g : 0];
            const uint32_t c = ok ? (uint32_t)__popcll(a ^ b) : (uint32_t)cmax;
            packed |= c << (8 * k);
          }
        }
        dst[g] = packed;
      }
#pragma unroll
      for (int k = 0; k < 4; k++) base[k] += nw >> 2;
    }
    if (left_only) continue;
    __syncthreads();
    // left-reference row: the rows of the band; right-reference row:
    // C_R(x, d) = band[x + d][d], or cmax past the edge
    uint32_t* dl = reinterpret_cast<uint32_t*>(CL + (size_t)y * W * Dp);
    uint32_t* dr = reinterpret_cast<uint32_t*>(CR + (size_t)y * W * Dp);
    for (int x = warp; x < W; x += nw) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(band + x * Ds);
      const int diag = x * Ds;   // band[x + d][d] = band[diag + d (Ds + 1)]
      const bool inside = x + Dp <= W;   // the whole diagonal is in the row (warp-uniform)
      for (int g = lane; g < groups; g += 32) {
        dl[x * groups + g] = src[g];
        const int d0 = 4 * g;
        const int o0 = diag + d0 * (Ds + 1);
        uint32_t packed = 0;
        if (inside) {
#pragma unroll
          for (int k = 0; k < 4; k++) packed |= (uint32_t)band[o0 + k * (Ds + 1)] << (8 * k);
        } else {
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const bool in = x + d0 + k < W;
            const uint32_t v = band[in ? o0 + k * (Ds + 1) : 0];
            packed |= (in ? v : (uint32_t)cmax) << (8 * k);
          }
        }
        dr[x * groups + g] = packed;
      }
    }
  }
  cp_async_wait<0>();
}

// Rows too wide for one CTA's shared memory (W x Dp > ~200 KB): each
// reference volume is computed on its own from x-tiles of census strings.
constexpr int kCostTileX = 64;

__global__ void __launch_bounds__(256)
    cost_tiled_kernel(const uint64_t* __restrict__ cref, const uint64_t* __restrict__ coth, int W,
                      int H, int D, int Dp, int cmax, int ref_is_right, uint8_t* __restrict__ out) {
  __shared__ uint64_t sref[kCostTileX];
  __shared__ uint64_t soth[kCostTileX + SF_MAX_DISPARITY];
  const int y = blockIdx.y;
  const int xs = blockIdx.x * kCostTileX;
  const int nx = min(kCostTileX, W - xs);
  const int o_lo = ref_is_right ? xs : xs - (Dp - 1);   // candidate columns [o_lo, o_lo + nx + Dp - 1)
  for (int i = threadIdx.x; i < nx; i += blockDim.x) sref[i] = cref[(size_t)y * W + xs + i];
  for (int i = threadIdx.x; i < nx + Dp - 1; i += blockDim.x) {
    const int xo = o_lo + i;
    soth[i] = (xo >= 0 && xo < W) ? coth[(size_t)y * W + xo] : 0ull;
  }
  __syncthreads();
  const int groups = Dp / 4;
  uint32_t* row = reinterpret_cast<uint32_t*>(out + ((size_t)y * W + xs) * Dp);
  for (int i = threadIdx.x; i < nx * groups; i += blockDim.x) {
    const int px = i / groups, d0 = (i - px * groups) * 4;
    const int x = xs + px;
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int d = d0 + k;
      const int xo = ref_is_right ? x + d : x - d;
      const uint32_t c = (d < D && xo >= 0 && xo < W) ? (uint32_t)__popcll(sref[px] ^ soth[xo - o_lo])
                                                       : (uint32_t)cmax;
      packed |= c << (8 * k);
    }
    row[i] = packed;
  }
}

// ---------------------------------------------------------------------------
// 2. horizontal paths
// ---------------------------------------------------------------------------
// A CTA walks PAIRS line pairs (two rows per register) of one pass in one
// direction (hline_rows, sf_sweep.cuh): 8 pairs (16 rows, 56 KB tiles) with
// chunks of 8, 16 or 32 disparities a thread; 2 pairs (4 rows, 16 KB tiles)
// with a warp per line pair, so that many small blocks spread the rows
// evenly over the SMs.  The merged sweep launch can run the same walk as
// tasks of its own queue.
constexpr int kHlinePairs = 8;
constexpr int kHlineTileBytes = 56 * 1024;     // one buffer (two CTAs fit an SM)
constexpr int kHlineWarpPairs = 2;
constexpr int kHlineWarpTileBytes = 16 * 1024;

template <int DC, int CHUNKS, int PAIRS, int TILE>
__global__ void __launch_bounds__(PAIRS * CHUNKS)
    hline_kernel(const __grid_constant__ HLineArgs a) {
  constexpr int kRows = 2 * PAIRS;
  extern __shared__ __align__(128) uint8_t hsmem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_fail;
  __shared__ uint16_t s_lut[256];
  // block -> (pass, direction, 16-row block); passes listed by prefix of
  // their block counts (2 directions x row blocks)
  int p = 0;
  {
    int lo = 0, hi = a.npass - 1;
    const int blk = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      const int start = a.block_prefix ? a.block_prefix[mid] : mid * a.uniform_blocks;
      if (start <= blk) lo = mid; else hi = mid - 1;
    }
    p = lo;
  }
  const PassDesc pd = a.pass_ptr ? a.pass_ptr[p] : a.inl[p];   // by value: fields in registers
  const int nrb = (pd.H + kRows - 1) / kRows;
  const int rem = blockIdx.x - (a.block_prefix ? a.block_prefix[p] : p * a.uniform_blocks);
  const int dir = rem / nrb;                 // 0: (+1,0), 1: (-1,0)
  const int rb = rem - dir * nrb;
  if (!((a.path_mask >> dir) & 1u)) return;  // whole CTA: direction disabled
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (pd.guide) fill_p2_table(s_lut, a.P1, a.P2);
  int ph[2] = {0, 0};
  hline_rows<DC, CHUNKS, true>(pd, dir, rb * kRows, PAIRS, a.P1, a.P2, hsmem, TILE, bars,
                               &s_fail, s_lut, ph, a.err);
}

}  // namespace

cudaError_t launch_cost_left(const CostPairs& job, int W, int H, int D, int Dp, int cmax, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COST, s);
  if (job.npairs < 1 || job.npairs > kMaxPass) return cudaErrorInvalidValue;
  CostPairs jl = job;
  for (int k = 0; k < kMaxPass; k++) jl.CR[k] = nullptr;
  // the persistent kernel without its band: two census rows in shared memory
  const size_t smem = 2 * ((size_t)W + 4 * (size_t)((W + 3) / 4)) * sizeof(uint64_t);
  if (smem > kCostPairSmemMax) {
    count_launches(job.npairs);
    dim3 grid((W + kCostTileX - 1) / kCostTileX, H);
    for (int k = 0; k < job.npairs; k++)
      cost_tiled_kernel<<<grid, 256, 0, s>>>(job.cL[k], job.cR[k], W, H, D, Dp, cmax, 0, job.CL[k]);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(cost_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  count_launches(1);
  cost_pair_kernel<<<std::min(job.npairs * H, sms), 1024, smem, s>>>(jl, W, H, D, Dp, cmax);
  return cudaGetLastError();
}

cudaError_t launch_cost_pair(const CostPairs& job, int W, int H, int D, int Dp, int cmax, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COST, s);
  if (job.npairs < 1 || job.npairs > kMaxPass) return cudaErrorInvalidValue;
  for (int k = 0; k < job.npairs; k++)
    if (!job.CR[k]) return cudaErrorInvalidValue;
  const size_t smem = cost_pair_smem(W, D);
  if (smem > kCostPairSmemMax) {
    count_launches(2 * job.npairs);
    dim3 grid((W + kCostTileX - 1) / kCostTileX, H);
    for (int k = 0; k < job.npairs; k++) {
      cost_tiled_kernel<<<grid, 256, 0, s>>>(job.cL[k], job.cR[k], W, H, D, Dp, cmax, 0, job.CL[k]);
      cost_tiled_kernel<<<grid, 256, 0, s>>>(job.cR[k], job.cL[k], W, H, D, Dp, cmax, 1, job.CR[k]);
    }
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(cost_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  count_launches(1);
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  cost_pair_kernel<<<std::min(job.npairs * H, sms), 1024, smem, s>>>(job, W, H, D, Dp, cmax);
  return cudaGetLastError();
}

template <int DC, int CHUNKS, int PAIRS = kHlinePairs, int TILE = kHlineTileBytes>
static cudaError_t hline_dispatch(const HLineArgs& a, cudaStream_t s) {
  if (a.block_rows != 2 * PAIRS) return cudaErrorInvalidValue;   // blocks counted for another walk
  const size_t smem = 2 * (size_t)TILE;
  cudaError_t e = cudaFuncSetAttribute(hline_kernel<DC, CHUNKS, PAIRS, TILE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (a.nblocks <= 0) return cudaSuccess;
  hline_kernel<DC, CHUNKS, PAIRS, TILE><<<a.nblocks, PAIRS * CHUNKS, smem, s>>>(a);
  return cudaGetLastError();
}

// Disparities per thread of the horizontal paths above D = 64.  4 (the
// default) gives a whole warp to a line pair (4 disparities a lane up to
// D = 128, 8 up to 256): a step's minimum is one warp-wide reduction per
// 16-bit lane, and the launch has four times the warps of 16-wide chunks.
// 16 (eight threads per line pair, three shuffle levels per step's minimum)
// and 32 (four threads, two levels, one warp per block) leave too few warps
// to cover each step's latency.  On the 1242 x 375, D = 128 frame: 0.03 ms
// less per plain frame and 0.12 ms less per learned frame than 16.
int g_hline_dc = 4;

int hline_block_rows(int Dmax) {
  return (g_hline_dc == 4 && Dmax > 64) ? 2 * kHlineWarpPairs : 2 * kHlinePairs;
}

int set_hline_dc(int dc) {
  if (dc != 4 && dc != 16 && dc != 32) return 1;
  g_hline_dc = dc;
  return 0;
}

cudaError_t launch_hline(const HLineArgs& a, cudaStream_t s) {
  StageTrace trace(SF_STAGE_AGGREGATE, s);
  count_launches(1);
  // the horizontal volumes do not depend on the sweeps' shape.  Each step of
  // a line waits for the minimum over its chunk group, so the walk is
  // latency bound (g_hline_dc: the chunk width).
  // A thread moves DC bytes of every pixel it walks, so DC must divide the
  // padded depth Dp of every pass (a multiple of 16): 32-wide chunks only
  // for passes of one size with Dp % 32 == 0 (a batch launch mixes depths),
  // and only above D = 64 (four 16-wide chunks already cover smaller D).
  if (a.block_rows == 2 * kHlineWarpPairs) {
    // a warp per line pair; lanes past a pass's depth carry padding costs
    if (a.Dmax <= 128) return hline_dispatch<4, 32, kHlineWarpPairs, kHlineWarpTileBytes>(a, s);
    return hline_dispatch<8, 32, kHlineWarpPairs, kHlineWarpTileBytes>(a, s);
  }
  bool wide = a.Dmax > 64 && a.pass_ptr == nullptr && a.npass >= 1;
  for (int k = 0; wide && k < a.npass; k++) wide = a.inl[k].Dp % 32 == 0;
  Shape sh;
  sh.dc = wide ? g_hline_dc : 16;
  sh.chunks = sh.dc == 8 ? 2 : 4;
  while (sh.chunks * sh.dc < a.Dmax) sh.chunks <<= 1;
  sh.halo = 0;
  if (sh.dc == 32) {
    switch (sh.chunks) {
      case 4: return hline_dispatch<32, 4>(a, s);
      default: return hline_dispatch<32, 8>(a, s);
    }
  }
  if (sh.dc == 16) {
    switch (sh.chunks) {
      case 4: return hline_dispatch<16, 4>(a, s);
      case 8: return hline_dispatch<16, 8>(a, s);
      default: return hline_dispatch<16, 16>(a, s);
    }
  }
  switch (sh.chunks) {
    case 2: return hline_dispatch<8, 2>(a, s);
    case 4: return hline_dispatch<8, 4>(a, s);
    case 8: return hline_dispatch<8, 8>(a, s);
    default: return hline_dispatch<8, 16>(a, s);
  }
}

// ---- kernel shape choice (built-in rule, or a tuned override per D class) ----
namespace {
struct ShapeOverride {
  int lo, hi, dc, halo, order;
};
ShapeOverride g_over[2][16];   // [table]
int g_nover[2] = {0, 0};
}  // namespace

// chunks of dc disparities covering D, at least two (owned pairs then fill
// whole warps)
static int chunks_for(int dc, int D) {
  int c = 2;
  while (c * dc < D) c <<= 1;
  return c;
}

// Built-in rule: both scan orders in one launch with 16 disparities per
// thread and bands of 9 rows (two CTAs per SM up to D = 128; measured the
// fastest at 1242 x 375, D = 128 on GB300: 1.38 ms a frame against 1.58 ms
// for the best two-launch shape); 8 disparities per thread up to D = 32.
static Shape builtin_shape(int D) {
  Shape s;
  s.dc = D > 32 ? 16 : 8;
  s.chunks = chunks_for(s.dc, D);
  s.halo = 8;
  s.order = 1;
  return s;
}

bool shape_supported(int dc, int chunks, int halo) {
#define SF_SUP(DC_, CH_, HA_) \
  if (dc == DC_ && chunks == CH_ && halo == HA_) return true;
  SF_SWEEP_SHAPES(SF_SUP)
#undef SF_SUP
  return false;
}

Shape shape_for(int D, int table) {
  const ShapeOverride* ov = table >= 0 ? g_over[table] : nullptr;
  for (int i = table >= 0 ? g_nover[table] - 1 : -1; i >= 0; i--) {
    if (D >= ov[i].lo && D <= ov[i].hi) {
      Shape s;
      s.dc = ov[i].dc;
      s.halo = ov[i].halo;
      s.order = ov[i].order;
      s.chunks = chunks_for(s.dc, D);
      return s;
    }
  }
  return builtin_shape(D);
}

int set_shape_override(int table, int d_lo, int d_hi, int dc, int halo, int order) {
  if (table < 0 || table > 1) return 1;
  if (d_lo < 1 || d_hi > SF_MAX_DISPARITY || d_lo > d_hi) return 1;
  ShapeOverride* ov = g_over[table];
  int& n = g_nover[table];
  if (dc == 0) {   // drop overrides of this class
    int w = 0;
    for (int i = 0; i < n; i++)
      if (!(ov[i].lo == d_lo && ov[i].hi == d_hi)) ov[w++] = ov[i];
    n = w;
    return 0;
  }
  if (order < 0 || order > 2) return 1;
  for (int D = d_lo; D <= d_hi; D++)
    if (!shape_supported(dc, chunks_for(dc, D), halo)) return 1;
  if (n == 16) return 1;
  ov[n++] = {d_lo, d_hi, dc, halo, order};
  return 0;
}

cudaError_t launch_sweep(const SweepArgs& a, int mode, cudaStream_t s) {
  StageTrace trace(SF_STAGE_SGM_SWEEP, s);
  count_launches(1);
  return a.variants ? launch_sweep_variants(a, mode, s) : launch_sweep_plain(a, mode, s);
}

}  // namespace fused
}  // namespace sf
