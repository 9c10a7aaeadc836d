// Host/device interface of the fused SGM kernels (sgm_fused.cu).
#pragma once

#include <algorithm>

#include "sf_internal.cuh"

namespace sf {
namespace fused {

constexpr int kTW = 32;     // owned columns per strip
constexpr int kMaxPass = 4;

// Launch shape chosen by D: a thread owns DC disparities of two lines; the
// disparities of a line pair are spread over `chunks` consecutive threads (a
// power of two); the band sweeps carry `halo` extra columns on each side of
// a strip and walk bands of halo + 1 rows.  `order` schedules the paths:
// 0 = the horizontal paths' launch, the down sweep's, then the up sweep's;
// 1 = the horizontal paths' launch, then both scan orders in one launch,
// meeting in the middle; 2 = everything in one launch (the horizontal paths'
// row blocks first in its queue).
struct Shape {
  int dc, chunks, halo, order;
};
// Tables of tuned overrides: the plain calls' and the learned calls' (their
// launches carry the left passes alone, half the work in flight).
// kShapeBuiltin asks for the built-in rule whatever is tuned.
constexpr int kShapeBuiltin = -1, kShapePlain = 0, kShapeLearned = 1;
// built-in rule unless an override of `table` covers D
Shape shape_for(int D, int table = kShapePlain);
bool shape_supported(int dc, int chunks, int halo);
int set_shape_override(int table, int d_lo, int d_hi, int dc, int halo, int order);   // 0 = ok
inline int padded_d(int D) { return ((D + 15) / 16) * 16; }
// Rows per block of the horizontal paths run inside a merged launch (launch
// mode 3) by its CTAs of (16 + halo) x chunks threads: above 64 disparities
// a warp per line pair, when the CTA is whole warps, as in the standalone
// walk; otherwise the sweep's own thread layout, 16 + halo line pairs.
__host__ __device__ constexpr int merged_hline_rows(int dc, int chunks, int halo) {
  return ((16 + halo) * chunks % 32 == 0 && dc * chunks > 64) ? 2 * ((16 + halo) * chunks / 32)
                                                                : 2 * (16 + halo);
}
inline int band_rows(int D, int table = kShapePlain) { return shape_for(D, table).halo + 1; }

// One stereo pass (one reference image) of the band sweeps and the
// horizontal paths: its sizes and buffers.
struct PassDesc {
  int W, H, D, Dp, J, nb;
  const uint8_t* cost;   // [H][W][Dp] uint8, this pass's reference image
  uint8_t* hfwd;         // [H][W][Dp] uint8, L of path (+1,0)
  uint8_t* hbwd;         // [H][W][Dp] uint8, L of path (-1,0)
  uint32_t* sdown;       // tile layout [H][J][16][chunks][dc] u32
  uint8_t* bs;           // band-end states [2 orders][2][3][W][Dp] u8
  int* flags_down;       // [J] bands completed by the down sweep
  int* flags_up;         // [J] bands completed by the up sweep
  int* flags_h;          // [2][ceil(H / 16)] row blocks of the horizontal paths done (merged launch with them)
  int16_t* dint;         // winner per pixel (up sweep), or nullptr
  float* dsub;           // subpixel winner (up sweep), or nullptr
  uint16_t* S;           // full aggregated cost [H][W][D] (up sweep), or nullptr
  const uint8_t* guide;  // reference image [H][gpitch] for the intensity-adaptive P2, or nullptr
  int gpitch;
};

struct HLineArgs {
  int P1, P2, Dmax, npass, nblocks;   // P2: the constant P2, or the base of the adaptive one
  int block_rows;              // rows per block: hline_block_rows(Dmax) when the blocks were counted
  int shape_table;             // kShapePlain, kShapeLearned or kShapeBuiltin
  uint32_t path_mask;
  int uniform_blocks;          // > 0: every pass has this many blocks
  const int* block_prefix;     // otherwise: first block of each pass [npass + 1]
  int* err;                    // set to 1 when a bounded copy wait gives up
  PassDesc inl[kMaxPass];      // descriptors in the parameter block (pass_ptr == nullptr)
  const PassDesc* pass_ptr;    // descriptors in device memory
};

struct SweepArgs {
  int P1, P2, subpixel, Dmax, npass, ntasks;
  int unique;                  // uniqueness ratio (percent) of the winners with a subpixel output, 0 = off
  int hl_tasks, hl_blocks;     // launch mode 3: horizontal-path tasks at the queue head, row blocks per direction
  int variants;                // 1: adaptive P2 or uniqueness requested (the kernels that compile them in)
  int shape_table;             // kShapePlain, kShapeLearned or kShapeBuiltin
  uint32_t path_mask;
  int en_h0, en_h1;
  int uniform_items;           // > 0: all passes alike, tasks per band
  const int* band_start;       // otherwise: first task of each band [nbands + 1]
  const int* band_npass;       // passes (sorted by band count, descending) active in a band
  const int* prefixJ;          // strip-count prefix over those passes [npass + 1]
  int nbands;
  int* task_counter;           // next task of the queue (zeroed before the launch)
  int* err;                    // set to 1 when a bounded wait gives up
  long long spin_limit;
  PassDesc inl[kMaxPass];
  const PassDesc* pass_ptr;
};

// per-pass buffer sizes (the shape is the launch's, chosen from its largest D)
inline size_t sdown_bytes(int W, int H, int Dshape, int table = kShapePlain) {
  const int J = (W + kTW - 1) / kTW;
  const Shape s = shape_for(Dshape, table);
  return (size_t)H * J * 16 * s.chunks * s.dc * sizeof(uint32_t);
}
inline size_t bs_bytes(int W, int D) { return (size_t)2 * 2 * 3 * W * padded_d(D); }
inline size_t cost_pair_smem(int W, int D) {
  return 2 * ((size_t)W * 8 + (size_t)((W + 3) / 4) * 32) + (size_t)W * (padded_d(D) + 4);
}
// rows whose census pair + distances exceed this use per-reference x-tiles
constexpr size_t kCostPairSmemMax = 227u * 1024u;

// Census strings and cost volumes of up to kMaxPass stereo pairs of one
// size: one persistent launch over the rows of all of them.
struct CostPairs {
  int npairs;
  const uint64_t* cL[kMaxPass];
  const uint64_t* cR[kMaxPass];
  uint8_t* CL[kMaxPass];
  uint8_t* CR[kMaxPass];     // nullptr in launch_cost_left
};
cudaError_t launch_cost_pair(const CostPairs& job, int W, int H, int D, int Dp, int cmax, cudaStream_t s);
// left-reference volumes only
cudaError_t launch_cost_left(const CostPairs& job, int W, int H, int D, int Dp, int cmax, cudaStream_t s);
cudaError_t launch_hline(const HLineArgs& a, cudaStream_t s);
// disparities per thread of the horizontal paths for D > 64 (16 or 32; 0 = ok)
int set_hline_dc(int dc);
// rows per block of the horizontal-path kernel for a launch of depth Dmax
int hline_block_rows(int Dmax);
// mode 0: down sweep, 1: up sweep, 2: both orders in one launch, 3: mode 2
// with the horizontal paths' row blocks at the head of its queue
cudaError_t launch_sweep(const SweepArgs& a, int mode, cudaStream_t s);
// the kernels without / with the SGM variants (sgm_sweep.cu, sgm_sweep_var.cu)
cudaError_t launch_sweep_plain(const SweepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_sweep_variants(const SweepArgs& a, int mode, cudaStream_t s);

}  // namespace fused
}  // namespace sf
