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
//   2. hline_kernel: the two horizontal paths (+1,0) and (-1,0), each row an
//      independent line; two rows share a register (u16x2 lanes).  Writes
//      L_r as uint8 volumes.
//   3. sweep_kernel<DOWN>: paths (0,+1), (+1,+1), (-1,+1) walking the image
//      top to bottom in bands of TH rows.  Each CTA owns a strip of 32
//      columns; the diagonal paths enter a strip from its neighbours, so the
//      band is computed on a trapezoid with TH-1 halo columns per side from
//      the neighbours' band-end states (global memory, published with
//      release/acquire flags; waits are bounded).  Writes the partial sum
//      S_down in a tile layout.
//   4. sweep_kernel<UP>: paths (0,-1), (-1,-1), (+1,-1) bottom to top, adds
//      S_down and both horizontal paths, and fuses winner-take-all and the
//      parabolic subpixel step (or writes the full aggregated cost).
// All arithmetic is exact integer math in 16-bit lanes (L_r <= cmax + P2,
// S <= 8 (cmax + P2) < 2^16).
#include <cooperative_groups.h>

#include "sf_fused.cuh"
#include "sgm_common.cuh"

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

// ---------------------------------------------------------------------------
// 1. cost volumes of a stereo pair
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512)
    cost_pair_kernel(const uint64_t* __restrict__ cL, const uint64_t* __restrict__ cR, int W, int H,
                     int D, int Dp, int cmax, uint8_t* __restrict__ CL, uint8_t* __restrict__ CR) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* sl = reinterpret_cast<uint64_t*>(smem);
  uint64_t* sr = sl + W;
  uint8_t* band = reinterpret_cast<uint8_t*>(sr + W);  // [W][Dp]: H(cL(x), cR(x-d))
  const int y = blockIdx.x;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    sl[i] = cL[(size_t)y * W + i];
    sr[i] = cR[(size_t)y * W + i];
  }
  __syncthreads();
  // all distances of this row, four disparities per thread iteration
  const int groups = Dp / 4;
  for (int i = threadIdx.x; i < W * groups; i += blockDim.x) {
    const int x = i / groups, d0 = (i - x * groups) * 4;
    const uint64_t a = sl[x];
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int d = d0 + k;
      const int xr = x - d;
      const uint32_t c = (d < D && xr >= 0) ? (uint32_t)__popcll(a ^ sr[xr]) : (uint32_t)cmax;
      packed |= c << (8 * k);
    }
    *reinterpret_cast<uint32_t*>(band + (size_t)x * Dp + d0) = packed;
  }
  __syncthreads();
  // left-reference row: a straight copy
  {
    const uint4* src = reinterpret_cast<const uint4*>(band);
    uint4* dst = reinterpret_cast<uint4*>(CL + (size_t)y * W * Dp);
    for (int i = threadIdx.x; i < W * Dp / 16; i += blockDim.x) dst[i] = src[i];
  }
  // right-reference row: C_R(x, d) = band[x + d][d], or cmax past the edge
  {
    uint32_t* dst = reinterpret_cast<uint32_t*>(CR + (size_t)y * W * Dp);
    for (int i = threadIdx.x; i < W * groups; i += blockDim.x) {
      const int x = i / groups, d0 = (i - x * groups) * 4;
      uint32_t packed = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int d = d0 + k;
        const int xl = x + d;
        const uint32_t c = (xl < W) ? (uint32_t)band[(size_t)xl * Dp + d] : (uint32_t)cmax;
        packed |= c << (8 * k);
      }
      dst[i] = packed;
    }
  }
}

// ---------------------------------------------------------------------------
// 2. horizontal paths
// ---------------------------------------------------------------------------
template <int CHUNKS>
__global__ void __launch_bounds__(256)
    hline_kernel(HLineArgs a) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int item = gt / CHUNKS;
  const int q = gt - item * CHUNKS;
  const int rows2 = (a.H + 1) / 2;
  const int per_pass = rows2 * 2;
  const bool active = item < a.npass * per_pass;
  const int p = active ? item / per_pass : 0;
  const int rem = item - p * per_pass;
  const int dir = rem / rows2;           // 0: (+1,0), 1: (-1,0)
  const int rp = rem - dir * rows2;
  const int y0 = 2 * rp, y1 = min(2 * rp + 1, a.H - 1);
  const int W = a.W, Dp = a.Dp;
  // chunks at or past the padded depth hold no data (D not a power of two)
  const bool enabled = active && ((a.path_mask >> dir) & 1u) && q * kDC < Dp;
  const uint8_t* C = a.cost[p];
  uint8_t* out = dir == 0 ? a.hfwd[p] : a.hbwd[p];
  const int d0 = q * kDC;
  const bool pad = d0 + kDC > a.D;
  const uint32_t p1x2 = a.P1 * 0x10001u, p2x2 = a.P2 * 0x10001u;
  uint32_t L[kDC], Cr[kDC], N[kDC];
#pragma unroll
  for (int i = 0; i < kDC; i++) L[i] = 0;
  uint32_t m = 0;
  const int step = dir == 0 ? 1 : -1;
  int x = dir == 0 ? 0 : W - 1;
  // prefetch the first column's costs
  uint4 ca = make_uint4(0, 0, 0, 0), cb = ca;
  if (enabled) {
    ca = __ldg(reinterpret_cast<const uint4*>(C + ((size_t)y0 * W + x) * Dp + d0));
    cb = __ldg(reinterpret_cast<const uint4*>(C + ((size_t)y1 * W + x) * Dp + d0));
  }
  for (int s = 0; s < W; s++, x += step) {
    bytes_to_pairs(ca, cb, Cr);
    if (pad) {
#pragma unroll
      for (int i = 0; i < kDC; i++)
        if (d0 + i >= a.D) Cr[i] = kPadCost2;
    }
    if (enabled && s + 1 < W) {
      const int xn = x + step;
      ca = __ldg(reinterpret_cast<const uint4*>(C + ((size_t)y0 * W + xn) * Dp + d0));
      cb = __ldg(reinterpret_cast<const uint4*>(C + ((size_t)y1 * W + xn) * Dp + d0));
    }
    uint32_t left = __shfl_up_sync(0xffffffffu, L[kDC - 1], 1, CHUNKS);
    uint32_t right = __shfl_down_sync(0xffffffffu, L[0], 1, CHUNKS);
    if (q == 0) left = (s == 0) ? 0u : kInf2;
    if (q == CHUNKS - 1) right = (s == 0) ? 0u : kInf2;
    const uint32_t acc = sgm_step16(L, Cr, left, right, m, p1x2, p2x2, N);
    m = group_min2<CHUNKS>(acc);
#pragma unroll
    for (int i = 0; i < kDC; i++) L[i] = N[i];
    if (enabled) {
      uint4 oa, ob;
      pairs_to_bytes(N, oa, ob);
      *reinterpret_cast<uint4*>(out + ((size_t)y0 * W + x) * Dp + d0) = oa;
      if (y1 != y0) *reinterpret_cast<uint4*>(out + ((size_t)y1 * W + x) * Dp + d0) = ob;
    }
  }
}

// ---------------------------------------------------------------------------
// 3./4. band sweeps
// ---------------------------------------------------------------------------
// Thread layout: t = pair * CHUNKS + q.  Pairs 0..15 own columns
// (x0 + c, x0 + 16 + c); pairs 16 .. 16+HALO-1 are halo pairs
// (x0 - HALO + h, x1 + h) carrying the diagonal paths into the strip.
// FL = the diagonal path fed from column x-1 ((+1,+1) down, (+1,-1) up),
// FR = the one fed from column x+1 ((-1,+1) down, (-1,-1) up).
template <int CHUNKS, bool UP>
__global__ void __launch_bounds__((16 + kHalo) * CHUNKS)
    sweep_kernel(SweepArgs a) {
  constexpr int NP = 16 + kHalo;
  constexpr int NT = NP * CHUNKS;
  constexpr int TH = kHalo + 1;
  extern __shared__ __align__(16) uint8_t smem[];
  // exchange buffers [parity][pair][chunk][16] for FL and FR, and pair mins
  uint32_t* xfl = reinterpret_cast<uint32_t*>(smem);
  uint32_t* xfr = xfl + 2 * NT * kDC;
  uint32_t* mfl = xfr + 2 * NT * kDC;     // [parity][pair]
  uint32_t* mfr = mfl + 2 * NP;
  uint32_t* srow = mfr + 2 * NP;          // [pair 0..15][chunk][16] (UP selection)
  __shared__ int s_abort;

  const int t = threadIdx.x;
  const int pr = t / CHUNKS;
  const int q = t - pr * CHUNKS;
  const bool owned = pr < 16;
  const int W = a.W, H = a.H, Dp = a.Dp, J = a.J;
  const int d0 = q * kDC;
  const bool pad = d0 + kDC > a.D;
  const bool live = d0 < Dp;   // chunks past the padded depth hold no data
  const uint32_t p1x2 = a.P1 * 0x10001u, p2x2 = a.P2 * 0x10001u;
  const bool en_v = (a.path_mask >> (UP ? 3 : 2)) & 1u;
  const bool en_fl = (a.path_mask >> (UP ? 6 : 4)) & 1u;
  const bool en_fr = (a.path_mask >> (UP ? 5 : 7)) & 1u;
  // lanes of owned pairs in this warp (owned and halo pairs share a warp
  // only when CHUNKS == 1)
  const unsigned own_mask = __ballot_sync(0xffffffffu, owned);
  if (t == 0) s_abort = 0;
  __syncthreads();

  for (int bi = 0; bi < a.nb; bi++) {
    const int band = UP ? (a.nb - 1 - bi) : bi;
    const int ytop = band * TH;
    const int nrows = min(TH, H - ytop);
    for (int item = blockIdx.x; item < a.items; item += gridDim.x) {
      const int p = item / J;
      const int j = item - p * J;
      const int x0 = j * kTW;
      // ---- wait for the neighbour strips to finish the previous band ----
      if (t == 0 && bi > 0) {
        long long spins = 0;
        const int* fl = a.flags + p * J;
        for (int n = j - 1; n <= j + 1; n += 2) {
          if (n < 0 || n >= J) continue;
          while (ld_acquire(fl + n) < bi) {
            if (++spins > a.spin_limit || *((volatile int*)a.err) != 0) {
              atomicExch(a.err, 1);
              s_abort = 1;
              break;
            }
            __nanosleep(64);
          }
          if (s_abort) break;
        }
        __threadfence();
      }
      __syncthreads();
      if (s_abort) return;

      // ---- columns of this thread's pair ----
      int xlo, xhi;
      if (owned) {
        xlo = x0 + pr;
        xhi = x0 + 16 + pr;
      } else {
        xlo = x0 - kHalo + (pr - 16);
        xhi = x0 + kTW + (pr - 16);
      }
      const bool lo_in = live && xlo >= 0 && xlo < W, hi_in = live && xhi >= 0 && xhi < W;
      // lanes whose predecessor column lies outside the image start a path
      const uint32_t fl_keep = ((xlo - 1 >= 0) ? 0x0000ffffu : 0u) | ((xhi - 1 >= 0) ? 0xffff0000u : 0u);
      const uint32_t fr_keep = ((xlo + 1 < W) ? 0x0000ffffu : 0u) | ((xhi + 1 < W) ? 0xffff0000u : 0u);

      const PassIO& io = a.io[p];
      const uint8_t* bsv = a.bs + ((size_t)(p * 2 + ((bi + 1) & 1)) * 3 + 0) * W * Dp;
      const uint8_t* bsl = bsv + (size_t)W * Dp;
      const uint8_t* bsr = bsl + (size_t)W * Dp;
      uint8_t* wsv = a.bs + ((size_t)(p * 2 + (bi & 1)) * 3 + 0) * W * Dp;
      uint8_t* wsl = wsv + (size_t)W * Dp;
      uint8_t* wsr = wsl + (size_t)W * Dp;

      uint32_t Lv[kDC], Lf[kDC], Lr[kDC], Cc[kDC];
      uint32_t mv = 0, mf = 0, mr = 0;
      // ---- predecessor states at the band boundary ----
      {
        const bool have = bi > 0;
        auto load_pair = [&](const uint8_t* base, int cl, int ch, uint32_t* r, uint32_t keep) {
          uint4 va = make_uint4(0, 0, 0, 0), vb = va;
          if (live && have && (keep & 0xffffu) && cl >= 0 && cl < W)
            va = __ldcg(reinterpret_cast<const uint4*>(base + (size_t)cl * Dp + d0));
          if (live && have && (keep & 0xffff0000u) && ch >= 0 && ch < W)
            vb = __ldcg(reinterpret_cast<const uint4*>(base + (size_t)ch * Dp + d0));
          bytes_to_pairs_u8(va, vb, r);
          if (pad) {
#pragma unroll
            for (int i = 0; i < kDC; i++)
              if (d0 + i >= a.D) r[i] = (have ? kPadCost2 : 0u) & keep;
          }
        };
        if (owned) load_pair(bsv, xlo, xhi, Lv, 0xffffffffu);
        else {
#pragma unroll
          for (int i = 0; i < kDC; i++) Lv[i] = 0;
        }
        load_pair(bsl, xlo - 1, xhi - 1, Lf, fl_keep);
        load_pair(bsr, xlo + 1, xhi + 1, Lr, fr_keep);
        uint32_t av = 0xffffffffu, af = 0xffffffffu, ar = 0xffffffffu;
#pragma unroll
        for (int i = 0; i < kDC; i++) {
          av = vmin2(av, Lv[i]);
          af = vmin2(af, Lf[i]);
          ar = vmin2(ar, Lr[i]);
        }
        mv = group_min2<CHUNKS>(av);
        mf = group_min2<CHUNKS>(af);
        mr = group_min2<CHUNKS>(ar);
        if (!have) mv = mf = mr = 0;
        mf &= fl_keep;
        mr &= fr_keep;
      }

      // prefetch the first row's costs
      auto cost_ptr = [&](int x, int y) {
        return reinterpret_cast<const uint4*>(io.cost + ((size_t)y * W + x) * Dp + d0);
      };
      const int yfirst = UP ? ytop + nrows - 1 : ytop;
      uint4 ca = make_uint4(0, 0, 0, 0), cb = ca;
      if (lo_in) ca = __ldg(cost_ptr(xlo, yfirst));
      if (hi_in) cb = __ldg(cost_ptr(xhi, yfirst));

      for (int k = 0; k < nrows; k++) {
        const int y = UP ? ytop + nrows - 1 - k : ytop + k;
        bytes_to_pairs(ca, cb, Cc);
        if (pad) {
#pragma unroll
          for (int i = 0; i < kDC; i++)
            if (d0 + i >= a.D) Cc[i] = kPadCost2;
        }
        if (k + 1 < nrows) {
          const int yn = UP ? y - 1 : y + 1;
          if (lo_in) ca = __ldg(cost_ptr(xlo, yn));
          if (hi_in) cb = __ldg(cost_ptr(xhi, yn));
        }
        const int par = k & 1;
        // ---- vertical path (owned pairs) ----
        uint32_t Nv[kDC];
        if (owned) {
          uint32_t left = __shfl_up_sync(own_mask, Lv[kDC - 1], 1, CHUNKS);
          uint32_t right = __shfl_down_sync(own_mask, Lv[0], 1, CHUNKS);
          const bool fresh = (bi == 0 && k == 0);
          if (q == 0) left = fresh ? 0u : kInf2;
          if (q == CHUNKS - 1) right = fresh ? 0u : kInf2;
          const uint32_t acc = sgm_step16(Lv, Cc, left, right, mv, p1x2, p2x2, Nv);
          mv = group_min2<CHUNKS>(acc, own_mask);
        }
        // ---- diagonal paths ----
        uint32_t Nf[kDC], Nr[kDC];
        {
          uint32_t left = __shfl_up_sync(0xffffffffu, Lf[kDC - 1], 1, CHUNKS);
          uint32_t right = __shfl_down_sync(0xffffffffu, Lf[0], 1, CHUNKS);
          if (q == 0) left = kInf2 & fl_keep;
          if (q == CHUNKS - 1) right = kInf2 & fl_keep;
          if (bi == 0 && k == 0) { if (q == 0) left = 0; if (q == CHUNKS - 1) right = 0; }
          const uint32_t acc = sgm_step16(Lf, Cc, left, right, mf, p1x2, p2x2, Nf);
          mf = group_min2<CHUNKS>(acc);
        }
        {
          uint32_t left = __shfl_up_sync(0xffffffffu, Lr[kDC - 1], 1, CHUNKS);
          uint32_t right = __shfl_down_sync(0xffffffffu, Lr[0], 1, CHUNKS);
          if (q == 0) left = kInf2 & fr_keep;
          if (q == CHUNKS - 1) right = kInf2 & fr_keep;
          if (bi == 0 && k == 0) { if (q == 0) left = 0; if (q == CHUNKS - 1) right = 0; }
          const uint32_t acc = sgm_step16(Lr, Cc, left, right, mr, p1x2, p2x2, Nr);
          mr = group_min2<CHUNKS>(acc);
        }
        // ---- accumulate and emit (owned pairs) ----
        if (owned) {
          uint32_t S[kDC];
#pragma unroll
          for (int i = 0; i < kDC; i++)
            S[i] = (en_v ? Nv[i] : 0u) + (en_fl ? Nf[i] : 0u) + (en_fr ? Nr[i] : 0u);
          const size_t tile = ((((size_t)p * H + y) * J + j) * 16 + pr) * CHUNKS + q;
          uint4* sd = reinterpret_cast<uint4*>(a.sdown) + tile * 4;
          if (!UP) {
#pragma unroll
            for (int w = 0; w < 4; w++)
              sd[w] = make_uint4(S[4 * w], S[4 * w + 1], S[4 * w + 2], S[4 * w + 3]);
          } else {
            // add the down sweep and the horizontal paths
#pragma unroll
            for (int w = 0; w < 4; w++) {
              const uint4 v = __ldcs(sd + w);
              S[4 * w] += v.x;
              S[4 * w + 1] += v.y;
              S[4 * w + 2] += v.z;
              S[4 * w + 3] += v.w;
            }
            uint32_t hf[kDC], hb[kDC];
            const uint4 z = make_uint4(0, 0, 0, 0);
            const size_t ol = ((size_t)y * W + xlo) * Dp + d0, oh = ((size_t)y * W + xhi) * Dp + d0;
            bytes_to_pairs_u8(lo_in && a.en_h0 ? __ldcs(reinterpret_cast<const uint4*>(io.hfwd + ol)) : z,
                           hi_in && a.en_h0 ? __ldcs(reinterpret_cast<const uint4*>(io.hfwd + oh)) : z, hf);
            bytes_to_pairs_u8(lo_in && a.en_h1 ? __ldcs(reinterpret_cast<const uint4*>(io.hbwd + ol)) : z,
                           hi_in && a.en_h1 ? __ldcs(reinterpret_cast<const uint4*>(io.hbwd + oh)) : z, hb);
#pragma unroll
            for (int i = 0; i < kDC; i++) S[i] += hf[i] + hb[i];
            if (pad) {
#pragma unroll
              for (int i = 0; i < kDC; i++)
                if (d0 + i >= a.D) S[i] = 0xffffffffu;
            }
            if (io.S) {
              // full aggregated cost, [H][W][D] uint16
#pragma unroll
              for (int i = 0; i < kDC; i++) {
                if (d0 + i < a.D) {
                  if (lo_in) io.S[((size_t)y * W + xlo) * a.D + d0 + i] = (uint16_t)(S[i] & 0xffffu);
                  if (hi_in) io.S[((size_t)y * W + xhi) * a.D + d0 + i] = (uint16_t)(S[i] >> 16);
                }
              }
            }
            if (io.dint) {
              // winner-take-all: smallest d with the minimal S, per lane
              uint32_t mn = 0xffffffffu;
#pragma unroll
              for (int i = 0; i < kDC; i++) mn = vmin2(mn, S[i]);
              const uint32_t gmin = group_min2<CHUNKS>(mn, own_mask);
              uint32_t first = 0xffffffffu;
#pragma unroll
              for (int i = kDC - 1; i >= 0; i--) {
                const uint32_t d2 = (uint32_t)(d0 + i) * 0x10001u;
                const uint32_t lo_eq = ((S[i] ^ gmin) & 0xffffu) == 0 ? 0x0000ffffu : 0u;
                const uint32_t hi_eq = ((S[i] ^ gmin) & 0xffff0000u) == 0 ? 0xffff0000u : 0u;
                const uint32_t eq = lo_eq | hi_eq;
                first = (first & ~eq) | (d2 & eq);
              }
              const uint32_t dstar2 = group_min2<CHUNKS>(first, own_mask);
              // neighbours S(d*-1), S(d*+1) through shared memory
              uint32_t* row = srow + (pr * CHUNKS + q) * kDC;
#pragma unroll
              for (int i = 0; i < kDC; i++) row[i] = S[i];
              __syncwarp(own_mask);
              if (q == 0) {
                const uint32_t* prow = srow + pr * CHUNKS * kDC;
#pragma unroll
                for (int lane = 0; lane < 2; lane++) {
                  const int x = lane ? xhi : xlo;
                  if (x < 0 || x >= W) continue;
                  const int sh = 16 * lane;
                  const int ds = (dstar2 >> sh) & 0xffff;
                  const int sv = (prow[ds] >> sh) & 0xffff;
                  float v = (float)ds;
                  if (a.subpixel && ds > 0 && ds < a.D - 1) {
                    const int am = (int)((prow[ds - 1] >> sh) & 0xffff) - sv;
                    const int bp = (int)((prow[ds + 1] >> sh) & 0xffff) - sv;
                    v = __fadd_rn((float)ds, __fdiv_rn((float)(am - bp), (float)(2 * (am + bp))));
                  }
                  io.dint[(size_t)y * W + x] = (int16_t)ds;
                  if (io.dsub) io.dsub[(size_t)y * W + x] = v;
                }
              }
              __syncwarp(own_mask);
            }
          }
        }
        // ---- diagonal hand-over to the next row ----
        uint32_t* bfl = xfl + (par * NT + t) * kDC;
        uint32_t* bfr = xfr + (par * NT + t) * kDC;
#pragma unroll
        for (int w = 0; w < 4; w++) {
          reinterpret_cast<uint4*>(bfl)[w] = make_uint4(Nf[4 * w], Nf[4 * w + 1], Nf[4 * w + 2], Nf[4 * w + 3]);
          reinterpret_cast<uint4*>(bfr)[w] = make_uint4(Nr[4 * w], Nr[4 * w + 1], Nr[4 * w + 2], Nr[4 * w + 3]);
        }
        if (q == 0) {
          mfl[par * NP + pr] = mf;
          mfr[par * NP + pr] = mr;
        }
        if (owned) {
#pragma unroll
          for (int i = 0; i < kDC; i++) Lv[i] = Nv[i];
        }
        if (k + 1 == nrows) {
          // band end: publish the states of the owned columns
          if (owned) {
            uint4 va, vb;
            pairs_to_bytes(Nv, va, vb);
            if (lo_in) *reinterpret_cast<uint4*>(wsv + (size_t)xlo * Dp + d0) = va;
            if (hi_in) *reinterpret_cast<uint4*>(wsv + (size_t)xhi * Dp + d0) = vb;
            pairs_to_bytes(Nf, va, vb);
            if (lo_in) *reinterpret_cast<uint4*>(wsl + (size_t)xlo * Dp + d0) = va;
            if (hi_in) *reinterpret_cast<uint4*>(wsl + (size_t)xhi * Dp + d0) = vb;
            pairs_to_bytes(Nr, va, vb);
            if (lo_in) *reinterpret_cast<uint4*>(wsr + (size_t)xlo * Dp + d0) = va;
            if (hi_in) *reinterpret_cast<uint4*>(wsr + (size_t)xhi * Dp + d0) = vb;
          }
          __syncthreads();   // exchange buffers are reused by the next item
          break;
        }
        __syncthreads();
        // FL from column x-1, FR from column x+1 (whole registers except at
        // the two seams of the pair layout)
        {
          int src;
          uint32_t sel = 0;
          int src2 = -1;
          if (owned) {
            if (pr > 0) src = pr - 1;
            else { src = 16 + kHalo - 1; src2 = 15; sel = 0x5410u; }   // (x0-1, x0+15)
          } else {
            const int h = pr - 16;
            if (h > 0) src = pr - 1;
            else { src = pr; src2 = 15; sel = 0x7610u; }             // (-, x1-1)
          }
          const uint32_t* s1 = xfl + (par * NT + src * CHUNKS + q) * kDC;
          uint32_t m1 = mfl[par * NP + src];
          if (src2 < 0) {
#pragma unroll
            for (int w = 0; w < 4; w++) {
              const uint4 v = reinterpret_cast<const uint4*>(s1)[w];
              Lf[4 * w] = v.x; Lf[4 * w + 1] = v.y; Lf[4 * w + 2] = v.z; Lf[4 * w + 3] = v.w;
            }
            mf = m1;
          } else {
            const uint32_t* s2 = xfl + (par * NT + src2 * CHUNKS + q) * kDC;
#pragma unroll
            for (int i = 0; i < kDC; i++) Lf[i] = prmt(s1[i], s2[i], sel);
            mf = prmt(m1, mfl[par * NP + src2], sel);
          }
        }
        {
          int src;
          uint32_t sel = 0;
          int src2 = -1;
          if (owned) {
            if (pr < 15) src = pr + 1;
            else { src = 0; src2 = 16; sel = 0x7632u; }               // (x0+16, x1)
          } else {
            const int h = pr - 16;
            if (h < kHalo - 1) src = pr + 1;
            else src = 0;                                             // (x0, -)
          }
          const uint32_t* s1 = xfr + (par * NT + src * CHUNKS + q) * kDC;
          uint32_t m1 = mfr[par * NP + src];
          if (src2 < 0) {
#pragma unroll
            for (int w = 0; w < 4; w++) {
              const uint4 v = reinterpret_cast<const uint4*>(s1)[w];
              Lr[4 * w] = v.x; Lr[4 * w + 1] = v.y; Lr[4 * w + 2] = v.z; Lr[4 * w + 3] = v.w;
            }
            mr = m1;
          } else {
            const uint32_t* s2 = xfr + (par * NT + src2 * CHUNKS + q) * kDC;
#pragma unroll
            for (int i = 0; i < kDC; i++) Lr[i] = prmt(s1[i], s2[i], sel);
            mr = prmt(m1, mfr[par * NP + src2], sel);
          }
        }
        // a lane whose predecessor column is outside the image restarts
        if (fl_keep != 0xffffffffu) {
#pragma unroll
          for (int i = 0; i < kDC; i++) Lf[i] &= fl_keep;
          mf &= fl_keep;
        }
        if (fr_keep != 0xffffffffu) {
#pragma unroll
          for (int i = 0; i < kDC; i++) Lr[i] &= fr_keep;
          mr &= fr_keep;
        }
      }
      // ---- publish progress ----
      __threadfence();
      __syncthreads();
      if (t == 0) st_release(a.flags + p * J + j, bi + 1);
    }
  }
}

}  // namespace

size_t sweep_smem_bytes(int chunks) {
  const int NP = 16 + kHalo, NT = NP * chunks;
  return (size_t)(2 * 2 * NT * kDC + 2 * 2 * NP + 16 * chunks * kDC) * sizeof(uint32_t);
}

cudaError_t launch_cost_pair(const uint64_t* cL, const uint64_t* cR, int W, int H, int D, int Dp,
                             int cmax, uint8_t* CL, uint8_t* CR, cudaStream_t s) {
  StageTrace trace(SF_STAGE_COST, s);
  const size_t smem = (size_t)W * 16 + (size_t)W * Dp;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(cost_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  count_launches(1);
  cost_pair_kernel<<<H, 512, smem, s>>>(cL, cR, W, H, D, Dp, cmax, CL, CR);
  return cudaGetLastError();
}

template <int CHUNKS>
static cudaError_t hline_dispatch(const HLineArgs& a, cudaStream_t s) {
  const int rows2 = (a.H + 1) / 2;
  const long long threads = (long long)a.npass * rows2 * 2 * CHUNKS;
  hline_kernel<CHUNKS><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_hline(const HLineArgs& a, cudaStream_t s) {
  StageTrace trace(SF_STAGE_AGGREGATE, s);
  count_launches(1);
  switch (chunks_for(a.D)) {
    case 1: return hline_dispatch<1>(a, s);
    case 2: return hline_dispatch<2>(a, s);
    case 4: return hline_dispatch<4>(a, s);
    case 8: return hline_dispatch<8>(a, s);
    default: return hline_dispatch<16>(a, s);
  }
}

template <int CHUNKS, bool UP>
static cudaError_t sweep_dispatch(const SweepArgs& a, cudaStream_t s, int* grid_out) {
  auto kern = sweep_kernel<CHUNKS, UP>;
  const size_t smem = sweep_smem_bytes(CHUNKS);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = (16 + kHalo) * CHUNKS;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int grid = std::min(a.items, per_sm * sms);
  if (grid_out) *grid_out = grid;
  SweepArgs args = a;
  void* params[] = {&args};
  // cooperative launch: every CTA is resident at once, so the bounded
  // neighbour waits always have a running producer
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), params, smem, s);
}

cudaError_t launch_sweep(const SweepArgs& a, bool up, cudaStream_t s) {
  StageTrace trace(SF_STAGE_SGM_SWEEP, s);
  count_launches(1);
  switch (chunks_for(a.D)) {
    case 1: return up ? sweep_dispatch<1, true>(a, s, nullptr) : sweep_dispatch<1, false>(a, s, nullptr);
    case 2: return up ? sweep_dispatch<2, true>(a, s, nullptr) : sweep_dispatch<2, false>(a, s, nullptr);
    case 4: return up ? sweep_dispatch<4, true>(a, s, nullptr) : sweep_dispatch<4, false>(a, s, nullptr);
    case 8: return up ? sweep_dispatch<8, true>(a, s, nullptr) : sweep_dispatch<8, false>(a, s, nullptr);
    default: return up ? sweep_dispatch<16, true>(a, s, nullptr) : sweep_dispatch<16, false>(a, s, nullptr);
  }
}

}  // namespace fused
}  // namespace sf
