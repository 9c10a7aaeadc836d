/*
 * Plain, slow CPU oracle for SGM stereo and the scene-flow combination of
 * "Combining Stereo Disparity and Optical Flow for Basic Scene Flow"
 * (Schuster et al., arXiv 1801.04720).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the bench's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA implementation.
 *
 * Every step follows the paper's order.  The paper names SGM with census
 * matching (Sec. 3.1, citing Hirschmueller 2008) and defines the combination
 * (Sec. 3.3, Eq. 3-5); the SGM recurrence written here is the cited method's
 * standard form with constant penalties P1 <= P2.  Integer work is exact;
 * subpixel refinement and the combination are evaluated in double precision.
 *
 * Array layouts (all row-major, pixel index i = y*W + x):
 *   image   uint8  [H][W]
 *   census  uint64 [H][W]
 *   cost    uint8  [H][W][D]   (d fastest)
 *   L_r, S  int32  [H][W][D]
 *   flow    float  [H][W][2]   (u, v)
 *   s4      double [H][W][4]   (u, v, d0, d1)
 *   motion, point double [H][W][3]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int clamp_int(int v, int lo, int hi) {
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

/* Census transform over a cw x ch window (cw, ch odd, cw*ch-1 <= 64 bits).
 * Bits are numbered in row-major window order (dy outer, dx inner), the
 * centre is skipped, and bit k is the k-th least significant bit.  A bit is
 * 1 iff the neighbour is strictly darker than the centre.  Neighbours outside
 * the image are taken from the nearest edge pixel (clamped coordinates).
 * Sec. 3.1 names SGM; the census window is the matching cost's parameter. */
void oracle_census(const uint8_t* img, int W, int H, int cw, int ch, uint64_t* out) {
  int rx = cw / 2, ry = ch / 2;
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      int centre = img[y * W + x];
      uint64_t bits = 0;
      int k = 0;
      for (int dy = -ry; dy <= ry; dy++) {
        for (int dx = -rx; dx <= rx; dx++) {
          if (dx == 0 && dy == 0) continue;
          int xx = clamp_int(x + dx, 0, W - 1);
          int yy = clamp_int(y + dy, 0, H - 1);
          if (img[yy * W + xx] < centre) bits |= ((uint64_t)1) << k;
          k++;
        }
      }
      out[y * W + x] = bits;
    }
  }
}

static int hamming64(uint64_t a, uint64_t b) {
  uint64_t v = a ^ b;
  int n = 0;
  while (v) {
    n += (int)(v & 1u);
    v >>= 1;
  }
  return n;
}

/* Matching cost volume: the Hamming distance between census strings.
 * Left reference (ref_is_right = 0): C(x,y,d) = H(cL(x,y), cR(x-d,y)),
 * right reference (ref_is_right = 1): C(x,y,d) = H(cR(x,y), cL(x+d,y)).
 * A candidate outside the image costs cmax (the number of census bits). */
void oracle_cost(const uint64_t* c_ref, const uint64_t* c_other, int W, int H, int D,
                 int ref_is_right, int cmax, uint8_t* cost) {
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      for (int d = 0; d < D; d++) {
        int xo = ref_is_right ? x + d : x - d;
        int c;
        if (xo < 0 || xo > W - 1)
          c = cmax;
        else
          c = hamming64(c_ref[y * W + x], c_other[y * W + xo]);
        cost[((size_t)y * W + x) * D + d] = (uint8_t)c;
      }
    }
  }
}

/* Penalty for a disparity change of two or more on the path step from
 * q = p - r to p.  Constant P2 unless `img` (the reference image of the pass,
 * uint8 [H][W]) is given: then the cited SGM (Hirschmueller 2008, cited in
 * Sec. 3.1) adapts it to the intensity step, P2 / |I(p) - I(q)| rounded down
 * and never below P1, keeping P2 where the intensities are equal. */
static int step_penalty(const uint8_t* img, int W, int x, int y, int qx, int qy, int P1, int P2) {
  if (!img) return P2;
  int g = (int)img[y * W + x] - (int)img[qy * W + qx];
  if (g < 0) g = -g;
  if (g == 0) return P2;
  int v = P2 / g;
  return v < P1 ? P1 : v;
}

/* One SGM path r = (rx, ry) (Sec. 3.1: eight paths radiate from each pixel).
 * L_r(p,d) = C(p,d) + min( L_r(p-r,d), L_r(p-r,d-1)+P1, L_r(p-r,d+1)+P1,
 *                          min_k L_r(p-r,k)+P2 ) - min_k L_r(p-r,k),
 * and L_r(p,d) = C(p,d) where p-r lies outside the image.  The d-1 / d+1
 * terms are left out at d = 0 and d = D-1.  Pixels are visited in an order
 * in which p-r always comes before p.  With a guide image `img` (may be NULL)
 * the P2 of each step is step_penalty()'s. */
void oracle_path_guided(const uint8_t* cost, const uint8_t* img, int W, int H, int D, int P1, int P2,
                        int rx, int ry, int32_t* L) {
  int y_first = (ry >= 0) ? 0 : H - 1, y_step = (ry >= 0) ? 1 : -1;
  int x_first = (rx >= 0) ? 0 : W - 1, x_step = (rx >= 0) ? 1 : -1;
  for (int iy = 0, y = y_first; iy < H; iy++, y += y_step) {
    for (int ix = 0, x = x_first; ix < W; ix++, x += x_step) {
      const uint8_t* c = cost + ((size_t)y * W + x) * D;
      int32_t* out = L + ((size_t)y * W + x) * D;
      int qx = x - rx, qy = y - ry;
      if (qx < 0 || qx > W - 1 || qy < 0 || qy > H - 1) {
        for (int d = 0; d < D; d++) out[d] = c[d];
        continue;
      }
      const int32_t* prev = L + ((size_t)qy * W + qx) * D;
      int32_t prev_min = prev[0];
      for (int k = 1; k < D; k++)
        if (prev[k] < prev_min) prev_min = prev[k];
      const int p2 = step_penalty(img, W, x, y, qx, qy, P1, P2);
      for (int d = 0; d < D; d++) {
        int32_t best = prev[d];
        if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
        if (d < D - 1 && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
        if (prev_min + p2 < best) best = prev_min + p2;
        out[d] = c[d] + best - prev_min;
      }
    }
  }
}

/* The path with constant penalties. */
void oracle_path(const uint8_t* cost, int W, int H, int D, int P1, int P2, int rx, int ry,
                 int32_t* L) {
  oracle_path_guided(cost, NULL, W, H, D, P1, P2, rx, ry, L);
}

/* The eight traversal directions, in the order of the path-mask bits. */
static const int kDirX[8] = {+1, -1, 0, 0, +1, -1, +1, -1};
static const int kDirY[8] = {0, 0, +1, -1, +1, -1, -1, +1};

void oracle_direction(int index, int* rx, int* ry) {
  *rx = kDirX[index];
  *ry = kDirY[index];
}

/* Aggregated cost S(p,d) = sum over the enabled paths r of L_r(p,d).
 * scratch holds one int32 [H][W][D] path buffer.  img: guide image for the
 * adaptive P2 of every path, or NULL for constant P2. */
void oracle_aggregate_guided(const uint8_t* cost, const uint8_t* img, int W, int H, int D, int P1,
                             int P2, uint32_t path_mask, int32_t* S, int32_t* scratch) {
  size_t n = (size_t)W * H * D;
  for (size_t i = 0; i < n; i++) S[i] = 0;
  for (int r = 0; r < 8; r++) {
    if (!((path_mask >> r) & 1u)) continue;
    oracle_path_guided(cost, img, W, H, D, P1, P2, kDirX[r], kDirY[r], scratch);
    for (size_t i = 0; i < n; i++) S[i] += scratch[i];
  }
}

void oracle_aggregate(const uint8_t* cost, int W, int H, int D, int P1, int P2,
                      uint32_t path_mask, int32_t* S, int32_t* scratch) {
  oracle_aggregate_guided(cost, NULL, W, H, D, P1, P2, path_mask, S, scratch);
}

/* Winner-take-all with parabolic subpixel refinement.  d* is the smallest d
 * reaching min_d S(p,d).  For 0 < d* < D-1 a parabola through
 * (d*-1, d*, d*+1) moves the estimate by (a-b) / (2(a+b)) with
 * a = S(d*-1) - S(d*) > 0 and b = S(d*+1) - S(d*) >= 0; at the ends of the
 * range (or with subpixel = 0) the estimate is d* itself. */
void oracle_select(const int32_t* S, int W, int H, int D, int subpixel, int16_t* dint,
                   double* dsub) {
  for (int i = 0; i < W * H; i++) {
    const int32_t* s = S + (size_t)i * D;
    int best = 0;
    for (int d = 1; d < D; d++)
      if (s[d] < s[best]) best = d;
    dint[i] = (int16_t)best;
    double v = (double)best;
    if (subpixel && best > 0 && best < D - 1) {
      double a = (double)(s[best - 1] - s[best]);
      double b = (double)(s[best + 1] - s[best]);
      v = (double)best + (a - b) / (2.0 * (a + b));
    }
    if (dsub) dsub[i] = v;
  }
}

/* Uniqueness filter on the winners of oracle_select (a post-filter of SGM
 * implementations; the paper only names SGM, Sec. 3.1).  With S0 = S(d*)
 * and S2 the smallest S(d) over |d - d*| >= 2, the winner is unique iff
 * 100 * S2 >= (100 + ratio) * S0 (percent; ratio = 0 keeps every winner,
 * and so does a curve with no d two away from d*).  Removed winners get a
 * NaN subpixel value; dint is left as it is. */
void oracle_uniqueness(const int32_t* S, int W, int H, int D, int ratio, const int16_t* dint,
                       double* dsub) {
  for (int i = 0; i < W * H; i++) {
    const int32_t* s = S + (size_t)i * D;
    int best = dint[i];
    int found = 0;
    int32_t s2 = 0;
    for (int d = 0; d < D; d++) {
      if (d >= best - 1 && d <= best + 1) continue;
      if (!found || s[d] < s2) s2 = s[d];
      found = 1;
    }
    if (found && 100 * (int64_t)s2 < (int64_t)(100 + ratio) * s[best]) dsub[i] = NAN;
  }
}

/* Left-right consistency check (Sec. 3.1): the left disparity at x is kept
 * iff x - dL >= 0 and |dL(x,y) - dR(x-dL(x,y), y)| <= tol on the integer
 * winner-take-all values, and the left winner was not removed before the
 * check (a NaN subpixel value: the uniqueness filter).  Kept pixels carry
 * the subpixel left value, the others NaN; valid is 1 / 0. */
void oracle_lr_check(const int16_t* dL, const int16_t* dR, const double* dL_sub, int W, int H,
                     int tol, uint8_t* valid, double* disp) {
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      int i = y * W + x;
      int dl = dL[i];
      int ok = 0;
      int xr = x - dl;
      if (xr >= 0 && !isnan(dL_sub[i])) {
        int diff = dl - (int)dR[y * W + xr];
        if (diff < 0) diff = -diff;
        ok = diff <= tol;
      }
      valid[i] = (uint8_t)ok;
      disp[i] = ok ? dL_sub[i] : NAN;
    }
  }
}

/* A disparity sample is usable when it survived the consistency check (is
 * not NaN) and is positive: Eq. 1 maps into the positive reals. */
static int disparity_usable(double d) { return !isnan(d) && d > 0.0; }

/* Combination (Sec. 3.3, Eq. 3-5).  x' = x + F(x) is evaluated as the float32
 * round-to-nearest sum and then widened.  S(x) is defined iff x' lies in the
 * closed pixel-centre domain [0, W-1] x [0, H-1], D0(x) is usable and every
 * bilinear tap of D1 with a non-zero Eq. 5 weight is usable.  Then
 * S = (u, v, d0, d1), the point is P0 = ((x-cx)B/d0, (y-cy)B/d0, fB/d0), the
 * warped point P1 = ((x'-cx)B/d1, (y'-cy)B/d1, fB/d1) and motion = P1 - P0.
 * Undefined pixels get NaN in every float output and valid = 0.  motion and
 * point may be NULL. */
void oracle_combine(const double* D0, const double* D1, const float* flow, int W, int H,
                    double f, double B, double cx, double cy, double* s4, double* motion,
                    double* point, uint8_t* valid) {
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      int i = y * W + x;
      float u = flow[2 * i], v = flow[2 * i + 1];
      double d0 = D0[i];
      double xp = (double)((float)x + u);
      double yp = (double)((float)y + v);
      int ok = disparity_usable(d0) && xp >= 0.0 && xp <= (double)(W - 1) && yp >= 0.0 &&
               yp <= (double)(H - 1);
      double d1 = 0.0;
      if (ok) {
        double x0 = floor(xp), y0 = floor(yp);
        double fx = xp - x0, fy = yp - y0;
        int ix = (int)x0, iy = (int)y0;
        double w[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy), (1.0 - fx) * fy, fx * fy};
        int tx[4] = {ix, ix + 1, ix, ix + 1};
        int ty[4] = {iy, iy, iy + 1, iy + 1};
        for (int t = 0; t < 4 && ok; t++) {
          if (w[t] == 0.0) continue;
          double dt = D1[ty[t] * W + tx[t]];
          if (!disparity_usable(dt))
            ok = 0;
          else
            d1 += w[t] * dt;
        }
      }
      valid[i] = (uint8_t)ok;
      if (!ok) {
        for (int k = 0; k < 4; k++) s4[4 * i + k] = NAN;
        for (int k = 0; k < 3; k++) {
          if (motion) motion[3 * i + k] = NAN;
          if (point) point[3 * i + k] = NAN;
        }
        continue;
      }
      s4[4 * i + 0] = (double)u;
      s4[4 * i + 1] = (double)v;
      s4[4 * i + 2] = d0;
      s4[4 * i + 3] = d1;
      double P0[3] = {(x - cx) * B / d0, (y - cy) * B / d0, f * B / d0};
      double P1[3] = {(xp - cx) * B / d1, (yp - cy) * B / d1, f * B / d1};
      for (int k = 0; k < 3; k++) {
        if (motion) motion[3 * i + k] = P1[k] - P0[k];
        if (point) point[3 * i + k] = P0[k];
      }
    }
  }
}

/* ---- Densification (the paper's future work, Sec. 5; Table 1's dense "All"
 * rows are the benchmark's own fill of a sparse submission, Sec. 4.1) ----
 *
 * Fill of a sparse map (NaN = missing), first along each row, then, for the
 * rows with nothing kept, along each column of the row-filled map.  Within a
 * line, a missing pixel between two kept ones at a and b takes:
 *   mode 0 (background): the smaller of the two values (the farther surface
 *     for a disparity);
 *   mode 1 (edge-aware): the value whose guide intensity is closer to the
 *     pixel's own (|I(p) - I(a)| against |I(p) - I(b)|), the smaller value on
 *     a tie;
 * a missing pixel with a kept value on one side only takes that value; a
 * line with nothing kept stays missing.  guide: uint8 [H][W] (mode 1). */
static double fill_choose(int mode, const uint8_t* guide, double va, double vb, size_t p, size_t a,
                          size_t b) {
  if (mode == 1) {
    int ia = abs((int)guide[p] - (int)guide[a]);
    int ib = abs((int)guide[p] - (int)guide[b]);
    if (ia < ib) return va;
    if (ib < ia) return vb;
  }
  return va < vb ? va : vb;
}

/* One line of n samples at in[i0 + k*step] -> out (same indexing); guide
 * indexed alike. */
static void fill_line(const double* in, const uint8_t* guide, int mode, int n, size_t i0, size_t step,
                      double* out) {
  for (int k = 0; k < n; k++) {
    size_t i = i0 + (size_t)k * step;
    if (!isnan(in[i])) {
      out[i] = in[i];
      continue;
    }
    int a = -1, b = -1;
    for (int j = k - 1; j >= 0; j--)
      if (!isnan(in[i0 + (size_t)j * step])) { a = j; break; }
    for (int j = k + 1; j < n; j++)
      if (!isnan(in[i0 + (size_t)j * step])) { b = j; break; }
    if (a >= 0 && b >= 0) {
      size_t ia = i0 + (size_t)a * step, ib = i0 + (size_t)b * step;
      out[i] = fill_choose(mode, guide, in[ia], in[ib], i, ia, ib);
    } else if (a >= 0) {
      out[i] = in[i0 + (size_t)a * step];
    } else if (b >= 0) {
      out[i] = in[i0 + (size_t)b * step];
    } else {
      out[i] = NAN;
    }
  }
}

void oracle_fill(const double* in, const uint8_t* guide, int mode, int W, int H, double* out,
                 double* rows) {
  for (int y = 0; y < H; y++) fill_line(in, guide, mode, W, (size_t)y * W, 1, rows);
  for (int x = 0; x < W; x++) fill_line(rows, guide, mode, H, (size_t)x, (size_t)W, out);
  /* the column pass only serves the rows the row pass left empty */
  for (size_t i = 0; i < (size_t)W * H; i++)
    if (!isnan(rows[i])) out[i] = rows[i];
}

/* Dense scene flow from a sparse result: d0 and d1 of s4 (NaN where the
 * combination left them undefined) each filled by oracle_fill, (u, v) taken
 * from the flow, then the back-projection of Sec. 3.3 at every pixel whose
 * filled disparities are both positive (the others NaN, valid 0):
 * P0 = ((x-cx)B/d0, (y-cy)B/d0, fB/d0), P1 at x' = fl32(x+u), y' = fl32(y+v)
 * with d1, motion = P1 - P0. */
void oracle_densify(const double* s4, const float* flow, const uint8_t* guide, int mode, int W, int H,
                    double f, double B, double cx, double cy, double* s4_out, double* motion,
                    double* point, uint8_t* valid, double* scratch) {
  size_t n = (size_t)W * H;
  double* d0 = scratch;
  double* d1 = scratch + n;
  double* f0 = scratch + 2 * n;
  double* f1 = scratch + 3 * n;
  double* rows = scratch + 4 * n;
  for (size_t i = 0; i < n; i++) {
    d0[i] = s4[4 * i + 2];
    d1[i] = s4[4 * i + 3];
  }
  oracle_fill(d0, guide, mode, W, H, f0, rows);
  oracle_fill(d1, guide, mode, W, H, f1, rows);
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      size_t i = (size_t)y * W + x;
      float u = flow[2 * i], v = flow[2 * i + 1];
      double a = f0[i], b = f1[i];
      int ok = !isnan(a) && !isnan(b) && a > 0.0 && b > 0.0;
      valid[i] = (uint8_t)ok;
      s4_out[4 * i + 0] = ok ? (double)u : NAN;
      s4_out[4 * i + 1] = ok ? (double)v : NAN;
      s4_out[4 * i + 2] = ok ? a : NAN;
      s4_out[4 * i + 3] = ok ? b : NAN;
      double xp = (double)((float)x + u), yp = (double)((float)y + v);
      double P0[3] = {(x - cx) * B / a, (y - cy) * B / a, f * B / a};
      double P1[3] = {(xp - cx) * B / b, (yp - cy) * B / b, f * B / b};
      for (int k = 0; k < 3; k++) {
        if (motion) motion[3 * i + k] = ok ? P1[k] - P0[k] : NAN;
        if (point) point[3 * i + k] = ok ? P0[k] : NAN;
      }
    }
  }
}

/* ---- Multi-frame extension (the paper's future work, Sec. 5: more than two
 * frame pairs, with an intermediate validation) ----
 *
 * K frames with disparity maps D^0 .. D^{K-1} (NaN = removed by the check) and
 * flows F_0 .. F_{K-2} (F_k maps frame k to k+1).  The reference pixel
 * x_0 = (x, y) of frame 0 is followed through every frame:
 *   x_{k+1} = x_k + F_k(x_k),
 * with F_0(x_0) the flow at the pixel itself and, for k >= 1, F_k(x_k) the
 * Eq. 5 bilinear interpolation of F_k at x_k (taps of weight 0 skipped).
 * Positions are float32 round-to-nearest sums and products in a fixed order
 * (the weights (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy, each times its tap,
 * summed in that order): they decide which pixels are read and whether the
 * chain stays in the image, so both sides take those decisions in the same
 * precision.  The disparity of frame k is D^0(x_0) for k = 0 and the Eq. 5
 * interpolation of D^k at x_k for k >= 1 (float64 sums), with the rule of
 * the combination: every tap of nonzero weight usable.  The chain is valid iff
 * every x_k lies in [0, W-1] x [0, H-1] and every disparity is usable: each
 * intermediate frame validates it.  Output: the 3D point of every frame,
 * P_k = ((x_k - cx) B / d_k, (y_k - cy) B / d_k, f B / d_k), NaN when invalid.
 * With K = 2 this is the combination of Sec. 3.3 (P_1 - P_0 its motion).
 *
 * D: K pointers to double [H][W]; F: K-1 pointers to float [H][W][2];
 * points: double [K][H][W][3]; valid: uint8 [H][W]. */
static float bilerp_f32(const float* m, int W, int stride, int ix, int iy, float fx, float fy) {
  float w00 = (1.0f - fx) * (1.0f - fy);
  float r = w00 * m[((size_t)iy * W + ix) * stride];
  if (fx != 0.0f) {
    float w10 = fx * (1.0f - fy);
    r = r + w10 * m[((size_t)iy * W + ix + 1) * stride];
  }
  if (fy != 0.0f) {
    float w01 = (1.0f - fx) * fy;
    r = r + w01 * m[((size_t)(iy + 1) * W + ix) * stride];
  }
  if (fx != 0.0f && fy != 0.0f) {
    float w11 = fx * fy;
    r = r + w11 * m[((size_t)(iy + 1) * W + ix + 1) * stride];
  }
  return r;
}

void oracle_chain(const double* const* D, const float* const* F, int K, int W, int H, double f, double B,
                  double cx, double cy, double* points, uint8_t* valid) {
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      size_t i = (size_t)y * W + x;
      float px = (float)x, py = (float)y;
      int ok = 1;
      for (int k = 0; k < K && ok; k++) {
        double d;
        if (k == 0) {
          d = D[0][i];
          ok = disparity_usable(d);
        } else {
          /* x_k from x_{k-1} and F_{k-1} */
          const float* Fk = F[k - 1];
          float u, v;
          if (k == 1) {
            u = Fk[2 * i];
            v = Fk[2 * i + 1];
          } else {
            float x0 = floorf(px), y0 = floorf(py);
            float fx = px - x0, fy = py - y0;
            u = bilerp_f32(Fk, W, 2, (int)x0, (int)y0, fx, fy);
            v = bilerp_f32(Fk + 1, W, 2, (int)x0, (int)y0, fx, fy);
          }
          px = px + u;
          py = py + v;
          if (!(px >= 0.0f && px <= (float)(W - 1) && py >= 0.0f && py <= (float)(H - 1))) {
            ok = 0;
            break;
          }
          float x0 = floorf(px), y0 = floorf(py);
          double fx = (double)(px - x0), fy = (double)(py - y0);
          int ix = (int)x0, iy = (int)y0;
          double w[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy), (1.0 - fx) * fy, fx * fy};
          int tx[4] = {ix, ix + 1, ix, ix + 1};
          int ty[4] = {iy, iy, iy + 1, iy + 1};
          d = 0.0;
          for (int t = 0; t < 4 && ok; t++) {
            if (w[t] == 0.0) continue;
            double dt = D[k][(size_t)ty[t] * W + tx[t]];
            if (!disparity_usable(dt)) ok = 0;
            else d += w[t] * dt;
          }
        }
        if (ok) {
          double* P = points + (((size_t)k * H * W) + i) * 3;
          P[0] = ((double)px - cx) * B / d;
          P[1] = ((double)py - cy) * B / d;
          P[2] = f * B / d;
        }
      }
      valid[i] = (uint8_t)ok;
      if (!ok)
        for (int k = 0; k < K; k++)
          for (int c = 0; c < 3; c++) points[(((size_t)k * H * W) + i) * 3 + c] = NAN;
    }
  }
}
