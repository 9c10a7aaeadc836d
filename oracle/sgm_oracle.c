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
