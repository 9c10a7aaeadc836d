/*
 * libsf - GB300 (sm_103a) scene flow from SGM stereo disparity and a given
 * optical flow, after Schuster et al., "Combining Stereo Disparity and Optical
 * Flow for Basic Scene Flow" (arXiv 1801.04720).
 *
 * C ABI.  Plain pointers and sizes only.  Unless a function says otherwise:
 *   - every array pointer is a DEVICE pointer owned by the caller; the library
 *     never allocates, frees or keeps a pointer after the call returns (the
 *     frame pipeline, sf_pipeline_*, is the one exception: it owns device
 *     memory between sf_pipeline_create and sf_pipeline_destroy);
 *   - parameter structs (sf_sgm_params, sf_camera) live in HOST memory and are
 *     read during the call only;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); the work
 *     is enqueued asynchronously on it and the function returns without
 *     waiting;
 *   - arguments are validated on the host before anything is launched; a bad
 *     argument returns SF_ERR_INVALID_ARG or SF_ERR_UNSUPPORTED and enqueues
 *     nothing;
 *   - a launch failure returns SF_ERR_CUDA; an error raised while a kernel
 *     runs surfaces at the next synchronisation of `stream` (or from a later
 *     call's launch check).
 * Nothing crosses the ABI as an exception.
 *
 * Layouts: images are uint8 rows of `pitch` bytes (pitch >= W); every other
 * array is dense row-major with pixel index i = y*W + x and, for volumes, the
 * disparity d fastest: cost / aggregated cost [H][W][D].
 *
 * Disparity convention: a left-image pixel (x, y) with disparity d matches the
 * right-image pixel (x - d, y); d runs over 0 .. D-1.
 */
#ifndef SF_H_
#define SF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SF_OK = 0,
  SF_ERR_INVALID_ARG = 1,   /* null pointer, size out of range, bad buffer size  */
  SF_ERR_UNSUPPORTED = 2,   /* valid request outside what this build supports     */
  SF_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed               */
  SF_ERR_TIMEOUT = 4        /* a bounded device-side wait gave up (batch kernel)  */
} sf_status;

#define SF_MAX_DISPARITY 256
#define SF_NUM_PATHS 8

/* SGM parameters (Sec. 3.1 names SGM with eight paths and the left-right
 * check; the values are the method's free parameters).
 *   census_w, census_h : census window, both odd, census_w*census_h - 1 <= 64;
 *                        the matching cost of a candidate outside the image is
 *                        cmax = census_w*census_h - 1.
 *   P1, P2             : path penalties for |delta d| = 1 and >= 2;
 *                        need P1 <= P2 and cmax + P2 <= 255.
 *   path_mask          : bit r enables traversal direction r, in the order
 *                        (+1,0) (-1,0) (0,+1) (0,-1) (+1,+1) (-1,-1) (+1,-1) (-1,+1)
 *                        where (rx, ry) is the step from p - r to p.
 *   D                  : number of disparities, 1..256 (values 0..D-1).
 *   subpixel           : 1 = parabolic refinement of the winner, 0 = off.
 *   lr_tol             : left-right tolerance in pixels, >= 0 (inclusive).
 *   adaptive_p2        : 0 = constant P2; 1 = the intensity-adaptive P2 of the
 *                        SGM the paper cites (Hirschmueller 2008): on the path
 *                        step from q = p - r to p the penalty for a change of
 *                        two or more disparities is P2 / |I(p) - I(q)|
 *                        (integer division), never below P1, and P2 where
 *                        I(p) = I(q); I is the pass's reference image.
 *   uniqueness         : ratio in percent, 0..99 (0 = off).  A left winner d*
 *                        is removed (it fails the left-right check) unless
 *                        100 * S2 >= (100 + uniqueness) * S(d*), S2 the
 *                        smallest S(d) over |d - d*| >= 2 (kept when there is
 *                        no such d).  A post-filter of SGM implementations;
 *                        the paper names SGM only. */
typedef struct {
  int32_t census_w, census_h;
  uint16_t P1, P2;
  uint32_t path_mask;
  int32_t D;
  int32_t subpixel;
  int32_t lr_tol;
  int32_t adaptive_p2;
  int32_t uniqueness;
} sf_sgm_params;

/* Pinhole stereo camera: focal length f (px), baseline B (m), principal point
 * (cx, cy) in pixels.  Used by the back-projection Z = f*B/d. */
typedef struct {
  float f, B, cx, cy;
} sf_camera;

/* Fills p with census 9x7, P1 = 7, P2 = 86, all 8 paths, D = 128, subpixel on,
 * lr_tol = 1, constant P2, no uniqueness filter. */
void sf_default_params(sf_sgm_params* p);

/* Human-readable name of a status code (static storage). */
const char* sf_status_string(sf_status s);

/* Census transform (the matching cost of SGM, Sec. 3.1).  Bit k of
 * census_out[y*W+x] (k = 0 least significant) is 1 iff the k-th window
 * neighbour, counted row-major with the centre skipped, is strictly darker
 * than the centre; neighbours outside the image take the nearest edge pixel.
 * img: uint8 [H][pitch]; census_out: uint64 [H][W]. */
sf_status sf_census(const uint8_t* img, int32_t W, int32_t H, int32_t pitch, int32_t census_w,
                    int32_t census_h, uint64_t* census_out, void* stream);

/* Matching cost volume (Sec. 3.1): Hamming distance of census strings.
 * ref_is_right = 0: cost(x,y,d) = H(cL(x,y), cR(x-d,y)), ref = left image;
 * ref_is_right = 1: cost(x,y,d) = H(cR(x,y), cL(x+d,y)), ref = right image.
 * Candidates outside the image cost cmax.  ref / other: uint8 [H][pitch];
 * cost_out: uint8 [H][W][D].  Census strings are computed inside the call. */
sf_status sf_cost_volume(const uint8_t* ref, const uint8_t* other, int32_t W, int32_t H,
                         int32_t pitch, const sf_sgm_params* p, int32_t ref_is_right,
                         uint8_t* cost_out, void* stream);

/* Workspace bytes with which sf_sgm_aggregate runs the fused band sweeps
 * (0 when D is not a multiple of 16: the staged kernels need none). */
size_t sf_aggregate_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p);

/* Semi-global aggregation over the enabled paths (Sec. 3.1, "eight different
 * paths"): S(p,d) = sum_r L_r(p,d) with
 *   L_r(p,d) = C(p,d) + min(L_r(p-r,d), L_r(p-r,d+-1) + P1, min_k L_r(p-r,k) + P2)
 *              - min_k L_r(p-r,k),
 * and L_r(p,d) = C(p,d) where p - r is outside the image.  Exact integers.
 * cost: uint8 [H][W][D]; agg_out: uint16 [H][W][D].  With D % 16 == 0, a
 * 16-byte aligned cost volume and a workspace of at least
 * sf_aggregate_workspace_size() bytes the fused band sweeps run; otherwise
 * (workspace may then be NULL) one kernel per path.  p->adaptive_p2 = 1 needs
 * the reference image: it returns SF_ERR_INVALID_ARG here (use
 * sf_sgm_aggregate_guided). */
sf_status sf_sgm_aggregate(const uint8_t* cost, int32_t W, int32_t H, const sf_sgm_params* p,
                           uint16_t* agg_out, void* workspace, size_t ws_bytes, void* stream);

/* sf_sgm_aggregate with the reference image of the pass as a guide, for
 * p->adaptive_p2 = 1 (Sec. 3.1's SGM with the cited paper's adaptive P2, see
 * sf_sgm_params): guide is uint8 [H][pitch] (device), the image the cost
 * volume was computed for (left image for the left-reference volume).  With
 * adaptive_p2 = 0 the guide is ignored and the result is sf_sgm_aggregate's.
 * Same workspace rules as sf_sgm_aggregate. */
sf_status sf_sgm_aggregate_guided(const uint8_t* cost, const uint8_t* guide, int32_t pitch, int32_t W,
                                  int32_t H, const sf_sgm_params* p, uint16_t* agg_out, void* workspace,
                                  size_t ws_bytes, void* stream);

/* Bytes of the scratch array built into the library for
 * sf_sgm_aggregate_noalloc (32 MiB per device). */
#define SF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* sf_sgm_aggregate without a caller-provided workspace.  The paper has no
 * counterpart: this is a calling convention of the library, not a step of the
 * method.  It computes exactly what sf_sgm_aggregate computes (same S, bit for
 * bit) with the fused band sweeps, whose scratch lives in a file-scope device
 * array of SF_NOALLOC_SCRATCH_BYTES inside the library instead of the
 * caller's workspace.
 *
 * Who needs it: callers that cannot allocate device memory, e.g. a host
 * program that owns no device allocator (no PyTorch or memory pool to draw a
 * workspace from), or a latency-bound loop that must not call cudaMalloc /
 * cudaFree (they can synchronise the whole device and take driver locks).
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *
 * cost: uint8 [H][W][D], 16-byte aligned; agg_out: uint16 [H][W][D];
 * err_out: one int32 in device memory or NULL; after the call has run on
 * `stream` it holds 0, or 1 if a bounded inter-CTA wait of the sweeps gave up
 * (agg_out is then invalid).  All pointers are device pointers; the
 * parameters are read on the host during the call.
 *
 * Limits: D % 16 == 0, and the scratch the sweeps need for W x H x D (about
 * 4 x W x H x D bytes, more when D is not a power of two, plus small tables)
 * must fit SF_NOALLOC_SCRATCH_BYTES (e.g. 320 x 240 at D = 64, 640 x 480 at
 * D = 16, 1242 x 40 at D = 128); larger requests and other D return
 * SF_ERR_UNSUPPORTED before anything is enqueued.  Other argument
 * errors return SF_ERR_INVALID_ARG as in sf_sgm_aggregate.
 *
 * Zero state: the flags, task counters and error word at the start of the
 * scratch are cleared on `stream` by every call (cudaMemsetAsync); no other
 * part of the scratch has to start at zero.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current; this may load the
 * library's device code).  Make that first call on each device before any
 * stream capture begins.  The current device must be the device of `stream`.
 * Every later call made outside stream capture looks the address up again,
 * so a device or context reset (which may move the array) is picked up;
 * a call under capture uses the address of the last call made outside it.
 *
 * Concurrency: there is ONE scratch array per device and process.  Two calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads, without ordering between them) use the same scratch and race;
 * their results are then undefined.  Order such calls on one stream or
 * synchronise between them. */
sf_status sf_sgm_aggregate_noalloc(const uint8_t* cost, int32_t W, int32_t H,
                                   const sf_sgm_params* p, uint16_t* agg_out, int32_t* err_out,
                                   void* stream);

/* Winner-take-all and parabolic subpixel refinement (Sec. 3.1).  d* is the
 * smallest d reaching min_d S; for subpixel = 1 and 0 < d* < D-1 the output is
 * d* + (a-b)/(2(a+b)) with a = S(d*-1)-S(d*), b = S(d*+1)-S(d*), else d*.
 * agg: uint16 [H][W][D]; disp_int_out: int16 [H][W]; disp_sub_out: float
 * [H][W] or NULL. */
sf_status sf_disparity_select(const uint16_t* agg, int32_t W, int32_t H, int32_t D,
                              int32_t subpixel, int16_t* disp_int_out, float* disp_sub_out,
                              void* stream);

/* Left-right consistency check (Sec. 3.1; it makes the disparity map
 * non-dense): valid(x,y) = [x - dL >= 0 and |dL(x,y) - dR(x-dL,y)| <= tol] on
 * the integer winners; disp_out = dL_sub where valid, NaN elsewhere.
 * dL, dR: int16 [H][W]; dL_sub: float [H][W]; valid_out: uint8 [H][W]
 * (1 / 0); disp_out: float [H][W]. */
sf_status sf_lr_check(const int16_t* dL, const int16_t* dR, const float* dL_sub, int32_t W,
                      int32_t H, int32_t tol, uint8_t* valid_out, float* disp_out, void* stream);

/* Scene-flow combination (Sec. 3.3, Eq. 3-5).  For each pixel x the target is
 * x' = x + F(x), computed as a float32 round-to-nearest sum.  S(x) is defined
 * iff x' lies in [0, W-1] x [0, H-1], D0(x) is a usable disparity, and every
 * tap of the bilinear interpolation of D1 at x' (Eq. 5) whose weight is not
 * zero is usable; usable = not NaN and > 0.  Then
 *   s4     = (u, v, d0, d1)                        with d1 = D1(x') by Eq. 5,
 *   point  = P0 = ((x-cx)B/d0, (y-cy)B/d0, fB/d0),
 *   motion = P1 - P0, P1 = ((x'-cx)B/d1, (y'-cy)B/d1, fB/d1);
 * otherwise every float output is NaN and valid_out = 0.
 * D0, D1: float [H][W] (NaN = removed by the check); flow: float [H][W][2];
 * s4_out: float [H][W][4]; motion_out, point_out: float [H][W][3] or NULL;
 * valid_out: uint8 [H][W]. */
sf_status sf_combine_sceneflow(const float* D0, const float* D1, const float* flow, int32_t W,
                               int32_t H, const sf_camera* cam, float* s4_out, float* motion_out,
                               float* point_out, uint8_t* valid_out, void* stream);

/* ---- more than two frames (the paper's future work, Sec. 5) ---------------
 * A sequence of K stereo frames (2 <= K <= SF_MAX_FRAMES) with the flows
 * F_0 .. F_{K-2} (F_k from frame k to frame k+1, float [H][W][2]).
 *
 * Chain: the reference pixel x_0 of frame 0 is followed through every frame,
 * x_{k+1} = x_k + F_k(x_k) (F_0 at the pixel itself, F_k for k >= 1 by the
 * bilinear interpolation of Eq. 5 at x_k; positions as float32 sums and
 * products in a fixed order).  Frame k's disparity is the Eq. 5 interpolation
 * of D^k at x_k with every tap of nonzero weight usable (not NaN, > 0), as in
 * the combination; the chain is valid iff every x_k lies in [0, W-1] x
 * [0, H-1] and every disparity is usable, so each intermediate frame validates
 * it.  Output: the 3D point of the reference pixel in every frame,
 * P_k = ((x_k - cx) B / d_k, (y_k - cy) B / d_k, f B / d_k).  With K = 2 this is
 * sf_combine_sceneflow (point = P_0, motion = P_1 - P_0). */
#define SF_MAX_FRAMES 64

/* The chain alone.  disps: K device pointers (host array) to float [H][W]
 * (NaN = removed); flows: K-1 device pointers (host array) to float
 * [H][W][2]; points_out: float [K][H][W][3] or NULL (NaN where invalid);
 * valid_out: uint8 [H][W] or NULL. */
sf_status sf_chain_sceneflow(const float* const* disps, const float* const* flows, int32_t K, int32_t W,
                             int32_t H, const sf_camera* cam, float* points_out, uint8_t* valid_out, void* stream);

/* Workspace bytes of sf_sequence_sceneflow for K frames; learned = 1 for the
 * learned-confidence mode (packed != NULL there). */
size_t sf_sequence_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p, int32_t K, int32_t learned);

/* The hot path over a sequence: the SGM disparity of every stereo frame ONCE
 * (K pairs, where K-1 separate quadruples would compute 2 (K-1)), with the
 * plain left-right check (packed == NULL) or the learned confidence
 * (packed, threshold as in sf_scene_flow_learned); then the combination of
 * Sec. 3.3 for each consecutive pair (k, k+1), and the chain above.
 * left, right: K device pointers (host arrays) to uint8 [H][pitch]; flows:
 * K-1 device pointers.  Outputs, each a host array of device pointers or
 * NULL: disp_out (K maps float [H][W], NaN where removed), s4_out and
 * valid_out (K-1 entries, as in sf_combine_sceneflow), motion_out (K-1
 * entries, each float [H][W][3] or NULL); points_out float [K][H][W][3] and
 * chain_valid_out uint8 [H][W] (device, or NULL: no chain).  s4_out and
 * valid_out are both given or both NULL.  workspace: at least
 * sf_sequence_workspace_size() bytes. */
sf_status sf_sequence_sceneflow(const uint8_t* const* left, const uint8_t* const* right, int32_t K, int32_t pitch,
                                const float* const* flows, int32_t W, int32_t H, const sf_sgm_params* p,
                                const sf_camera* cam, const void* packed, float threshold, float* const* disp_out,
                                float* const* s4_out, uint8_t* const* valid_out, float* const* motion_out,
                                float* points_out, uint8_t* chain_valid_out, void* workspace, size_t ws_bytes,
                                void* stream);

/* ---- densification (the paper's future work, Sec. 5) ----------------------
 * The method's scene flow is sparse (Sec. 3.3); Table 1's dense rows come from
 * the benchmark's own fill of a sparse submission (Sec. 4.1).  A map whose
 * missing values are NaN is filled along each row, then, for the rows with
 * nothing kept, along each column of the row-filled map.  Within a line a
 * missing pixel between kept values a (before) and b (after) takes
 *   SF_FILL_BACKGROUND: min(a, b), the farther surface of a disparity map;
 *   SF_FILL_EDGE_AWARE: the one whose guide intensity is closer to the
 *                       pixel's own intensity (min(a, b) on a tie);
 * with one kept side it takes that value; a line with nothing kept stays NaN
 * (every pixel of a map with nothing kept stays NaN). */
#define SF_FILL_BACKGROUND 0
#define SF_FILL_EDGE_AWARE 1

/* Fills the NaN entries of a float map.  in, out: float [H][W], distinct
 * buffers (in == out returns SF_ERR_INVALID_ARG); guide: uint8 [H][pitch]
 * (the reference image), required for SF_FILL_EDGE_AWARE, ignored (may be
 * NULL) for SF_FILL_BACKGROUND. */
sf_status sf_fill_disparity(const float* in, int32_t W, int32_t H, const uint8_t* guide, int32_t pitch,
                            int32_t mode, float* out, void* stream);

/* Dense scene flow from a sparse result of sf_combine_sceneflow /
 * sf_scene_flow: d0 and d1 of s4_in (channels 2 and 3, NaN where undefined;
 * d1 is the warped disparity of t+1 at the reference pixel) are each filled as
 * in sf_fill_disparity, (u, v) is taken from the flow, and the
 * back-projection of Sec. 3.3 is evaluated at every pixel whose filled d0 and
 * d1 are both positive: s4_out = (u, v, d0, d1), point = P0, motion = P1 - P0
 * with x' = x + F(x) as a float32 sum; elsewhere NaN and valid 0.
 * s4_in, s4_out: float [H][W][4], distinct, 16-byte aligned; flow: float
 * [H][W][2]; motion_out, point_out: float [H][W][3] or NULL; valid_out: uint8
 * [H][W]; guide as in sf_fill_disparity (the left image at t). */
sf_status sf_densify_sceneflow(const float* s4_in, const float* flow, int32_t W, int32_t H, const sf_camera* cam,
                               const uint8_t* guide, int32_t pitch, int32_t mode, float* s4_out,
                               float* motion_out, float* point_out, uint8_t* valid_out, void* stream);

/* Workspace bytes for sf_sgm_full and sf_scene_flow at this size. */
size_t sf_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p);

/* Whole SGM for one rectified stereo pair (Sec. 3.1): census, cost,
 * aggregation and selection with the left image as reference and again with
 * the right image as reference, then the left-right check.
 * left, right: uint8 [H][pitch].  Outputs (each may be NULL except disp_out):
 * dL_out, dR_out: int16 [H][W] integer winners; valid_out: uint8 [H][W];
 * disp_out: float [H][W] (subpixel left disparity, NaN where invalid).
 * workspace: device buffer of at least sf_workspace_size() bytes, 256-byte
 * aligned, owned by the caller, contents undefined on return. */
sf_status sf_sgm_full(const uint8_t* left, const uint8_t* right, int32_t W, int32_t H,
                      int32_t pitch, const sf_sgm_params* p, int16_t* dL_out, int16_t* dR_out,
                      uint8_t* valid_out, float* disp_out, void* workspace, size_t ws_bytes,
                      void* stream);

/* The whole hot path for one stereo quadruple (Sec. 3): SGM disparity D0 on
 * (left_t, right_t) and D1 on (left_t1, right_t1), each with its left-right
 * check, then the combination with the given flow.  Images: uint8 [H][pitch];
 * flow: float [H][W][2]; outputs as in sf_combine_sceneflow; D0_out, D1_out:
 * float [H][W] or NULL (the checked subpixel disparities).  workspace: at least
 * sf_workspace_size() bytes. */
sf_status sf_scene_flow(const uint8_t* left_t, const uint8_t* right_t, const uint8_t* left_t1,
                        const uint8_t* right_t1, int32_t pitch, const float* flow, int32_t W,
                        int32_t H, const sf_sgm_params* p, const sf_camera* cam, float* s4_out,
                        float* motion_out, float* point_out, uint8_t* valid_out, float* D0_out,
                        float* D1_out, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace bytes for sf_scene_flow_host: sf_workspace_size() plus
 * device staging for the inputs and outputs. */
size_t sf_scene_flow_host_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p);

/* sf_scene_flow with HOST inputs and outputs: the four images (uint8 [H][W],
 * dense), flow and the outputs are host pointers (pinned memory gives
 * asynchronous copies; pageable memory works but copies synchronously).  The
 * call copies the inputs to the device workspace, runs the path, copies the
 * outputs back and waits for `stream`.  motion_out / point_out may be NULL. */
sf_status sf_scene_flow_host(const uint8_t* left_t, const uint8_t* right_t,
                             const uint8_t* left_t1, const uint8_t* right_t1, const float* flow,
                             int32_t W, int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                             float* s4_out, float* motion_out, float* point_out,
                             uint8_t* valid_out, void* dev_workspace, size_t ws_bytes,
                             void* stream);

/* ---- frame pipeline: host buffers, copies overlapped with compute -------- */

/* A pipeline of scene-flow frames of one size W x H, for a stream of
 * quadruples that live in host memory.  It holds `depth` (2..8) staging slots
 * in device memory for a frame's inputs and outputs, the sf_scene_flow
 * workspace, and three streams (copies in, compute, copies out) ordered by
 * events, so that while frame k computes, frame k+1's inputs are copied in
 * and frame k-1's outputs copied out.  The computation is sf_scene_flow's,
 * one frame at a time.  Unlike the other calls, the pipeline owns device
 * memory: allocated here (on the current device), freed by
 * sf_pipeline_destroy.  Returns SF_ERR_INVALID_ARG for a bad size, params,
 * camera or depth, SF_ERR_CUDA if an allocation fails. */
typedef struct sf_pipeline sf_pipeline;
sf_status sf_pipeline_create(int32_t W, int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                             int32_t depth, sf_pipeline** out);

/* Queues one frame and returns without waiting for it.  HOST pointers: the
 * four images (uint8 [H][W], dense), flow (float [H][W][2]) and the outputs
 * s4_out (float [H][W][4]), motion_out / point_out (float [H][W][3] or NULL)
 * and valid_out (uint8 [H][W]).  Pinned host memory gives asynchronous
 * copies; with pageable memory each copy blocks the host.  The inputs must
 * stay unchanged, and the outputs unread, until sf_pipeline_wait for this
 * frame returns.  *ticket (ticket may be NULL) numbers the frame: 0, 1, ...
 * Thread-safe with respect to other calls on the same pipeline. */
sf_status sf_pipeline_submit(sf_pipeline* pl, const uint8_t* left_t, const uint8_t* right_t,
                             const uint8_t* left_t1, const uint8_t* right_t1, const float* flow,
                             float* s4_out, float* motion_out, float* point_out, uint8_t* valid_out,
                             int64_t* ticket);

/* Blocks until the outputs of frame `ticket` (and of every frame submitted
 * before it) are in host memory.  An error raised by that work returns
 * SF_ERR_CUDA; an unknown ticket SF_ERR_INVALID_ARG. */
sf_status sf_pipeline_wait(sf_pipeline* pl, int64_t ticket);

/* Waits for every queued frame, then frees the pipeline's streams, events and
 * device memory. */
sf_status sf_pipeline_destroy(sf_pipeline* pl);

/* ---- batches of quadruples with uneven sizes ------------------------------ */

/* One quadruple of a batch: device pointers as in sf_scene_flow, its own size
 * W x H, row pitch and number of disparities D (1..256), its own camera. */
typedef struct {
  const uint8_t* left_t;
  const uint8_t* right_t;
  const uint8_t* left_t1;
  const uint8_t* right_t1;
  int32_t pitch;
  const float* flow;        /* [H][W][2] */
  int32_t W, H, D;
  sf_camera cam;
  float* s4_out;            /* [H][W][4], 16-byte aligned */
  float* motion_out;        /* [H][W][3] or NULL */
  float* point_out;         /* [H][W][3] or NULL */
  uint8_t* valid_out;       /* [H][W] */
  float* D0_out;            /* [H][W] or NULL */
  float* D1_out;            /* [H][W] or NULL */
} sf_batch_item;

#define SF_BATCH_GRAPH 1u   /* capture the batch into a CUDA graph once per
                               signature (items, params, workspace, stream)
                               and replay it on later calls */

/* Workspace bytes for sf_batch_run over these items (0 if an item is
 * invalid or too wide for the fused kernels). */
size_t sf_batch_workspace_size(const sf_batch_item* items, int32_t n, const sf_sgm_params* p);

/* The whole hot path for n quadruples at once (Sec. 3; the batch is this
 * library's addition).  The stereo passes of all items share persistent
 * sweep launches, one per kernel shape (items are grouped by D): a band-major
 * task queue walks every (item, pass, band, strip).  p->D is ignored (each
 * item has its own D); the other parameters apply to every item.  With
 * SF_BATCH_GRAPH the first call for a signature records a CUDA graph
 * (its set-up copies the batch's descriptor tables synchronously, so that
 * first call must not itself be under stream capture) and later calls replay
 * it; graph mode needs a created stream (not NULL: the legacy default
 * stream cannot be captured).  Outputs as in sf_scene_flow, per item. */
sf_status sf_batch_run(const sf_batch_item* items, int32_t n, const sf_sgm_params* p,
                       uint32_t flags, void* workspace, size_t ws_bytes, void* stream);

/* Destroys the CUDA graphs cached by sf_batch_run (host-side resources). */
void sf_batch_release_graphs(void);

/* Bounds the device memory a batch holds at a time (no counterpart in the
 * paper): with bytes > 0, sf_batch_run takes the items in consecutive waves,
 * each as many items as keep its buffers within `bytes` (at least one item),
 * one wave after another over one shared region, so the workspace is about
 * the largest wave's buffers instead of the whole batch's.  0 (the default):
 * one wave.  Process-wide; sf_batch_workspace_size follows it, and a cached
 * graph is keyed by it.  Outputs are identical for every limit. */
sf_status sf_set_batch_wave_limit(size_t bytes);

/* Kernel shape of the band sweeps for a class of disparity counts, as chosen
 * by an autotuner: every D in [d_lo, d_hi] then runs with `dc` disparities
 * per thread (8 or 16) and `halo` halo columns (8 or 16; the band height is
 * halo + 1).  Combinations the build does not provide, or too few threads
 * for D, return SF_ERR_UNSUPPORTED; dc = 0 restores the built-in choice for
 * the class.  Process-wide; results are identical for every shape. */
sf_status sf_set_sweep_shape(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo);

/* sf_set_sweep_shape with the scheduling order of the paths as well (no
 * counterpart in the paper, which sums the eight paths of Sec. 3.1 in any
 * order: the sum is exact).  order = 0: the horizontal paths, then the three
 * downward paths (0,+1), (+1,+1), (-1,+1) in one launch walking the image top
 * to bottom, then the three upward paths in a second launch walking bottom to
 * top, which adds everything and selects.  order = 1: the horizontal paths,
 * then both vertical scan orders in ONE launch, started from opposite ends of
 * the image: each band of rows is finished (sums, winner, subpixel) by
 * whichever order reaches it second, the other having left its partial sum,
 * so twice as many band tasks are available at a time.  order = 2: order 1
 * with the horizontal paths in the same launch: their row blocks head its
 * task queue and the band tasks that finish rows wait for those rows' blocks,
 * so the horizontal walks overlap the first half of the sweeps (batches of
 * uneven items run them in their own launch, as in order 1).  Integers are
 * identical in every order and shape.  Other orders, or shapes the build
 * does not provide, return SF_ERR_UNSUPPORTED. */
sf_status sf_set_sweep_schedule(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo, int32_t order);

/* sf_set_sweep_schedule for the learned launches of one frame's two left
 * passes (sf_sgm_learned, sf_scene_flow_learned), which keep a table of
 * their own: they carry half the work of the plain frame's four passes, so
 * another shape or order can pay there.  Learned launches of more passes
 * (sf_scene_flow_learned_frames with two or more frames, the learned
 * sequence) use the plain table.  Same arguments, rules and status codes;
 * results are identical in every order and shape.  A learned workspace is
 * sized for the shape in force when it is sized. */
sf_status sf_set_learned_sweep_schedule(int32_t d_lo, int32_t d_hi, int32_t dc, int32_t halo, int32_t order);

/* ---- tracing and counters (host-side bookkeeping; no paper counterpart) --- */

/* Stage ids written by the tracer. */
typedef enum {
  SF_STAGE_CENSUS = 0,      /* census transform                              */
  SF_STAGE_COST = 1,        /* stored cost volume                            */
  SF_STAGE_AGGREGATE = 2,   /* path aggregation (one stereo pass)            */
  SF_STAGE_SELECT = 3,      /* winner-take-all + subpixel                    */
  SF_STAGE_LRCHECK = 4,     /* left-right check                              */
  SF_STAGE_COMBINE = 5,     /* scene-flow combination                        */
  SF_STAGE_SGM_SWEEP = 6,   /* fused cost + aggregation sweep                */
  SF_STAGE_FEATURES = 7,    /* learned path: features of the cost curve      */
  SF_STAGE_CONFNET = 8,     /* learned path: confidence network inference    */
  SF_STAGE_DENSIFY = 9,     /* densification of a sparse result              */
  SF_NUM_STAGES = 10
} sf_stage;

/* Arms the tracer: from now on every stage the library enqueues is bracketed
 * by cudaEventRecord() of the next two events of `events` (cudaEvent_t
 * handles created by the caller) on the stage's stream, and the stage id is
 * appended to stage_out.  Recording stops silently when events run out.  The
 * arrays must stay valid until sf_trace_disarm().  Not thread-safe: arm and
 * disarm from the thread that enqueues the work. */
sf_status sf_trace_arm(void* const* events, int32_t n_events, int32_t* stage_out);

/* Disarms the tracer; returns the number of stage records made (each used
 * two events). */
int32_t sf_trace_disarm(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (all threads), for launch accounting. */
uint64_t sf_kernel_launches(void);

/* Test hooks for failure detection (no counterpart in the paper).
 * SF_DEBUG_SPIN_LIMIT: polls a bounded inter-CTA wait of the band sweeps
 *   makes before it gives up (0 restores the default, about one second).
 * SF_DEBUG_SKIP_TASKS: the down sweep's task queue starts at this task, so
 *   the skipped tasks never run and the bands after them wait for flags that
 *   nothing sets; the waits run out, set the workspace error word
 *   (sf_check_workspace then returns SF_ERR_TIMEOUT) and the kernels return
 *   normally.  0 (the default) skips nothing.
 * SF_DEBUG_HLINE_DC: disparities per thread of the horizontal-path kernel for
 *   D > 64: 4 for a whole warp per line pair (4 disparities a lane up to
 *   D = 128, 8 above), or 16 or 32; 0 restores the default, 4.  Results are
 *   identical.
 * Process-wide; not for production use. */
#define SF_DEBUG_SPIN_LIMIT 1
#define SF_DEBUG_SKIP_TASKS 2
#define SF_DEBUG_HLINE_DC 3
sf_status sf_debug_set(int32_t key, int64_t value);

/* Process-wide choice between the fused stereo kernels (1, default) and the
 * staged kernels (0: stored cost volume, one kernel per path, separate
 * selection).  Both compute the same integers; the staged kernels also serve
 * the request the fused ones do not take (D not a multiple of 16 in
 * sf_sgm_aggregate). */
sf_status sf_set_fused(int32_t enable);

/* Reads the device-side error word of a workspace used by sf_sgm_full
 * (npairs = 1) or sf_scene_flow (npairs = 2) with these sizes; waits for
 * `stream`.  Returns SF_ERR_TIMEOUT if a bounded inter-CTA wait of the band
 * sweeps gave up (the outputs of that call are then invalid), SF_OK
 * otherwise. */
sf_status sf_check_workspace(const void* workspace, int32_t W, int32_t H, const sf_sgm_params* p,
                             int32_t npairs, void* stream);

/* ==== Learned confidence ====================================================
 * No counterpart in the paper: the paper keeps a disparity where the
 * left-right check of Sec. 3.1 passes, which costs a second SGM pass with the
 * right image as reference.  These calls predict that check's outcome from
 * the left pass alone, with a small network trained on labels made by the
 * check itself.
 *
 * Features (bfloat16 [H][W][8], per pixel of the left pass, S = sum of the
 * eight paths, d* its first argmin, S0 = S(d*)):
 *   0  S0 / 1024
 *   1  (S2 - S0) / 256, S2 = min S(d) over |d - d*| >= 2 (S0 if none)
 *   2  curvature / 256: S(d*-1) + S(d*+1) - 2 S0, or 2 (S(nb) - S0) at an end
 *   3  path disagreement / 16: sum over the groups {(+1,0),(-1,0)},
 *      {(0,+1),(+1,+1),(-1,+1)}, {(0,-1),(-1,-1),(+1,-1)} of
 *      min(|d*_group - d*|, 16), d*_group the first argmin of the group's sum
 *   4  d* / 128
 *   5  clamp(x - d*, 0, 64) / 64
 *   6  C(d*) / 64
 *   7  visibility margin / 16: with u(x) = x - d*(x) the right-image column
 *      pixel x matches and m(x) the minimum of u over the pixels right of x
 *      in the same row, clamp(m(x) - u(x), -16, 16); 16 for the last pixel
 *      (<= 0: a pixel to the right covers x's match, x is occluded)
 * Each is an integer over a power of two, rounded once to bfloat16.
 *
 * Network: z1 = b1 + conv3x3(f, W1), a1 = bf16(relu(z1)); a2, a3 likewise
 * with W2, W3 (32 channels); logit z4 = b4 + conv3x3(a3, W4); probability
 * sigmoid(z4).  Zero padding, weights rounded to bfloat16, fp32 biases and
 * accumulation.  A pixel is accepted iff x - d* >= 0 and prob >= threshold.
 * Parameters (fp32, this order): W1 [32][3][3][8], b1 [32], W2 [32][3][3][32],
 * b2 [32], W3 [32][3][3][32], b3 [32], W4 [1][3][3][32], b4 [1]. */
#define SF_CONFNET_FEATURES 8
#define SF_CONFNET_CHANNELS 32

/* Number of network parameters (21121). */
int32_t sf_confnet_param_count(void);

/* Seeded initial parameters, written to the device buffer `params` (fp32,
 * sf_confnet_param_count() values, 4-byte aligned): each weight of a layer
 * with ci input channels is sqrt(2 / (9 ci)) times a standard normal sample
 * (He initialisation), each bias 0.  Sample i depends only on (seed, i): a
 * splitmix64 hash of both gives two uniforms, Box-Muller turns them into a
 * normal.  Asynchronous on `stream`. */
sf_status sf_confnet_init(float* params, uint64_t seed, void* stream);

/* Writes the device parameters to a file at `path` (host string): the bytes
 * "SFCN", then little-endian uint32 version (1), features (8), channels (32),
 * count (21121), then count float32 values in the order above.  Copies
 * synchronously on the legacy default stream, which does not wait for
 * non-blocking streams: finish the work that wrote `params` first.  A file
 * that cannot be written returns SF_ERR_INVALID_ARG. */
sf_status sf_confnet_save(const float* params, const char* path);

/* Reads a file written by sf_confnet_save into the device buffer `params`.
 * A missing file, another format, version or size, or trailing bytes return
 * SF_ERR_INVALID_ARG and leave `params` unchanged. */
sf_status sf_confnet_load(const char* path, float* params);

/* Bytes of the packed inference weights written by sf_confnet_pack. */
size_t sf_confnet_packed_bytes(void);

/* Packs device fp32 parameters into the device blob `packed` (16-byte
 * aligned, sf_confnet_packed_bytes() bytes) used by the inference calls. */
sf_status sf_confnet_pack(const float* params, void* packed, void* stream);

/* Network inference on the tensor cores.  features: bf16 [H][W][8];
 * dint, dsub: the left pass's winners (needed for valid_out / disp_out);
 * prob_out: float [H][W] or NULL; valid_out: uint8 [H][W] or NULL
 * (1 = accepted); disp_out: float [H][W] or NULL (dsub where accepted, NaN
 * elsewhere).  All device pointers.  The kernel's waits for its own
 * tensor-core work are bounded; should one give up, the outputs of the tiles
 * not yet done stay unwritten (the learned-path calls report that case as
 * SF_ERR_TIMEOUT through their workspace error word; this call has none). */
sf_status sf_confnet_infer(const void* packed, const uint16_t* features, const int16_t* dint,
                           const float* dsub, int32_t W, int32_t H, float threshold, float* prob_out,
                           uint8_t* valid_out, float* disp_out, void* stream);

/* Optimiser settings of one training step: Adam (bias-corrected, step >= 1)
 * on the loss sum(w (softplus(z) - y z)) / sum(w), w = 1 for label 1, w_neg
 * for label 0, 0 for label 255. */
typedef struct {
  float lr, beta1, beta2, eps, w_neg;
  int32_t step;
} sf_confnet_hparams;

/* Workspace bytes of sf_confnet_train_step for a batch of B images of W x H. */
size_t sf_confnet_train_workspace_size(int32_t B, int32_t W, int32_t H);

/* One training step on the CUDA cores: forward with the inference roundings
 * (bf16 weights and activations, fp32 sums), loss, gradients (rounding taken
 * as identity), then Adam on `params` (skipped when adam_m or adam_v is
 * NULL).  features: bf16 [B][H][W][8]; labels: uint8 [B][H][W] or NULL
 * (forward only); grad_out: float [param_count] or NULL (gradient before the
 * update); loss_out: one device float or NULL; logits_out: float [B][H][W]
 * or NULL.  All device pointers except hp. */
sf_status sf_confnet_train_step(float* params, float* adam_m, float* adam_v, const uint16_t* features,
                                const uint8_t* labels, int32_t B, int32_t W, int32_t H,
                                const sf_confnet_hparams* hp, float* grad_out, float* loss_out,
                                float* logits_out, void* workspace, size_t ws_bytes, void* stream);

/* The Adam update alone, with a given gradient (device, param_count floats). */
sf_status sf_confnet_adam(float* params, float* adam_m, float* adam_v, const float* grad,
                          const sf_confnet_hparams* hp, void* stream);

/* Workspace bytes of sf_sgm_learned (npairs = 1), sf_scene_flow_learned
 * (npairs = 2) or sf_scene_flow_learned_frames (npairs = 2 n); npairs <= 4. */
size_t sf_learned_workspace_size(int32_t W, int32_t H, const sf_sgm_params* p, int32_t npairs);

/* Stereo with learned confidence: census, the left-reference cost, the eight
 * paths (path_mask must be 0xFF), the features, then (packed != NULL) the
 * network and the acceptance rule.  dint_out: int16 [H][W] or NULL;
 * features_out: bf16 [H][W][8] or NULL; prob_out, valid_out, disp_out as in
 * sf_confnet_infer (ignored when packed is NULL). */
sf_status sf_sgm_learned(const uint8_t* left, const uint8_t* right, int32_t W, int32_t H,
                         int32_t pitch, const sf_sgm_params* p, const void* packed, float threshold,
                         int16_t* dint_out, float* prob_out, uint8_t* valid_out, float* disp_out,
                         uint16_t* features_out, void* workspace, size_t ws_bytes, void* stream);

/* Scene flow with learned confidence in place of both left-right checks:
 * D0 and D1 from sf_sgm_learned on the pairs at t and t+1, then the
 * combination of Sec. 3.3 exactly as in sf_scene_flow.  Outputs as in
 * sf_scene_flow; workspace of sf_learned_workspace_size(W, H, p, 2). */
sf_status sf_scene_flow_learned(const uint8_t* left_t, const uint8_t* right_t, const uint8_t* left_t1,
                                const uint8_t* right_t1, int32_t pitch, const float* flow, int32_t W,
                                int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                                const void* packed, float threshold, float* s4_out, float* motion_out,
                                float* point_out, uint8_t* valid_out, float* D0_out, float* D1_out,
                                void* workspace, size_t ws_bytes, void* stream);

/* One frame of sf_scene_flow_learned_frames: the four images (same pitch
 * and size for every frame), the flow and the outputs, as in
 * sf_scene_flow_learned. */
typedef struct {
  const uint8_t* left_t;
  const uint8_t* right_t;
  const uint8_t* left_t1;
  const uint8_t* right_t1;
  const float* flow;
  float* s4_out;
  float* motion_out;
  float* point_out;
  uint8_t* valid_out;
  float* D0_out;
  float* D1_out;
} sf_learned_frame;

/* sf_scene_flow_learned for n frames of one size (n = 1 or 2): their 2n
 * left passes share the sweep launches, so two frames keep as many SMs busy
 * as the four passes of one plain frame.  Workspace of
 * sf_learned_workspace_size(W, H, p, 2 n). */
sf_status sf_scene_flow_learned_frames(const sf_learned_frame* frames, int32_t n, int32_t pitch, int32_t W,
                                       int32_t H, const sf_sgm_params* p, const sf_camera* cam,
                                       const void* packed, float threshold, void* workspace, size_t ws_bytes,
                                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SF_H_ */
