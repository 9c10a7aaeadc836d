"""CPU oracle for the SGM + scene-flow hot path (arXiv 1801.04720).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this module.  The CUDA product path never
calls it and shares no code with it.

The arithmetic lives in ``sgm_oracle.c`` (plain C loops, integers exact,
subpixel and scene flow in float64); this module builds it with gcc, loads it
with ctypes and adapts numpy arrays.  Each function names the passage of the
paper it follows:

* census / cost: the matching cost of SGM (Sec. 3.1 names SGM, citing
  Hirschmueller 2008); census window, P1, P2 and D are the method's parameters.
* ``path_cost`` / ``aggregate``: the eight-path semi-global aggregation
  (Sec. 3.1, "eight different paths"); with a guide image, the P2 of each
  path step adapts to the intensity step as in the cited SGM (Hirschmueller
  2008): P2 / |I(p) - I(p-r)| rounded down, never below P1.
* ``uniqueness``: removes winners whose cost is not clearly below every
  disparity two or more away (a post-filter of SGM implementations).
* ``select``: winner-take-all with parabolic subpixel refinement.
* ``lr_check``: the left-right consistency check that makes the disparity map
  non-dense (Sec. 3.1).
* ``combine``: Eq. 3-5 of Sec. 3.3, with the back-projection Z = fB/d.
* ``chain``: more than two frames (the paper's future work, Sec. 5): the
  reference pixel followed through every frame by the flows, each
  intermediate frame's disparity validating the chain, and its 3D point in
  every frame; two frames give the combination of Sec. 3.3.
* ``fill`` / ``densify``: filling the gaps of the sparse result, the paper's
  future work (Sec. 5); Table 1's dense rows come from the benchmark's own
  background fill of a sparse submission (Sec. 4.1).  Background fill, or an
  edge-aware choice by guide intensity; then the back-projection of Sec. 3.3
  at every filled pixel.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(brute force, closed forms, invariants).  The exact subpixel value of a real
scene has no pin beyond its closed form on integer inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# The eight traversal directions r = (rx, ry), in path-mask bit order.
DIRECTIONS = [(+1, 0), (-1, 0), (0, +1), (0, -1), (+1, +1), (-1, -1), (+1, -1), (-1, +1)]


def build(force: bool = False) -> str:
    """Compile sgm_oracle.c into a shared library with gcc (plain -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        # every floating-point operation rounded on its own (no fused
        # multiply-add contraction, which some targets apply by default)
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                        "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i = ctypes.c_int
            d = ctypes.c_double
            lib.oracle_census.argtypes = [P, i, i, i, i, P]
            lib.oracle_cost.argtypes = [P, P, i, i, i, i, i, P]
            lib.oracle_path.argtypes = [P, i, i, i, i, i, i, i, P]
            lib.oracle_path_guided.argtypes = [P, P, i, i, i, i, i, i, i, P]
            lib.oracle_aggregate.argtypes = [P, i, i, i, i, i, ctypes.c_uint32, P, P]
            lib.oracle_aggregate_guided.argtypes = [P, P, i, i, i, i, i, ctypes.c_uint32, P, P]
            lib.oracle_uniqueness.argtypes = [P, i, i, i, i, P, P]
            lib.oracle_fill.argtypes = [P, P, i, i, i, P, P]
            lib.oracle_densify.argtypes = [P, P, P, i, i, i, d, d, d, d, P, P, P, P, P]
            lib.oracle_chain.argtypes = [P, P, i, i, i, d, d, d, d, P, P]
            lib.oracle_select.argtypes = [P, i, i, i, i, P, P]
            lib.oracle_lr_check.argtypes = [P, P, P, i, i, i, P, P]
            lib.oracle_combine.argtypes = [P, P, P, i, i, d, d, d, d, P, P, P, P]
            for fn in ("oracle_census", "oracle_cost", "oracle_path", "oracle_aggregate",
                       "oracle_select", "oracle_lr_check", "oracle_combine", "oracle_path_guided",
                       "oracle_aggregate_guided", "oracle_uniqueness", "oracle_fill", "oracle_densify",
                       "oracle_chain"):
                getattr(lib, fn).restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def census(img: np.ndarray, cw: int = 9, ch: int = 7) -> np.ndarray:
    """Census transform (uint64 per pixel), clamped border, strict '<'."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), dtype=np.uint64)
    _load().oracle_census(_ptr(img), W, H, cw, ch, _ptr(out))
    return out


def cost_volume(c_ref: np.ndarray, c_other: np.ndarray, D: int, ref_is_right: bool = False,
                cmax: int = 62) -> np.ndarray:
    """Hamming matching cost uint8 [H][W][D]; out-of-image candidates cost cmax."""
    c_ref = np.ascontiguousarray(c_ref, dtype=np.uint64)
    c_other = np.ascontiguousarray(c_other, dtype=np.uint64)
    H, W = c_ref.shape
    out = np.empty((H, W, D), dtype=np.uint8)
    _load().oracle_cost(_ptr(c_ref), _ptr(c_other), W, H, D, int(ref_is_right), cmax, _ptr(out))
    return out


def _guide(img, H, W):
    if img is None:
        return None, None
    g = np.ascontiguousarray(img, dtype=np.uint8)
    assert g.shape == (H, W)
    return g, _ptr(g)


def path_cost(cost: np.ndarray, P1: int, P2: int, r: tuple[int, int], img=None) -> np.ndarray:
    """L_r for one traversal direction r = (rx, ry), int32 [H][W][D].  With a
    guide image (uint8 [H][W]) the P2 of each step is intensity-adaptive."""
    cost = np.ascontiguousarray(cost, dtype=np.uint8)
    H, W, D = cost.shape
    out = np.empty((H, W, D), dtype=np.int32)
    g, gp = _guide(img, H, W)
    _load().oracle_path_guided(_ptr(cost), gp, W, H, D, P1, P2, r[0], r[1], _ptr(out))
    return out


def aggregate(cost: np.ndarray, P1: int, P2: int, path_mask: int = 0xFF, img=None) -> np.ndarray:
    """S = sum of L_r over the enabled paths, int32 [H][W][D]."""
    cost = np.ascontiguousarray(cost, dtype=np.uint8)
    H, W, D = cost.shape
    S = np.empty((H, W, D), dtype=np.int32)
    scratch = np.empty((H, W, D), dtype=np.int32)
    g, gp = _guide(img, H, W)
    _load().oracle_aggregate_guided(_ptr(cost), gp, W, H, D, P1, P2, path_mask & 0xFF, _ptr(S),
                                    _ptr(scratch))
    return S


def uniqueness(S: np.ndarray, dint: np.ndarray, dsub: np.ndarray, ratio: int) -> np.ndarray:
    """Copy of dsub with NaN where the winner is not unique:
    100 * min_{|d - d*| >= 2} S(d) < (100 + ratio) * S(d*)."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    H, W, D = S.shape
    dint = np.ascontiguousarray(dint, dtype=np.int16)
    out = np.array(dsub, dtype=np.float64, copy=True, order="C")
    _load().oracle_uniqueness(_ptr(S), W, H, D, int(ratio), _ptr(dint), _ptr(out))
    return out


def select(S: np.ndarray, subpixel: bool = True):
    """Winner-take-all (smallest d on ties) and parabolic subpixel (float64)."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    H, W, D = S.shape
    dint = np.empty((H, W), dtype=np.int16)
    dsub = np.empty((H, W), dtype=np.float64)
    _load().oracle_select(_ptr(S), W, H, D, int(subpixel), _ptr(dint), _ptr(dsub))
    return dint, dsub


def lr_check(dL: np.ndarray, dR: np.ndarray, dL_sub: np.ndarray, tol: int = 1):
    """Left-right consistency check: (valid uint8, disparity float64 with NaN)."""
    dL = np.ascontiguousarray(dL, dtype=np.int16)
    dR = np.ascontiguousarray(dR, dtype=np.int16)
    dL_sub = np.ascontiguousarray(dL_sub, dtype=np.float64)
    H, W = dL.shape
    valid = np.empty((H, W), dtype=np.uint8)
    disp = np.empty((H, W), dtype=np.float64)
    _load().oracle_lr_check(_ptr(dL), _ptr(dR), _ptr(dL_sub), W, H, tol, _ptr(valid), _ptr(disp))
    return valid, disp


def combine(D0: np.ndarray, D1: np.ndarray, flow: np.ndarray, f: float, B: float,
            cx: float, cy: float):
    """Scene flow by Eq. 3-5: returns (s4, motion, point, valid)."""
    D0 = np.ascontiguousarray(D0, dtype=np.float64)
    D1 = np.ascontiguousarray(D1, dtype=np.float64)
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    H, W = D0.shape
    s4 = np.empty((H, W, 4), dtype=np.float64)
    motion = np.empty((H, W, 3), dtype=np.float64)
    point = np.empty((H, W, 3), dtype=np.float64)
    valid = np.empty((H, W), dtype=np.uint8)
    _load().oracle_combine(_ptr(D0), _ptr(D1), _ptr(flow), W, H, f, B, cx, cy, _ptr(s4),
                           _ptr(motion), _ptr(point), _ptr(valid))
    return s4, motion, point, valid


def sgm_pass(ref_census: np.ndarray, other_census: np.ndarray, D: int, P1: int, P2: int,
             ref_is_right: bool, cmax: int, path_mask: int = 0xFF, subpixel: bool = True,
             guide=None, unique: int = 0):
    """One SGM pass: cost, aggregation (intensity-adaptive P2 when `guide`,
    the pass's reference image, is given), selection, and the uniqueness
    filter when unique > 0.  Returns (dint, dsub)."""
    C = cost_volume(ref_census, other_census, D, ref_is_right, cmax)
    S = aggregate(C, P1, P2, path_mask, img=guide)
    dint, dsub = select(S, subpixel)
    if unique:
        dsub = uniqueness(S, dint, dsub, unique)
    return dint, dsub


def disparity(left: np.ndarray, right: np.ndarray, D: int = 128, P1: int = 7, P2: int = 86,
              cw: int = 9, ch: int = 7, tol: int = 1, path_mask: int = 0xFF,
              subpixel: bool = True, adaptive_p2: bool = False, uniqueness: int = 0):
    """Full SGM disparity for one stereo pair with the left-right check.

    adaptive_p2: each pass adapts P2 to its reference image's intensity
    steps.  uniqueness: ratio in percent of the filter on the left winners
    (0 = off); a removed winner fails the check.

    Returns a dict with dL, dR (int16), dL_sub (float64), valid (uint8) and
    disp (float64, NaN where the check failed)."""
    cmax = cw * ch - 1
    cL = census(left, cw, ch)
    cR = census(right, cw, ch)
    dL, dL_sub = sgm_pass(cL, cR, D, P1, P2, False, cmax, path_mask, subpixel,
                          guide=left if adaptive_p2 else None, unique=uniqueness)
    dR, _ = sgm_pass(cR, cL, D, P1, P2, True, cmax, path_mask, subpixel,
                     guide=right if adaptive_p2 else None)
    valid, disp = lr_check(dL, dR, dL_sub, tol)
    return {"dL": dL, "dR": dR, "dL_sub": dL_sub, "valid": valid, "disp": disp}


def scene_flow(quad, flow: np.ndarray, f: float, B: float, cx: float, cy: float, **sgm_kw):
    """The whole path: SGM at t and t+1, then the combination of Eq. 4-5.

    quad = (left_t, right_t, left_t1, right_t1)."""
    r0 = disparity(quad[0], quad[1], **sgm_kw)
    r1 = disparity(quad[2], quad[3], **sgm_kw)
    s4, motion, point, valid = combine(r0["disp"], r1["disp"], flow, f, B, cx, cy)
    return {"t0": r0, "t1": r1, "s4": s4, "motion": motion, "point": point, "valid": valid}


def fill(a: np.ndarray, guide=None, mode: int = 0) -> np.ndarray:
    """Fill of a sparse map (NaN = missing): rows first, then the columns for
    the rows left empty; mode 0 background (smaller bounding value), mode 1
    edge-aware (bounding value of the closer guide intensity, smaller on a
    tie).  float64 [H][W]."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    H, W = a.shape
    g, gp = _guide(guide, H, W)
    if mode == 1 and g is None:
        raise ValueError("the edge-aware fill needs a guide image")
    out = np.empty((H, W), dtype=np.float64)
    rows = np.empty((H, W), dtype=np.float64)
    _load().oracle_fill(_ptr(a), gp, int(mode), W, H, _ptr(out), _ptr(rows))
    return out


def densify(s4: np.ndarray, flow: np.ndarray, f: float, B: float, cx: float, cy: float, guide=None,
            mode: int = 0):
    """Dense scene flow from a sparse s4 [H][W][4] (NaN where undefined):
    returns (s4, motion, point, valid) with d0 and d1 filled by ``fill``."""
    s4 = np.ascontiguousarray(s4, dtype=np.float64)
    H, W = s4.shape[:2]
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    g, gp = _guide(guide, H, W)
    if mode == 1 and g is None:
        raise ValueError("the edge-aware fill needs a guide image")
    s4o = np.empty((H, W, 4))
    motion = np.empty((H, W, 3))
    point = np.empty((H, W, 3))
    valid = np.empty((H, W), dtype=np.uint8)
    scratch = np.empty(5 * H * W)
    _load().oracle_densify(_ptr(s4), _ptr(flow), gp, int(mode), W, H, f, B, cx, cy, _ptr(s4o), _ptr(motion),
                           _ptr(point), _ptr(valid), _ptr(scratch))
    return s4o, motion, point, valid


def chain(disps, flows, f: float, B: float, cx: float, cy: float):
    """Trajectories through K frames: disps K maps float64 [H][W] (NaN =
    removed), flows K-1 maps float32 [H][W][2].  Returns (points float64
    [K][H][W][3], valid uint8 [H][W])."""
    K = len(disps)
    assert len(flows) == K - 1 and K >= 2
    D = [np.ascontiguousarray(d, dtype=np.float64) for d in disps]
    F = [np.ascontiguousarray(fl, dtype=np.float32) for fl in flows]
    H, W = D[0].shape
    dp = (ctypes.c_void_p * K)(*[d.ctypes.data for d in D])
    fp = (ctypes.c_void_p * max(K - 1, 1))(*([fl.ctypes.data for fl in F] or [0]))
    points = np.empty((K, H, W, 3))
    valid = np.empty((H, W), dtype=np.uint8)
    _load().oracle_chain(ctypes.cast(dp, ctypes.c_void_p), ctypes.cast(fp, ctypes.c_void_p), K, W, H, f, B, cx, cy,
                         _ptr(points), _ptr(valid))
    return points, valid
