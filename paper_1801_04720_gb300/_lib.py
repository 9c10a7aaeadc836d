"""Thin ctypes binding of libsf (include/sf.h).

Argument marshalling only: every step of the path runs in libsf's CUDA
kernels.  Functions take torch tensors that already live on the GPU (device
memory and streams are PyTorch's), pass their data pointers and the current
CUDA stream, and raise ``SFError`` on a non-OK status.  If libsf.so is missing
the first call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsf.so")

SF_OK = 0
STATUS_NAMES = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_UNSUPPORTED", 3: "SF_ERR_CUDA",
                4: "SF_ERR_TIMEOUT"}

# The functions include/sf.h declares (checked by the CPU export test).
EXPORTED = [
    "sf_default_params", "sf_status_string", "sf_census", "sf_cost_volume",
    "sf_aggregate_workspace_size", "sf_sgm_aggregate", "sf_disparity_select", "sf_lr_check",
    "sf_combine_sceneflow", "sf_workspace_size", "sf_sgm_full", "sf_scene_flow",
    "sf_scene_flow_host_workspace_size", "sf_scene_flow_host", "sf_trace_arm",
    "sf_trace_disarm", "sf_kernel_launches", "sf_set_fused", "sf_check_workspace",
    "sf_batch_workspace_size", "sf_batch_run", "sf_batch_release_graphs", "sf_set_sweep_shape",
    "sf_set_sweep_schedule", "sf_set_learned_sweep_schedule", "sf_sgm_aggregate_guided", "sf_fill_disparity", "sf_densify_sceneflow",
    "sf_chain_sceneflow", "sf_sequence_workspace_size", "sf_sequence_sceneflow", "sf_set_batch_wave_limit",
    "sf_sgm_aggregate_noalloc", "sf_confnet_param_count", "sf_confnet_packed_bytes",
    "sf_confnet_pack", "sf_confnet_infer", "sf_confnet_train_workspace_size",
    "sf_confnet_train_step", "sf_confnet_adam", "sf_learned_workspace_size", "sf_sgm_learned",
    "sf_scene_flow_learned", "sf_scene_flow_learned_frames", "sf_debug_set",
    "sf_pipeline_create", "sf_pipeline_submit", "sf_pipeline_wait", "sf_pipeline_destroy",
    "sf_confnet_init", "sf_confnet_save", "sf_confnet_load",
]

SF_DEBUG_SPIN_LIMIT = 1
SF_DEBUG_SKIP_TASKS = 2
SF_DEBUG_HLINE_DC = 3

SF_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

SF_BATCH_GRAPH = 1

STAGE_NAMES = ["census", "cost", "aggregate", "select", "lrcheck", "combine", "sgm_sweep",
               "features", "confnet", "densify"]

SF_FILL_BACKGROUND = 0
SF_FILL_EDGE_AWARE = 1


class SFError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} returned {STATUS_NAMES.get(status, status)}")


class SgmParams(ctypes.Structure):
    _fields_ = [("census_w", ctypes.c_int32), ("census_h", ctypes.c_int32),
                ("P1", ctypes.c_uint16), ("P2", ctypes.c_uint16), ("path_mask", ctypes.c_uint32),
                ("D", ctypes.c_int32), ("subpixel", ctypes.c_int32), ("lr_tol", ctypes.c_int32),
                ("adaptive_p2", ctypes.c_int32), ("uniqueness", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("f", ctypes.c_float), ("B", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float)]


class BatchItem(ctypes.Structure):
    _fields_ = [("left_t", ctypes.c_void_p), ("right_t", ctypes.c_void_p),
                ("left_t1", ctypes.c_void_p), ("right_t1", ctypes.c_void_p),
                ("pitch", ctypes.c_int32), ("flow", ctypes.c_void_p), ("W", ctypes.c_int32),
                ("H", ctypes.c_int32), ("D", ctypes.c_int32), ("cam", Camera),
                ("s4_out", ctypes.c_void_p), ("motion_out", ctypes.c_void_p),
                ("point_out", ctypes.c_void_p), ("valid_out", ctypes.c_void_p),
                ("D0_out", ctypes.c_void_p), ("D1_out", ctypes.c_void_p)]


class ConfnetHparams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("w_neg", ctypes.c_float), ("step", ctypes.c_int32)]


def hparams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, w_neg=1.0, step=1):
    return ConfnetHparams(lr, beta1, beta2, eps, w_neg, step)


def params(D=128, P1=7, P2=86, census_w=9, census_h=7, path_mask=0xFF, subpixel=True, lr_tol=1,
           adaptive_p2=False, uniqueness=0):
    return SgmParams(census_w, census_h, P1, P2, path_mask, D, int(subpixel), lr_tol, int(adaptive_p2),
                     int(uniqueness))


def camera(f, B, cx, cy):
    return Camera(f, B, cx, cy)


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libsf.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libsf.so not found at {path}: run __graft_entry__.build() "
                               "(the CUDA library is required; there is no fallback)")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        sz = ctypes.c_size_t
        PP = ctypes.POINTER(SgmParams)
        PC = ctypes.POINTER(Camera)
        PH = ctypes.POINTER(ConfnetHparams)
        sig = {
            "sf_default_params": (None, [PP]),
            "sf_status_string": (ctypes.c_char_p, [i32]),
            "sf_census": (i32, [P, i32, i32, i32, i32, i32, P, P]),
            "sf_cost_volume": (i32, [P, P, i32, i32, i32, PP, i32, P, P]),
            "sf_aggregate_workspace_size": (sz, [i32, i32, PP]),
            "sf_sgm_aggregate": (i32, [P, i32, i32, PP, P, P, sz, P]),
            "sf_sgm_aggregate_noalloc": (i32, [P, i32, i32, PP, P, P, P]),
            "sf_disparity_select": (i32, [P, i32, i32, i32, i32, P, P, P]),
            "sf_lr_check": (i32, [P, P, P, i32, i32, i32, P, P, P]),
            "sf_combine_sceneflow": (i32, [P, P, P, i32, i32, PC, P, P, P, P, P]),
            "sf_workspace_size": (sz, [i32, i32, PP]),
            "sf_sgm_full": (i32, [P, P, i32, i32, i32, PP, P, P, P, P, P, sz, P]),
            "sf_scene_flow": (i32, [P, P, P, P, i32, P, i32, i32, PP, PC, P, P, P, P, P, P, P, sz, P]),
            "sf_scene_flow_host_workspace_size": (sz, [i32, i32, PP]),
            "sf_scene_flow_host": (i32, [P, P, P, P, P, i32, i32, PP, PC, P, P, P, P, P, sz, P]),
            "sf_pipeline_create": (i32, [i32, i32, PP, PC, i32, ctypes.POINTER(P)]),
            "sf_pipeline_submit": (i32, [P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int64)]),
            "sf_pipeline_wait": (i32, [P, ctypes.c_int64]),
            "sf_pipeline_destroy": (i32, [P]),
            "sf_trace_arm": (i32, [P, i32, P]),
            "sf_trace_disarm": (i32, []),
            "sf_kernel_launches": (ctypes.c_uint64, []),
            "sf_set_fused": (i32, [i32]),
            "sf_batch_workspace_size": (sz, [P, i32, PP]),
            "sf_batch_run": (i32, [P, i32, PP, ctypes.c_uint32, P, sz, P]),
            "sf_batch_release_graphs": (None, []),
            "sf_set_sweep_shape": (i32, [i32, i32, i32, i32]),
            "sf_set_sweep_schedule": (i32, [i32, i32, i32, i32, i32]),
            "sf_set_learned_sweep_schedule": (i32, [i32, i32, i32, i32, i32]),
            "sf_sgm_aggregate_guided": (i32, [P, P, i32, i32, i32, PP, P, P, sz, P]),
            "sf_fill_disparity": (i32, [P, i32, i32, P, i32, i32, P, P]),
            "sf_chain_sceneflow": (i32, [P, P, i32, i32, i32, PC, P, P, P]),
            "sf_set_batch_wave_limit": (i32, [sz]),
            "sf_sequence_workspace_size": (sz, [i32, i32, PP, i32, i32]),
            "sf_sequence_sceneflow": (i32, [P, P, i32, i32, P, i32, i32, PP, PC, P, ctypes.c_float, P, P, P, P,
                                            P, P, P, sz, P]),
            "sf_densify_sceneflow": (i32, [P, P, i32, i32, PC, P, i32, i32, P, P, P, P, P]),
            "sf_check_workspace": (i32, [P, i32, i32, PP, i32, P]),
            "sf_debug_set": (i32, [i32, ctypes.c_int64]),
            "sf_scene_flow_learned_frames": (i32, [P, i32, i32, i32, i32, PP, PC, P, ctypes.c_float, P, sz,
                                                   P]),
            "sf_confnet_param_count": (i32, []),
            "sf_confnet_init": (i32, [P, ctypes.c_uint64, P]),
            "sf_confnet_save": (i32, [P, ctypes.c_char_p]),
            "sf_confnet_load": (i32, [ctypes.c_char_p, P]),
            "sf_confnet_packed_bytes": (sz, []),
            "sf_confnet_pack": (i32, [P, P, P]),
            "sf_confnet_infer": (i32, [P, P, P, P, i32, i32, ctypes.c_float, P, P, P, P]),
            "sf_confnet_train_workspace_size": (sz, [i32, i32, i32]),
            "sf_confnet_train_step": (i32, [P, P, P, P, P, i32, i32, i32, PH, P, P, P, P, sz, P]),
            "sf_confnet_adam": (i32, [P, P, P, P, PH, P]),
            "sf_learned_workspace_size": (sz, [i32, i32, PP, i32]),
            "sf_sgm_learned": (i32, [P, P, i32, i32, i32, PP, P, ctypes.c_float, P, P, P, P, P, P,
                                     sz, P]),
            "sf_scene_flow_learned": (i32, [P, P, P, P, i32, P, i32, i32, PP, PC, P, ctypes.c_float,
                                            P, P, P, P, P, P, P, sz, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(fn, st):
    if st != SF_OK:
        raise SFError(fn, st)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CUDA tensor of dtype {dtype}")
    return t


# ---- calls with the ABI's names ------------------------------------------

def sf_census(img, cw=9, ch=7, out=None, stream=None):
    _dev(img, torch.uint8, "img")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.int64, device=img.device)
    _check("sf_census", load().sf_census(_ptr(img), W, H, img.stride(0), cw, ch, _ptr(out),
                                         _stream(stream)))
    return out


def sf_cost_volume(ref, other, p: SgmParams, ref_is_right=False, out=None, stream=None):
    _dev(ref, torch.uint8, "ref")
    _dev(other, torch.uint8, "other")
    H, W = ref.shape
    if out is None:
        out = torch.empty((H, W, p.D), dtype=torch.uint8, device=ref.device)
    _check("sf_cost_volume", load().sf_cost_volume(_ptr(ref), _ptr(other), W, H, ref.stride(0),
                                                   ctypes.byref(p), int(ref_is_right), _ptr(out),
                                                   _stream(stream)))
    return out


def sf_aggregate_workspace_size(W, H, p: SgmParams):
    return int(load().sf_aggregate_workspace_size(W, H, ctypes.byref(p)))


def sf_sgm_aggregate(cost, p: SgmParams, out=None, ws="auto", stream=None):
    """ws="auto" allocates the fused-path workspace; ws=None runs the staged
    kernels (one per path)."""
    _dev(cost, torch.uint8, "cost")
    H, W, D = cost.shape
    if D != p.D:
        raise ValueError("cost volume depth must equal p.D")
    if out is None:
        out = torch.empty((H, W, D), dtype=torch.int16, device=cost.device)
    if isinstance(ws, str):
        n = sf_aggregate_workspace_size(W, H, p)
        ws = torch.empty(n, dtype=torch.uint8, device=cost.device) if n else None
    nbytes = ws.numel() if ws is not None else 0
    _check("sf_sgm_aggregate", load().sf_sgm_aggregate(_ptr(cost), W, H, ctypes.byref(p), _ptr(out),
                                                       _ptr(ws), nbytes, _stream(stream)))
    return out


def sf_sgm_aggregate_guided(cost, guide, p: SgmParams, out=None, ws="auto", stream=None):
    """sf_sgm_aggregate with the pass's reference image (uint8 [H][W]) as the
    guide of the intensity-adaptive P2."""
    _dev(cost, torch.uint8, "cost")
    _dev(guide, torch.uint8, "guide")
    H, W, D = cost.shape
    if D != p.D or tuple(guide.shape) != (H, W):
        raise ValueError("cost volume depth must equal p.D and the guide be [H][W]")
    if out is None:
        out = torch.empty((H, W, D), dtype=torch.int16, device=cost.device)
    if isinstance(ws, str):
        n = sf_aggregate_workspace_size(W, H, p)
        ws = torch.empty(n, dtype=torch.uint8, device=cost.device) if n else None
    nbytes = ws.numel() if ws is not None else 0
    _check("sf_sgm_aggregate_guided",
           load().sf_sgm_aggregate_guided(_ptr(cost), _ptr(guide), guide.stride(0), W, H, ctypes.byref(p),
                                          _ptr(out), _ptr(ws), nbytes, _stream(stream)))
    return out


def sf_sgm_aggregate_noalloc(cost, p: SgmParams, out, err=None, stream=None):
    """S of `cost` into the caller's `out` (uint16/int16 [H][W][D]) with the
    library's built-in scratch: no device allocation.  `err` (one int32 on
    the device, optional) receives the sweeps' bounded-wait status."""
    _dev(cost, torch.uint8, "cost")
    H, W, D = cost.shape
    if D != p.D:
        raise ValueError("cost volume depth must equal p.D")
    _check("sf_sgm_aggregate_noalloc",
           load().sf_sgm_aggregate_noalloc(_ptr(cost), W, H, ctypes.byref(p), _ptr(out), _ptr(err),
                                           _stream(stream)))
    return out


def sf_debug_set(key: int, value: int):
    _check("sf_debug_set", load().sf_debug_set(int(key), int(value)))


def sf_set_fused(enable: bool):
    _check("sf_set_fused", load().sf_set_fused(int(bool(enable))))


def sf_check_workspace(ws, W, H, p: SgmParams, npairs, stream=None):
    """Raises SFError(SF_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check("sf_check_workspace", load().sf_check_workspace(_ptr(ws), W, H, ctypes.byref(p), npairs,
                                                           _stream(stream)))


def sf_disparity_select(agg, subpixel=True, dint=None, dsub=None, stream=None):
    _dev(agg, torch.int16, "agg")
    H, W, D = agg.shape
    if dint is None:
        dint = torch.empty((H, W), dtype=torch.int16, device=agg.device)
    if dsub is None:
        dsub = torch.empty((H, W), dtype=torch.float32, device=agg.device)
    _check("sf_disparity_select", load().sf_disparity_select(_ptr(agg), W, H, D, int(subpixel),
                                                             _ptr(dint), _ptr(dsub), _stream(stream)))
    return dint, dsub


def sf_lr_check(dL, dR, dL_sub, tol=1, valid=None, disp=None, stream=None):
    H, W = dL.shape
    if valid is None:
        valid = torch.empty((H, W), dtype=torch.uint8, device=dL.device)
    if disp is None:
        disp = torch.empty((H, W), dtype=torch.float32, device=dL.device)
    _check("sf_lr_check", load().sf_lr_check(_ptr(dL), _ptr(dR), _ptr(dL_sub), W, H, tol,
                                             _ptr(valid), _ptr(disp), _stream(stream)))
    return valid, disp


def sf_combine_sceneflow(D0, D1, flow, cam: Camera, want_motion=True, want_point=True, out=None,
                         stream=None):
    H, W = D0.shape
    dev = D0.device
    if out is None:
        out = {
            "s4": torch.empty((H, W, 4), dtype=torch.float32, device=dev),
            "motion": torch.empty((H, W, 3), dtype=torch.float32, device=dev) if want_motion else None,
            "point": torch.empty((H, W, 3), dtype=torch.float32, device=dev) if want_point else None,
            "valid": torch.empty((H, W), dtype=torch.uint8, device=dev),
        }
    _check("sf_combine_sceneflow",
           load().sf_combine_sceneflow(_ptr(D0), _ptr(D1), _ptr(flow), W, H, ctypes.byref(cam),
                                       _ptr(out["s4"]), _ptr(out["motion"]), _ptr(out["point"]),
                                       _ptr(out["valid"]), _stream(stream)))
    return out


def sf_fill_disparity(d, guide=None, mode=SF_FILL_BACKGROUND, out=None, stream=None):
    """Fills the NaN entries of a float [H][W] map (densification)."""
    _dev(d, torch.float32, "d")
    H, W = d.shape
    if out is None:
        out = torch.empty_like(d)
    if guide is not None:
        _dev(guide, torch.uint8, "guide")
    _check("sf_fill_disparity", load().sf_fill_disparity(_ptr(d), W, H, _ptr(guide),
                                                         guide.stride(0) if guide is not None else 0,
                                                         int(mode), _ptr(out), _stream(stream)))
    return out


def sf_densify_sceneflow(s4, flow, cam: Camera, guide=None, mode=SF_FILL_BACKGROUND, out=None, stream=None):
    """Dense scene flow from a sparse s4 [H][W][4] (NaN where undefined)."""
    _dev(s4, torch.float32, "s4")
    H, W = s4.shape[:2]
    dev = s4.device
    if out is None:
        out = {"s4": torch.empty((H, W, 4), dtype=torch.float32, device=dev),
               "motion": torch.empty((H, W, 3), dtype=torch.float32, device=dev),
               "point": torch.empty((H, W, 3), dtype=torch.float32, device=dev),
               "valid": torch.empty((H, W), dtype=torch.uint8, device=dev)}
    if guide is not None:
        _dev(guide, torch.uint8, "guide")
    _check("sf_densify_sceneflow",
           load().sf_densify_sceneflow(_ptr(s4), _ptr(flow), W, H, ctypes.byref(cam), _ptr(guide),
                                       guide.stride(0) if guide is not None else 0, int(mode), _ptr(out["s4"]),
                                       _ptr(out["motion"]), _ptr(out["point"]), _ptr(out["valid"]),
                                       _stream(stream)))
    return out


SF_MAX_FRAMES = 64


def _ptr_array(ts):
    """Host array of device pointers (None -> NULL entries)."""
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])
    return ctypes.cast(arr, ctypes.c_void_p), arr


def sf_chain_sceneflow(disps, flows, cam: Camera, points=True, stream=None):
    """Trajectories of frame 0's pixels through K frames: disps K float
    [H][W] maps, flows K-1 float [H][W][2].  Returns {"points" [K][H][W][3],
    "valid" [H][W]}."""
    K = len(disps)
    H, W = disps[0].shape
    dev = disps[0].device
    out = {"points": torch.empty((K, H, W, 3), dtype=torch.float32, device=dev) if points else None,
           "valid": torch.empty((H, W), dtype=torch.uint8, device=dev)}
    dp, _k1 = _ptr_array(disps)
    fp, _k2 = _ptr_array(flows)
    _check("sf_chain_sceneflow", load().sf_chain_sceneflow(dp, fp, K, W, H, ctypes.byref(cam), _ptr(out["points"]),
                                                           _ptr(out["valid"]), _stream(stream)))
    return out


def alloc_sequence_outputs(K, W, H, device="cuda", chain=True, motion=False):
    f32 = torch.float32
    return {"disp": [torch.empty((H, W), dtype=f32, device=device) for _ in range(K)],
            "s4": [torch.empty((H, W, 4), dtype=f32, device=device) for _ in range(K - 1)],
            "valid": [torch.empty((H, W), dtype=torch.uint8, device=device) for _ in range(K - 1)],
            "motion": [torch.empty((H, W, 3), dtype=f32, device=device) for _ in range(K - 1)] if motion else None,
            "points": torch.empty((K, H, W, 3), dtype=f32, device=device) if chain else None,
            "chain_valid": torch.empty((H, W), dtype=torch.uint8, device=device) if chain else None}


def sf_sequence_sceneflow(lefts, rights, flows, p: SgmParams, cam: Camera, packed=None, threshold=0.5,
                          ws=None, chain=True, motion=False, out=None, stream=None):
    """The hot path over K stereo frames, each frame's SGM once; returns
    {"disp": K maps, "s4", "valid", "motion": K-1 each, "points", "chain_valid"}."""
    K = len(lefts)
    H, W = lefts[0].shape
    dev = lefts[0].device
    if ws is None:
        n = load().sf_sequence_workspace_size(W, H, ctypes.byref(p), K, int(packed is not None))
        ws = torch.empty(n, dtype=torch.uint8, device=dev)
    if out is None:
        out = alloc_sequence_outputs(K, W, H, dev, chain=chain, motion=motion)
    motion = out["motion"] is not None
    keep = []
    arrs = []
    for group in (lefts, rights, flows, out["disp"], out["s4"], out["valid"]):
        a, k = _ptr_array(group)
        arrs.append(a)
        keep.append(k)
    mo = None
    if motion:
        mo, k = _ptr_array(out["motion"])
        keep.append(k)
    _check("sf_sequence_sceneflow",
           load().sf_sequence_sceneflow(arrs[0], arrs[1], K, lefts[0].stride(0), arrs[2], W, H, ctypes.byref(p),
                                        ctypes.byref(cam), _ptr(packed), float(threshold), arrs[3], arrs[4], arrs[5],
                                        mo, _ptr(out["points"]), _ptr(out["chain_valid"]), _ptr(ws), ws.numel(),
                                        _stream(stream)))
    return out


def sf_workspace_size(W, H, p: SgmParams):
    return int(load().sf_workspace_size(W, H, ctypes.byref(p)))


def workspace(W, H, p: SgmParams, device="cuda"):
    n = sf_workspace_size(W, H, p)
    if n == 0:
        raise ValueError("invalid size or parameters")
    return torch.empty(n, dtype=torch.uint8, device=device)


def sf_sgm_full(left, right, p: SgmParams, ws=None, out=None, stream=None):
    _dev(left, torch.uint8, "left")
    _dev(right, torch.uint8, "right")
    H, W = left.shape
    dev = left.device
    if ws is None:
        ws = workspace(W, H, p, dev)
    if out is None:
        out = {"dL": torch.empty((H, W), dtype=torch.int16, device=dev),
               "dR": torch.empty((H, W), dtype=torch.int16, device=dev),
               "valid": torch.empty((H, W), dtype=torch.uint8, device=dev),
               "disp": torch.empty((H, W), dtype=torch.float32, device=dev)}
    _check("sf_sgm_full", load().sf_sgm_full(_ptr(left), _ptr(right), W, H, left.stride(0),
                                             ctypes.byref(p), _ptr(out["dL"]), _ptr(out["dR"]),
                                             _ptr(out["valid"]), _ptr(out["disp"]), _ptr(ws),
                                             ws.numel(), _stream(stream)))
    return out


def alloc_scene_flow_outputs(W, H, device="cuda", motion=True, point=True, disparities=True):
    f32 = torch.float32
    return {"s4": torch.empty((H, W, 4), dtype=f32, device=device),
            "motion": torch.empty((H, W, 3), dtype=f32, device=device) if motion else None,
            "point": torch.empty((H, W, 3), dtype=f32, device=device) if point else None,
            "valid": torch.empty((H, W), dtype=torch.uint8, device=device),
            "D0": torch.empty((H, W), dtype=f32, device=device) if disparities else None,
            "D1": torch.empty((H, W), dtype=f32, device=device) if disparities else None}


def sf_scene_flow(imgs, flow, p: SgmParams, cam: Camera, ws=None, out=None, stream=None):
    """imgs = (left_t, right_t, left_t1, right_t1), uint8 [H][W] CUDA tensors."""
    for k, im in enumerate(imgs):
        _dev(im, torch.uint8, f"imgs[{k}]")
    _dev(flow, torch.float32, "flow")
    H, W = imgs[0].shape
    dev = imgs[0].device
    if ws is None:
        ws = workspace(W, H, p, dev)
    if out is None:
        out = alloc_scene_flow_outputs(W, H, dev)
    _check("sf_scene_flow",
           load().sf_scene_flow(_ptr(imgs[0]), _ptr(imgs[1]), _ptr(imgs[2]), _ptr(imgs[3]),
                                imgs[0].stride(0), _ptr(flow), W, H, ctypes.byref(p),
                                ctypes.byref(cam), _ptr(out["s4"]), _ptr(out["motion"]),
                                _ptr(out["point"]), _ptr(out["valid"]), _ptr(out["D0"]),
                                _ptr(out["D1"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def sf_scene_flow_host_workspace_size(W, H, p: SgmParams):
    return int(load().sf_scene_flow_host_workspace_size(W, H, ctypes.byref(p)))


def sf_scene_flow_host(imgs, flow, p: SgmParams, cam: Camera, dev_ws, out, stream=None):
    """Host-buffer variant: imgs / flow / out are CPU tensors (pinned for async
    copies); dev_ws is a CUDA uint8 tensor of sf_scene_flow_host_workspace_size."""
    H, W = imgs[0].shape
    _check("sf_scene_flow_host",
           load().sf_scene_flow_host(_ptr(imgs[0]), _ptr(imgs[1]), _ptr(imgs[2]), _ptr(imgs[3]),
                                     _ptr(flow), W, H, ctypes.byref(p), ctypes.byref(cam),
                                     _ptr(out["s4"]), _ptr(out.get("motion")),
                                     _ptr(out.get("point")), _ptr(out["valid"]), _ptr(dev_ws),
                                     dev_ws.numel(), _stream(stream)))
    return out


class Pipeline:
    """sf_pipeline_*: scene flow of host-memory quadruples of one size, the
    copies of neighbouring frames overlapped with the computation.
    ``submit`` takes CPU tensors (pinned for asynchronous copies) and returns
    a ticket; the frame's outputs are in its ``out`` tensors once ``wait``
    returns for that ticket.  The tensors must stay alive until then."""

    def __init__(self, W, H, p: SgmParams, cam: Camera, depth=2):
        self._h = ctypes.c_void_p()
        _check("sf_pipeline_create", load().sf_pipeline_create(W, H, ctypes.byref(p), ctypes.byref(cam),
                                                               depth, ctypes.byref(self._h)))
        self.W, self.H, self.depth = W, H, depth
        self._held = {}

    def submit(self, imgs, flow, out):
        shapes = [(im, torch.uint8, (self.H, self.W), f"imgs[{k}]") for k, im in enumerate(imgs)]
        shapes += [(flow, torch.float32, (self.H, self.W, 2), "flow"),
                   (out["s4"], torch.float32, (self.H, self.W, 4), "s4"),
                   (out["valid"], torch.uint8, (self.H, self.W), "valid")]
        shapes += [(out[k], torch.float32, (self.H, self.W, 3), k) for k in ("motion", "point")
                   if out.get(k) is not None]
        for t, dt, shape, name in shapes:
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dt or tuple(t.shape) != shape:
                raise ValueError(f"{name}: expected a host {dt} tensor of shape {shape}")
        t = ctypes.c_int64()
        _check("sf_pipeline_submit",
               load().sf_pipeline_submit(self._h, _ptr(imgs[0]), _ptr(imgs[1]), _ptr(imgs[2]), _ptr(imgs[3]),
                                         _ptr(flow), _ptr(out["s4"]), _ptr(out.get("motion")),
                                         _ptr(out.get("point")), _ptr(out["valid"]), ctypes.byref(t)))
        self._held[t.value] = (imgs, flow, out)
        return t.value

    def wait(self, ticket):
        _check("sf_pipeline_wait", load().sf_pipeline_wait(self._h, ticket))
        for k in [k for k in self._held if k <= ticket]:
            del self._held[k]

    def close(self):
        if self._h:
            st = load().sf_pipeline_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._held.clear()
            _check("sf_pipeline_destroy", st)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self._h:
                load().sf_pipeline_destroy(self._h)
        except Exception:
            pass


class StageTracer:
    """Arms libsf's tracer with a pool of CUDA events; after the traced work
    has finished, ``durations()`` returns {stage name: [ms, ...]}."""

    def __init__(self, n_records=4096):
        self.events = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_records)]
        for e in self.events:
            e.record()            # materialise the handles
        torch.cuda.synchronize()
        self._handles = (ctypes.c_void_p * len(self.events))(
            *[ctypes.c_void_p(e.cuda_event) for e in self.events])
        self._stages = (ctypes.c_int32 * n_records)()
        self.records = 0

    def __enter__(self):
        _check("sf_trace_arm", load().sf_trace_arm(self._handles, len(self.events), self._stages))
        return self

    def __exit__(self, *exc):
        self.records = load().sf_trace_disarm()
        return False

    def durations(self):
        torch.cuda.synchronize()
        out = {}
        for k in range(self.records):
            name = STAGE_NAMES[self._stages[k]]
            ms = self.events[2 * k].elapsed_time(self.events[2 * k + 1])
            out.setdefault(name, []).append(ms)
        return out


def kernel_launches():
    return int(load().sf_kernel_launches())


# ---- batches ----------------------------------------------------------------

def _vp(t):
    return t.data_ptr() if t is not None else None


def make_batch(scenes, outs):
    """scenes: list of dicts with CUDA tensors left_t, right_t, left_t1, right_t1,
    flow and ints D plus a Camera cam; outs: matching dicts from
    alloc_scene_flow_outputs.  Returns a ctypes array of BatchItem."""
    arr = (BatchItem * len(scenes))()
    for i, (sc, o) in enumerate(zip(scenes, outs)):
        H, W = sc["left_t"].shape
        arr[i] = BatchItem(_vp(sc["left_t"]), _vp(sc["right_t"]), _vp(sc["left_t1"]),
                           _vp(sc["right_t1"]), sc["left_t"].stride(0), _vp(sc["flow"]), W, H,
                           sc["D"], sc["cam"], _vp(o["s4"]), _vp(o.get("motion")),
                           _vp(o.get("point")), _vp(o["valid"]), _vp(o.get("D0")), _vp(o.get("D1")))
    return arr


def sf_batch_workspace_size(items, p: SgmParams):
    return int(load().sf_batch_workspace_size(items, len(items), ctypes.byref(p)))


def sf_batch_run(items, p: SgmParams, ws, graph=False, stream=None):
    _check("sf_batch_run", load().sf_batch_run(items, len(items), ctypes.byref(p),
                                               SF_BATCH_GRAPH if graph else 0, _ptr(ws), ws.numel(),
                                               _stream(stream)))


def sf_batch_release_graphs():
    load().sf_batch_release_graphs()


def sf_set_batch_wave_limit(nbytes):
    _check("sf_set_batch_wave_limit", load().sf_set_batch_wave_limit(int(nbytes)))


def sf_set_sweep_shape(d_lo, d_hi, dc, halo):
    _check("sf_set_sweep_shape", load().sf_set_sweep_shape(d_lo, d_hi, dc, halo))


def sf_set_sweep_schedule(d_lo, d_hi, dc, halo, order):
    _check("sf_set_sweep_schedule", load().sf_set_sweep_schedule(d_lo, d_hi, dc, halo, order))


def sf_set_learned_sweep_schedule(d_lo, d_hi, dc, halo, order):
    """Schedule of the learned calls; dc = 0 drops the class."""
    _check("sf_set_learned_sweep_schedule",
           load().sf_set_learned_sweep_schedule(d_lo, d_hi, dc, halo, order))


# ---- learned confidence ------------------------------------------------------

def confnet_param_count() -> int:
    return int(load().sf_confnet_param_count())


def confnet_init(seed, device="cuda", stream=None):
    """sf_confnet_init: seeded He-normal parameters (fp32 device tensor)."""
    params = torch.empty(int(load().sf_confnet_param_count()), dtype=torch.float32, device=device)
    _check("sf_confnet_init", load().sf_confnet_init(_ptr(params), int(seed) & (2 ** 64 - 1), _stream(stream)))
    return params


def confnet_save(params, path):
    """sf_confnet_save, after the work queued on this device has finished."""
    _dev(params, torch.float32, "params")
    torch.cuda.synchronize(params.device)
    _check("sf_confnet_save", load().sf_confnet_save(_ptr(params), os.fsencode(path)))


def confnet_load(path, device="cuda"):
    params = torch.empty(int(load().sf_confnet_param_count()), dtype=torch.float32, device=device)
    _check("sf_confnet_load", load().sf_confnet_load(os.fsencode(path), _ptr(params)))
    return params


def confnet_pack(params_t, stream=None):
    """fp32 parameters (device) -> packed bf16 inference blob (device uint8)."""
    _dev(params_t, torch.float32, "params")
    packed = torch.empty(int(load().sf_confnet_packed_bytes()), dtype=torch.uint8,
                         device=params_t.device)
    _check("sf_confnet_pack", load().sf_confnet_pack(_ptr(params_t), _ptr(packed), _stream(stream)))
    return packed


def confnet_infer(packed, features, dint=None, dsub=None, threshold=0.5, prob=True, stream=None):
    """Network inference; returns {"prob", "valid", "disp"} (None where not asked)."""
    H, W = features.shape[0], features.shape[1]
    dev = features.device
    out = {"prob": torch.empty((H, W), dtype=torch.float32, device=dev) if prob else None,
           "valid": torch.empty((H, W), dtype=torch.uint8, device=dev) if dint is not None else None,
           "disp": torch.empty((H, W), dtype=torch.float32, device=dev) if dint is not None else None}
    _check("sf_confnet_infer",
           load().sf_confnet_infer(_ptr(packed), _ptr(features), _ptr(dint), _ptr(dsub), W, H,
                                   float(threshold), _ptr(out["prob"]), _ptr(out["valid"]),
                                   _ptr(out["disp"]), _stream(stream)))
    return out


def confnet_train_workspace(B, W, H, device):
    n = int(load().sf_confnet_train_workspace_size(B, W, H))
    if n == 0:
        raise ValueError("batch too large for one training step")
    return torch.empty(n, dtype=torch.uint8, device=device)


def confnet_train_step(params_t, m, v, features, labels, hp: ConfnetHparams, ws=None, grad=None,
                       loss=None, logits=None, stream=None):
    """features: bf16-as-int16 [B][H][W][8]; labels uint8 [B][H][W] or None."""
    B, H, W = features.shape[0], features.shape[1], features.shape[2]
    if ws is None:
        ws = confnet_train_workspace(B, W, H, features.device)
    _check("sf_confnet_train_step",
           load().sf_confnet_train_step(_ptr(params_t), _ptr(m), _ptr(v), _ptr(features),
                                        _ptr(labels), B, W, H, ctypes.byref(hp), _ptr(grad),
                                        _ptr(loss), _ptr(logits), _ptr(ws), ws.numel(),
                                        _stream(stream)))


def confnet_adam(params_t, m, v, grad, hp: ConfnetHparams, stream=None):
    _check("sf_confnet_adam", load().sf_confnet_adam(_ptr(params_t), _ptr(m), _ptr(v), _ptr(grad),
                                                     ctypes.byref(hp), _stream(stream)))


def learned_workspace(W, H, p: SgmParams, npairs, device):
    n = int(load().sf_learned_workspace_size(W, H, ctypes.byref(p), npairs))
    if n == 0:
        raise ValueError("unsupported learned-path size")
    return torch.empty(n, dtype=torch.uint8, device=device)


def sf_sgm_learned(left, right, p: SgmParams, packed=None, threshold=0.5, ws=None, features=True,
                   stream=None):
    """Left pass + features (+ network when `packed` is given).  Returns
    {"dint", "features", "prob", "valid", "disp"}."""
    H, W = left.shape
    dev = left.device
    if ws is None:
        ws = learned_workspace(W, H, p, 1, dev)
    out = {"dint": torch.empty((H, W), dtype=torch.int16, device=dev),
           "features": torch.empty((H, W, 8), dtype=torch.int16, device=dev) if features else None,
           "prob": torch.empty((H, W), dtype=torch.float32, device=dev) if packed is not None else None,
           "valid": torch.empty((H, W), dtype=torch.uint8, device=dev) if packed is not None else None,
           "disp": torch.empty((H, W), dtype=torch.float32, device=dev) if packed is not None else None}
    _check("sf_sgm_learned",
           load().sf_sgm_learned(_ptr(left), _ptr(right), W, H, W, ctypes.byref(p), _ptr(packed),
                                 float(threshold), _ptr(out["dint"]), _ptr(out["prob"]),
                                 _ptr(out["valid"]), _ptr(out["disp"]), _ptr(out["features"]),
                                 _ptr(ws), ws.numel(), _stream(stream)))
    return out


def sf_scene_flow_learned(images, flow, p: SgmParams, cam: Camera, packed, threshold, ws=None,
                          out=None, stream=None):
    left_t, right_t, left_t1, right_t1 = images
    H, W = left_t.shape
    dev = left_t.device
    if ws is None:
        ws = learned_workspace(W, H, p, 2, dev)
    if out is None:
        out = alloc_scene_flow_outputs(W, H, dev)
    _check("sf_scene_flow_learned",
           load().sf_scene_flow_learned(_ptr(left_t), _ptr(right_t), _ptr(left_t1), _ptr(right_t1),
                                        W, _ptr(flow), W, H, ctypes.byref(p), ctypes.byref(cam),
                                        _ptr(packed), float(threshold), _ptr(out["s4"]),
                                        _ptr(out["motion"]), _ptr(out["point"]), _ptr(out["valid"]),
                                        _ptr(out["D0"]), _ptr(out["D1"]), _ptr(ws), ws.numel(),
                                        _stream(stream)))
    return out


class LearnedFrame(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("left_t", "right_t", "left_t1", "right_t1", "flow",
                                                 "s4_out", "motion_out", "point_out", "valid_out",
                                                 "D0_out", "D1_out")]


def sf_scene_flow_learned_frames(scenes, p: SgmParams, cam: Camera, packed, threshold, ws=None,
                                 outs=None, stream=None):
    """scenes: list of (images, flow) of one size; returns the outputs per frame."""
    H, W = scenes[0][0][0].shape
    dev = scenes[0][0][0].device
    n = len(scenes)
    if ws is None:
        ws = learned_workspace(W, H, p, 2 * n, dev)
    if outs is None:
        outs = [alloc_scene_flow_outputs(W, H, dev) for _ in range(n)]
    arr = (LearnedFrame * n)()
    for k, ((imgs, flow), o) in enumerate(zip(scenes, outs)):
        arr[k] = LearnedFrame(*[_ptr(v) for v in (imgs[0], imgs[1], imgs[2], imgs[3], flow, o["s4"],
                                                  o["motion"], o["point"], o["valid"], o["D0"], o["D1"])])
    _check("sf_scene_flow_learned_frames",
           load().sf_scene_flow_learned_frames(arr, n, W, W, H, ctypes.byref(p), ctypes.byref(cam),
                                               _ptr(packed), float(threshold), _ptr(ws), ws.numel(),
                                               _stream(stream)))
    return outs
