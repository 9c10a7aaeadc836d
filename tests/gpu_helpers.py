"""Shared helpers for the GPU parity tests (inputs, transfers, tolerances)."""
import multiprocessing as mp

import numpy as np

# Tolerances stated by the method's accuracy targets: integer outputs exact,
# subpixel disparity within 1e-4 px, FP32 scene flow within 1e-5 relative.
SUBPIXEL_ATOL = 1e-4
SCENEFLOW_RTOL = 1e-5


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def to_np(t, dtype=None):
    a = t.detach().cpu().numpy()
    if dtype is not None:
        a = a.view(dtype) if a.dtype.itemsize == np.dtype(dtype).itemsize else a.astype(dtype)
    return a


def assert_nan_equal_close(gpu, ref, atol, what):
    gn, rn = np.isnan(gpu), np.isnan(ref)
    assert np.array_equal(gn, rn), f"{what}: NaN pattern differs at {np.argwhere(gn != rn)[:5]}"
    m = ~rn
    if m.any():
        err = np.abs(gpu[m].astype(np.float64) - ref[m])
        assert err.max() <= atol, f"{what}: max err {err.max()} > {atol}"


def assert_sceneflow_close(gpu_out, ref_s4, ref_motion, ref_point, ref_valid):
    """valid exact; floats within 1e-5 relative, measured against max(|ref|,
    ||P0||_inf) for the 3D quantities (motion is a difference of nearly equal
    vectors)."""
    gv = gpu_out["valid"]
    assert np.array_equal(gv, ref_valid), f"valid differs at {np.argwhere(gv != ref_valid)[:5]}"
    m = ref_valid == 1
    assert np.isnan(gpu_out["s4"][~m]).all()
    s4g = gpu_out["s4"][m].astype(np.float64)
    s4r = ref_s4[m]
    assert (np.abs(s4g - s4r) <= SCENEFLOW_RTOL * np.abs(s4r) + 1e-30).all(), \
        f"s4 max rel err {np.max(np.abs(s4g - s4r) / np.maximum(np.abs(s4r), 1e-30))}"
    if ref_point is not None and gpu_out.get("point") is not None:
        scale = np.abs(ref_point[m]).max(axis=1, keepdims=True)
        pg = gpu_out["point"][m].astype(np.float64)
        assert (np.abs(pg - ref_point[m]) <= SCENEFLOW_RTOL * np.maximum(np.abs(ref_point[m]), scale)).all()
        if ref_motion is not None and gpu_out.get("motion") is not None:
            mg = gpu_out["motion"][m].astype(np.float64)
            err = np.abs(mg - ref_motion[m])
            bound = SCENEFLOW_RTOL * np.maximum(np.abs(ref_motion[m]), scale)
            assert (err <= bound).all(), f"motion max err/bound {np.max(err / bound)}"


def _oracle_disparity(args):
    from oracle import oracle
    left, right, kw = args
    return oracle.disparity(left, right, **kw)


def oracle_disparities_parallel(pairs, **kw):
    """Oracle SGM for several stereo pairs in spawned worker processes (safe to
    start after the GPU is in use)."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(pairs), 4)) as pool:
        return pool.map(_oracle_disparity, [(l, r, kw) for l, r in pairs])
