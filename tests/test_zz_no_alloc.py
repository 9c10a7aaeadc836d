"""sf_sgm_aggregate_noalloc: aggregation with the library's built-in scratch
array instead of a caller workspace.  It must give the same S, bit for bit,
as sf_sgm_aggregate (fused workspace path and staged kernels), on two calls
in a row, and reject requests beyond its fixed scratch size.  The file name
sorts last so that the calls also run after every other test in a session;
it passes alone too."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import to_dev, to_np


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


CASES = [(64, 48, 16, 0xFF), (320, 240, 64, 0xFF), (640, 480, 16, 0xFF), (1242, 40, 128, 0xFF),
         (97, 41, 32, 0x5A), (130, 37, 48, 0xFF)]


@pytest.mark.gpu
@pytest.mark.parametrize("W,H,D,mask", CASES)
def test_noalloc_equals_workspace_path(sf, W, H, D, mask):
    import torch
    p = sf.params(D=D, path_mask=mask)
    rng = np.random.default_rng(W * 7 + H * 3 + D)
    costs = [to_dev(rng.integers(0, 63, size=(H, W, D), dtype=np.uint8)) for _ in range(2)]
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for c in costs:                                   # two calls in a row, different inputs
        out = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        sf.sf_sgm_aggregate_noalloc(c, p, out, err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        fused = to_np(sf.sf_sgm_aggregate(c, p, ws="auto"), np.uint16)
        staged = to_np(sf.sf_sgm_aggregate(c, p, ws=None), np.uint16)
        got = to_np(out, np.uint16)
        assert np.array_equal(got, fused)
        assert np.array_equal(got, staged)


@pytest.mark.gpu
def test_noalloc_back_to_back_without_sync(sf):
    import torch
    W, H, D = 200, 60, 64
    p = sf.params(D=D)
    rng = np.random.default_rng(5)
    a = to_dev(rng.integers(0, 63, size=(H, W, D), dtype=np.uint8))
    b = to_dev(rng.integers(0, 63, size=(H, W, D), dtype=np.uint8))
    oa = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
    ob = torch.empty_like(oa)
    sf.sf_sgm_aggregate_noalloc(a, p, oa)          # same stream: ordered, no race
    sf.sf_sgm_aggregate_noalloc(b, p, ob)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(oa, np.uint16), to_np(sf.sf_sgm_aggregate(a, p, ws=None), np.uint16))
    assert np.array_equal(to_np(ob, np.uint16), to_np(sf.sf_sgm_aggregate(b, p, ws=None), np.uint16))


@pytest.mark.gpu
def test_noalloc_rejects_oversize_and_unsupported_depth(sf):
    import torch
    fake = ctypes.c_void_p(256)        # never dereferenced: rejected on the host
    lib = sf.load()
    for (W, H, D) in [(1242, 375, 128), (320, 240, 128), (2048, 1024, 256)]:
        p = sf.params(D=D)
        assert lib.sf_sgm_aggregate_noalloc(fake, W, H, ctypes.byref(p), fake, None, None) == 2
    p = sf.params(D=24)                 # not a multiple of 16
    assert lib.sf_sgm_aggregate_noalloc(fake, 64, 48, ctypes.byref(p), fake, None, None) == 2
    p = sf.params(D=16)
    assert lib.sf_sgm_aggregate_noalloc(None, 64, 48, ctypes.byref(p), fake, None, None) == 1
    torch.cuda.synchronize()
