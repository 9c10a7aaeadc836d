"""The frame pipeline (host buffers, copies overlapped with compute): every
frame's outputs equal sf_scene_flow's on the same inputs bit for bit, with
several frames in flight through fewer staging slots, and the argument
errors."""
import numpy as np
import pytest

from gpu_helpers import to_dev, to_np
from paper_1801_04720_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


def _host_out(H, W, motion=True):
    import torch
    return {"s4": torch.empty((H, W, 4)).pin_memory(),
            "motion": torch.empty((H, W, 3)).pin_memory() if motion else None,
            "point": torch.empty((H, W, 3)).pin_memory() if motion else None,
            "valid": torch.empty((H, W), dtype=torch.uint8).pin_memory()}


def _same(a, b):
    return np.array_equal(np.nan_to_num(a, nan=-7.0), np.nan_to_num(b, nan=-7.0))


@pytest.mark.parametrize("depth,n_frames", [(2, 5), (3, 7)])
def test_pipeline_matches_device_path(sf, depth, n_frames):
    import torch
    W, H, D = 160, 96, 32
    quads = [synth.fronto_planes(W=W, H=H, D=D, disparities=(3, 9 + k, 20 + k), seed=40 + k)
             for k in range(n_frames)]
    cam = quads[0].camera
    p = sf.params(D=D)
    c = sf.camera(cam.f, cam.B, cam.cx, cam.cy)
    outs = [_host_out(H, W, motion=(k % 2 == 0)) for k in range(n_frames)]
    with sf.Pipeline(W, H, p, c, depth=depth) as pl:
        tickets = []
        for k, q in enumerate(quads):
            imgs = [torch.from_numpy(im).pin_memory() for im in q.images()]
            tickets.append(pl.submit(imgs, torch.from_numpy(q.flow).pin_memory(), outs[k]))
        assert tickets == list(range(n_frames))
        pl.wait(tickets[-1])
        pl.wait(tickets[0])          # an older frame: already complete
    for k, q in enumerate(quads):
        ref = sf.sf_scene_flow([to_dev(im) for im in q.images()], to_dev(q.flow), p, c)
        for key in ("s4", "valid") + (("motion", "point") if k % 2 == 0 else ()):
            assert _same(outs[k][key].numpy(), to_np(ref[key])), (k, key)


def test_pipeline_argument_errors(sf):
    import torch
    p = sf.params(D=16)
    c = sf.camera(100.0, 0.5, 31.5, 23.5)
    with pytest.raises(sf.SFError):
        sf.Pipeline(64, 48, p, c, depth=1)
    with pytest.raises(sf.SFError):
        sf.Pipeline(64, 48, p, sf.camera(0.0, 0.5, 31.5, 23.5), depth=2)
    with sf.Pipeline(64, 48, p, c, depth=2) as pl:
        with pytest.raises(sf.SFError):
            pl.wait(0)               # nothing submitted yet
        with pytest.raises(ValueError):
            pl.submit([torch.zeros((48, 64), dtype=torch.uint8, device="cuda")] * 4,
                      torch.zeros((48, 64, 2)), _host_out(48, 64))
