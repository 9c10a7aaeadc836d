"""Parity at the full automotive size (1242x375, D=128) and at the large-stream
size (2048x1024, D=256) through the same entry points and launch
configuration the bench times: every integer disparity and mask bit-exact
against the oracle, subpixel disparity within 1e-4 px, and the combination
within 1e-5 relative on the same float32 maps."""
import numpy as np
import pytest

from gpu_helpers import oracle_disparities_parallel, to_dev, to_np
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


@pytest.fixture(scope="module")
def scene_and_oracle():
    q = synth.automotive(seed=0)
    r0, r1 = oracle_disparities_parallel([(q.left_t, q.right_t), (q.left_t1, q.right_t1)], D=128)
    return q, r0, r1


def test_full_size_scene_flow(sf, oracle_mod, scene_and_oracle):
    from test_gpu_parity import _scene_flow_parity
    q, r0, r1 = scene_and_oracle
    got = _scene_flow_parity(sf, oracle_mod, q, dict(D=128), oracle_results=(r0, r1))
    assert got["valid"].mean() > 0.3


def test_full_size_integer_disparities(sf, scene_and_oracle):
    q, r0, r1 = scene_and_oracle
    p = sf.params(D=128)
    for (l, r), ref in (((q.left_t, q.right_t), r0), ((q.left_t1, q.right_t1), r1)):
        out = sf.sf_sgm_full(to_dev(l), to_dev(r), p)
        assert np.array_equal(to_np(out["dL"]), ref["dL"])
        assert np.array_equal(to_np(out["dR"]), ref["dR"])
        assert np.array_equal(to_np(out["valid"]), ref["valid"])


@pytest.fixture(scope="module")
def stream_and_oracle():
    # one frame of the large-stream recipe: 2048x1024, D = 256, 40 moving segments
    q = synth.stream(1, seed=0)[0]
    r0, r1 = oracle_disparities_parallel([(q.left_t, q.right_t), (q.left_t1, q.right_t1)], D=256)
    return q, r0, r1


def test_stream_size_scene_flow(sf, oracle_mod, stream_and_oracle):
    from test_gpu_parity import _scene_flow_parity
    q, r0, r1 = stream_and_oracle
    assert q.shape == (1024, 2048) and q.D == 256
    got = _scene_flow_parity(sf, oracle_mod, q, dict(D=256), oracle_results=(r0, r1))
    assert got["valid"].mean() > 0.3


def test_stream_size_integer_disparities(sf, stream_and_oracle):
    q, r0, r1 = stream_and_oracle
    p = sf.params(D=256)
    for (l, r), ref in (((q.left_t, q.right_t), r0), ((q.left_t1, q.right_t1), r1)):
        out = sf.sf_sgm_full(to_dev(l), to_dev(r), p)
        assert np.array_equal(to_np(out["dL"]), ref["dL"])
        assert np.array_equal(to_np(out["dR"]), ref["dR"])
        assert np.array_equal(to_np(out["valid"]), ref["valid"])
    # the learned path's left pass is the same integer SGM
    lo = sf.sf_sgm_learned(to_dev(q.left_t), to_dev(q.right_t), p, packed=None)
    assert np.array_equal(to_np(lo["dint"]), r0["dL"])
