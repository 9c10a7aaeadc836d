"""Failure detection without a GPU fault: the band sweeps' inter-CTA waits
are bounded.  A test hook makes the down sweep's queue skip the first band,
so every later task waits for flags that nothing sets; the waits give up,
the workspace error word reports SF_ERR_TIMEOUT, the kernels return, and the
context stays usable for the next (correct) call."""
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
    yield _lib
    _lib.sf_debug_set(_lib.SF_DEBUG_SKIP_TASKS, 0)
    _lib.sf_debug_set(_lib.SF_DEBUG_SPIN_LIMIT, 0)


def test_bounded_wait_reports_timeout_and_context_survives(sf, oracle_mod):
    import torch
    q = synth.fronto_planes(W=200, H=60, D=64, disparities=(2, 20, 55), seed=9)
    H, W = q.shape
    p = sf.params(D=64)
    left, right = to_dev(q.left_t), to_dev(q.right_t)
    ws = sf.workspace(W, H, p, "cuda")
    J = (W + 31) // 32
    try:
        sf.sf_debug_set(sf.SF_DEBUG_SPIN_LIMIT, 1 << 12)
        sf.sf_debug_set(sf.SF_DEBUG_SKIP_TASKS, 2 * J)      # band 0 of both passes
        sf.sf_sgm_full(left, right, p, ws=ws)
        torch.cuda.synchronize()
        with pytest.raises(sf.SFError) as e:
            sf.sf_check_workspace(ws, W, H, p, 1)
        assert e.value.status == 4                            # SF_ERR_TIMEOUT
    finally:
        sf.sf_debug_set(sf.SF_DEBUG_SKIP_TASKS, 0)
        sf.sf_debug_set(sf.SF_DEBUG_SPIN_LIMIT, 0)
    # the context is intact: the next call is correct and reports no error
    out = sf.sf_sgm_full(left, right, p, ws=ws)
    torch.cuda.synchronize()
    sf.sf_check_workspace(ws, W, H, p, 1)
    r = oracle_mod.disparity(q.left_t, q.right_t, D=64)
    assert np.array_equal(to_np(out["dL"]), r["dL"])
    assert np.array_equal(to_np(out["valid"]), r["valid"])


def test_debug_hook_rejects_bad_values(sf):
    with pytest.raises(sf.SFError):
        sf.sf_debug_set(sf.SF_DEBUG_SPIN_LIMIT, -1)
    with pytest.raises(sf.SFError):
        sf.sf_debug_set(99, 0)
