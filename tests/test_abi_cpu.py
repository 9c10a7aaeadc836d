"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/sf.h declares, and rejects bad arguments on the host
before touching the GPU (so these run without one)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1801_04720_gb300 import _lib
    assert set(_lib.EXPORTED) <= set(declared_functions())
    sf_h = set(n for n in declared_functions() if not n.startswith(("sf_batch", "sf_confnet")))
    assert sf_h <= set(_lib.EXPORTED) | set(n for n in declared_functions() if n not in sf_h)


def test_defaults_and_status_strings(lib):
    from paper_1801_04720_gb300 import _lib
    p = _lib.SgmParams()
    lib.sf_default_params(ctypes.byref(p))
    assert (p.census_w, p.census_h, p.P1, p.P2, p.path_mask, p.D, p.subpixel, p.lr_tol) == \
        (9, 7, 7, 86, 0xFF, 128, 1, 1)
    assert lib.sf_status_string(0) == b"SF_OK"
    assert lib.sf_status_string(4) == b"SF_ERR_TIMEOUT"


def test_workspace_size_is_host_only(lib):
    from paper_1801_04720_gb300 import _lib
    p = _lib.params()
    n = lib.sf_workspace_size(1242, 375, ctypes.byref(p))
    N, D = 1242 * 375, 128
    assert n >= N * D * 3           # cost + aggregated cost at least
    assert lib.sf_workspace_size(0, 375, ctypes.byref(p)) == 0


def _p(**kw):
    from paper_1801_04720_gb300 import _lib
    return _lib.params(**kw)


FAKE = ctypes.c_void_p(0x100000)   # never dereferenced: validation fails first


@pytest.mark.parametrize("kw,expected", [
    (dict(D=0), 1), (dict(D=257), 1), (dict(census_w=8), 1), (dict(census_h=4), 1),
    (dict(census_w=11, census_h=7), 1), (dict(P1=90, P2=86), 1), (dict(P2=200), 2),
    (dict(path_mask=0x1FF), 1), (dict(lr_tol=-1), 1)])
def test_bad_params_rejected_before_launch(lib, kw, expected):
    p = _p(**kw)
    st = lib.sf_cost_volume(FAKE, FAKE, 64, 48, 64, ctypes.byref(p), 0, FAKE, None)
    assert st == expected


def test_null_pointers_and_sizes_rejected(lib):
    p = _p(D=16)
    assert lib.sf_census(None, 64, 48, 64, 9, 7, FAKE, None) == 1
    assert lib.sf_census(FAKE, 64, 48, 63, 9, 7, FAKE, None) == 1      # pitch < W
    assert lib.sf_census(FAKE, 8, 48, 8, 9, 7, FAKE, None) == 1        # W < census width
    assert lib.sf_census(FAKE, -1, 48, 64, 9, 7, FAKE, None) == 1
    assert lib.sf_sgm_aggregate(None, 64, 48, ctypes.byref(p), FAKE, None, 0, None) == 1
    assert lib.sf_disparity_select(FAKE, 64, 48, 0, 1, FAKE, None, None) == 1
    assert lib.sf_lr_check(FAKE, FAKE, None, 64, 48, 1, FAKE, FAKE, None) == 1
    assert lib.sf_lr_check(FAKE, FAKE, FAKE, 64, 48, -2, FAKE, FAKE, None) == 1
    from paper_1801_04720_gb300 import _lib
    cam = _lib.camera(100.0, 0.5, 31.5, 23.5)
    assert lib.sf_combine_sceneflow(FAKE, FAKE, FAKE, 64, 48, None, FAKE, None, None, FAKE, None) == 1
    bad_cam = _lib.camera(-1.0, 0.5, 31.5, 23.5)
    assert lib.sf_combine_sceneflow(FAKE, FAKE, FAKE, 64, 48, ctypes.byref(bad_cam), FAKE, None,
                                    None, FAKE, None) == 1
    # misaligned s4 output (needs 16-byte alignment for float4 stores)
    assert lib.sf_combine_sceneflow(FAKE, FAKE, FAKE, 64, 48, ctypes.byref(cam),
                                    ctypes.c_void_p(0x100004), None, None, FAKE, None) == 1
    # workspace too small
    assert lib.sf_sgm_full(FAKE, FAKE, 64, 48, 64, ctypes.byref(p), None, None, None, FAKE, FAKE,
                           16, None) == 1
