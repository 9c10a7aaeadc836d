"""sf_confnet_init / sf_confnet_save / sf_confnet_load: the seeded
initialisation against its published definition (splitmix64, Box-Muller, He
scaling) recomputed here on the host, its statistics, and the file format
(round trip, and every malformed file rejected)."""
import math
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
LAYERS = [(8, 32), (32, 32), (32, 32), (32, 1)]


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04720_gb300 import _lib, build
    build.build()
    _lib.load()
    return _lib


def splitmix64(x):
    """Steele, Lea and Flood (2014), the splitmix64 output function."""
    x = (x + 0x9E3779B97F4A7C15) & M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


def expected_param(seed, i):
    o = 0
    for ci, co in LAYERS:
        nw = 9 * ci * co
        if i < o + nw:
            h1 = splitmix64(seed ^ splitmix64(2 * i))
            h2 = splitmix64(seed ^ splitmix64(2 * i + 1))
            u1 = ((h1 >> 40) + 1) / 2.0 ** 24
            u2 = (h2 >> 40) / 2.0 ** 24
            return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2) * math.sqrt(2.0 / (9 * ci))
        if i < o + nw + co:
            return 0.0
        o += nw + co
    raise IndexError(i)


def test_init_matches_published_definition(sf):
    seed = 1234567
    got = sf.confnet_init(seed).cpu().numpy().astype(np.float64)
    assert got.size == 21121
    idx = list(range(0, 21121, 97)) + [2303, 2304, 2335, 2336, 21119, 21120]
    for i in idx:
        want = expected_param(seed, i)
        # fp32 log, cos and sqrt: a few ulps of the largest factor
        assert abs(got[i] - want) <= 2e-6 * max(1.0, abs(want)) * 4, (i, got[i], want)


def test_init_statistics_and_determinism(sf):
    a = sf.confnet_init(7).cpu().numpy()
    b = sf.confnet_init(7).cpu().numpy()
    c = sf.confnet_init(8).cpu().numpy()
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    o = 0
    for ci, co in LAYERS:
        w = a[o:o + 9 * ci * co].astype(np.float64)
        o += 9 * ci * co
        assert np.all(a[o:o + co] == 0.0)            # biases
        o += co
        std = math.sqrt(2.0 / (9 * ci))
        n = w.size
        assert abs(w.mean()) < 5 * std / math.sqrt(n)
        assert abs(w.std() / std - 1.0) < 5 * math.sqrt(0.5 / n) + 0.01
        if n > 1000:   # normal shape: mass within one standard deviation
            assert abs(np.mean(np.abs(w) < std) - 0.6827) < 5 * math.sqrt(0.22 / n)
    assert o == a.size


def test_save_load_round_trip(sf, tmp_path):
    import torch
    p = sf.confnet_init(3)
    path = tmp_path / "w.sfcn"
    sf.confnet_save(p, str(path))
    raw = path.read_bytes()
    assert raw[:4] == b"SFCN"
    assert struct.unpack("<4I", raw[4:20]) == (1, 8, 32, 21121)
    assert len(raw) == 20 + 4 * 21121
    assert np.array_equal(np.frombuffer(raw[20:], dtype="<f4"), p.cpu().numpy())
    q = sf.confnet_load(str(path))
    assert torch.equal(p, q)


@pytest.mark.parametrize("damage", ["magic", "version", "count", "truncated", "trailing", "missing"])
def test_load_rejects_malformed_files(sf, tmp_path, damage):
    p = sf.confnet_init(4)
    path = tmp_path / "w.sfcn"
    sf.confnet_save(p, str(path))
    raw = bytearray(path.read_bytes())
    if damage == "magic":
        raw[0:4] = b"XXXX"
    elif damage == "version":
        raw[4:8] = struct.pack("<I", 2)
    elif damage == "count":
        raw[16:20] = struct.pack("<I", 21120)
    elif damage == "truncated":
        raw = raw[:-4]
    elif damage == "trailing":
        raw += b"\0"
    if damage == "missing":
        path = tmp_path / "absent.sfcn"
    else:
        path.write_bytes(bytes(raw))
    with pytest.raises(sf.SFError):
        sf.confnet_load(str(path))


def test_train_step_from_library_init(sf):
    import torch
    params = sf.confnet_init(11)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    g = torch.Generator().manual_seed(0)
    feats = (torch.rand((2, 24, 40, 8), generator=g) * 2).to(torch.bfloat16).view(torch.int16).cuda()
    labels = (torch.rand((2, 24, 40), generator=g) > 0.3).to(torch.uint8).cuda()
    before = params.clone()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ws = sf.confnet_train_workspace(2, 40, 24, "cuda")
    sf.confnet_train_step(params, m, v, feats, labels, sf.hparams(lr=1e-3, step=1), ws=ws, loss=loss)
    torch.cuda.synchronize()
    assert math.isfinite(float(loss.item())) and float(loss.item()) > 0
    assert not torch.equal(before, params)
