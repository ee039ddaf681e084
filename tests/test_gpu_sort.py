"""The stable (key, value) radix sort behind tile binning and the depth order (Sec. 3.1-3.2),
called through the C ABI and compared bit for bit with NumPy's stable argsort: the 8-bit
passes (up to 16 and above 20 key bits) and the two wide passes (17 to 20 bits), on sizes
that end inside a tile, span several sort blocks and leave ragged tails."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2406_11836_gb300 import build, rgs
    build.build()
    return rgs


def _check(R, n, end_bit, seed, dist="uniform"):
    g = np.random.default_rng(seed)
    if dist == "uniform":
        keys = g.integers(0, 2**end_bit, size=n, dtype=np.uint64).astype(np.uint32)
    elif dist == "few":   # long runs of equal keys: stability decides the whole order
        keys = g.integers(0, 5, size=n, dtype=np.uint64).astype(np.uint32) << np.uint32(max(end_bit - 3, 0))
    else:                 # already sorted runs, as the later passes of a tile sort see them
        keys = np.sort(g.integers(0, 2**end_bit, size=n, dtype=np.uint64)).astype(np.uint32)
        keys = np.roll(keys, n // 3)
    vals = np.arange(n, dtype=np.uint32)
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    vd = torch.from_numpy(vals.view(np.int32)).cuda()
    ks, vs = R.sort_pairs(kd, vd, end_bit)
    got_k = ks.cpu().numpy().view(np.uint32)
    got_v = vs.cpu().numpy().view(np.uint32)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(got_v, vals[order]), f"n={n} end_bit={end_bit}: values out of stable order"
    assert np.array_equal(got_k, keys[order]), f"n={n} end_bit={end_bit}: keys"


@pytest.mark.parametrize("end_bit", [8, 16, 17, 19, 20, 21, 31])
@pytest.mark.parametrize("n", [1, 2, 8191, 8193, 65537, 300_001])
def test_sort_matches_stable_argsort(R, n, end_bit):
    _check(R, n, end_bit, seed=n * 31 + end_bit)


@pytest.mark.parametrize("end_bit", [17, 19, 20])
@pytest.mark.parametrize("dist", ["few", "runs"])
def test_wide_passes_keep_equal_keys_in_input_order(R, end_bit, dist):
    _check(R, 1_000_003, end_bit, seed=end_bit, dist=dist)


def test_sort_large_19_bit_keys(R):
    """Tile-instance keys of a 4K view with 16 subsets: 19 bits, tens of millions of pairs."""
    _check(R, 24_000_017, 19, seed=5)


def test_sort_empty_and_argument_checks(R):
    import ctypes
    from paper_2406_11836_gb300.rgs import RGSError
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    ks, vs = R.sort_pairs(e, e, 19)
    assert ks.numel() == 0 and vs.numel() == 0
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(RGSError):
        R.sort_pairs(x, x.clone(), 0)
    with pytest.raises(RGSError):
        R.sort_pairs(x, x.clone(), 33)
    L = R.lib()
    alt = ctypes.c_int(0)
    assert L.rgs_sort_pairs(None, None, None, None, 4, 8, None, 0, None, ctypes.byref(alt)) != 0
