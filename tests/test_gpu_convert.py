"""The integer-pipe binary32 <-> binary64 conversions of the mixed-precision kernels
against IEEE conversions (numpy), element by element, bit for bit (GB300 only)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def doubles(seed=0, n=1 << 22):
    rng = np.random.default_rng(seed)
    # magnitudes over the whole binary32 range and beyond, both signs
    e = rng.uniform(-160.0, 140.0, size=n)
    d = np.sign(rng.uniform(-1, 1, size=n)) * np.exp2(e)
    # exact ties: a binary32 value plus half its ulp (normal and subnormal), and its neighbours
    f = rng.uniform(-1e3, 1e3, size=4096).astype(np.float32)
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    sub = (rng.integers(1, 1 << 23, size=4096) * 2.0 ** -149) * np.sign(rng.uniform(-1, 1, 4096))
    sulp = 2.0 ** -149
    ties = np.concatenate([f + 0.5 * ulp, f - 0.5 * ulp, sub + 0.5 * sulp, sub - 0.5 * sulp,
                           np.nextafter(f + 0.5 * ulp, np.inf), np.nextafter(sub + 0.5 * sulp, -np.inf)])
    fmax = float(np.finfo(np.float32).max)
    special = np.array([0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24),
                        2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150, 2.0 ** -150 * (1 + 2.0 ** -52),
                        2.0 ** -151, 5e-324, -5e-324, 2.0 ** 128, 1.0, -1.0, 1.0 + 2.0 ** -24,
                        1.0 + 3 * 2.0 ** -24])
    return np.concatenate([d, ties, special])


def floats(seed=1, n=1 << 22):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    edge = np.array([0, 1, 2, 0x7FFFFF, 0x800000, 0x7F7FFFFF, 0x7F800000, 0x80000000, 0x80000001, 0x807FFFFF,
                     0xFF800000, 0x3F800000], dtype=np.uint32)
    sub = np.arange(0, 1 << 16, dtype=np.uint32) * 127 + 1          # spread over the subnormals
    return np.concatenate([bits, edge, sub, sub | 0x80000000]).view(np.float32)


def test_conversions_match_ieee():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_05988_gb300 import build, pcg as C
    build.build()
    d = doubles()
    f = floats()
    n = min(d.size, f.size)
    d, f = d[:n], f[:n]
    dd = torch.from_numpy(d).cuda()
    ff = torch.from_numpy(f).cuda()
    fo = torch.empty(n, dtype=torch.float32, device="cuda")
    do = torch.empty(n, dtype=torch.float64, device="cuda")
    assert C.lib().pcg_convert_check(dd.data_ptr(), fo.data_ptr(), ff.data_ptr(), do.data_ptr(), n) == C.PCG_OK
    got32 = fo.cpu().numpy()
    got64 = do.cpu().numpy()
    with np.errstate(over="ignore"):
        want32 = d.astype(np.float32)
    with np.errstate(invalid="ignore"):                # signalling NaN inputs
        want64 = f.astype(np.float64)
    nan32 = np.isnan(want32)
    assert np.array_equal(np.isnan(got32), nan32)
    assert np.array_equal(got32[~nan32].view(np.uint32), want32[~nan32].view(np.uint32))
    nan64 = np.isnan(want64)
    assert np.array_equal(np.isnan(got64), nan64)
    assert np.array_equal(got64[~nan64].view(np.uint64), want64[~nan64].view(np.uint64))
    assert C.lib().pcg_convert_check(None, None, None, None, 0) == C.PCG_OK
    assert C.lib().pcg_convert_check(None, None, None, None, -1) == C.PCG_EINVAL
