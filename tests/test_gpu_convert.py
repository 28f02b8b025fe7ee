"""The mixed-precision kernels' number-format conversions, built from the
IEEE-754 bit patterns with integer instructions, against the hardware
conversions (round to nearest, ties to even) and the double-single
invariants, bit for bit, through sisdc_convert."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import sisdc as S   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


SPECIAL = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 1e-40, -1e-45, 1.1754943508222875e-38,
           1.1754942106924411e-38, 3.4028234663852886e+38, 3.4028235677973366e+38, 3.4028236e+38, 1e300,
           -1e300, 2.0 ** -74, 2.0 ** -75, -(2.0 ** -74) * 1.5, 2.0 ** 127, 2.0 ** 128,
           np.nextafter(2.0 ** 128, 0.0), 1.0, -1.0, 0.1, 1.0 / 3.0]


def sample_doubles(seed, n=100000):
    rng = np.random.default_rng(seed)
    x = rng.choice([-1.0, 1.0], n) * np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-160, 160, n))
    # values at, just above and just below the halfway points between floats
    f = rng.uniform(-1e3, 1e3, n // 4).astype(np.float32)
    h = np.spacing(np.abs(f)).astype(np.float64) / 2
    f = f.astype(np.float64)
    ties = np.concatenate([f + h, f - h, f + h * (1 + 2.0 ** -30), f + h * (1 - 2.0 ** -30)])
    return np.concatenate([x, ties, np.array(SPECIAL)])


def same_bits(a, b):
    """Equal bit patterns, with any NaN matching any NaN."""
    an, bn = torch.isnan(a), torch.isnan(b)
    assert torch.equal(an, bn)
    it = torch.int32 if a.dtype == torch.float32 else torch.int64
    ok = ~an
    return torch.equal(a[ok].view(it), b[ok].view(it))


def trunc_to_24_bits(x):
    """x (float64 array) with all but the leading 24 significand bits cleared."""
    b = x.view(np.int64) & ~np.int64((1 << 29) - 1)
    return b.view(np.float64)


def test_double_to_float_rounds_like_hardware(dev):
    x = torch.from_numpy(sample_doubles(1)).to(dev)
    assert same_bits(S.sisdc_convert(0, x), x.float())


def test_float_to_double_exact(dev):
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    with np.errstate(over="ignore"):          # the specials include values beyond the float range
        f = np.concatenate([bits.view(np.float32), np.array(SPECIAL, dtype=np.float32)])
    x = torch.from_numpy(f).to(dev)
    assert same_bits(S.sisdc_convert(1, x), x.double())


def test_double_single_split(dev):
    xs = sample_doubles(3)
    xs = xs[np.isfinite(xs)]
    x = torch.from_numpy(xs).to(dev)
    hl = S.sisdc_convert(2, x).cpu().numpy().astype(np.float64)
    hi, lo = hl[:, 0], hl[:, 1]
    a = np.abs(xs)
    fast = (a >= 2.0 ** -74) & (a < 2.0 ** 128)
    # fast path: hi = x truncated to 24 bits, lo = the remainder truncated to 24 bits
    hi_ref = trunc_to_24_bits(xs[fast])
    lo_ref = trunc_to_24_bits(xs[fast] - hi_ref)
    assert np.array_equal(hi[fast], hi_ref) and np.array_equal(lo[fast], lo_ref)
    err = np.abs((hi[fast] + lo[fast]) - xs[fast])
    assert np.all(err <= 2.0 ** -47 * a[fast])
    nz = fast & (hi != 0)
    with np.errstate(over="ignore"):          # ulp of the largest float is beyond the float range
        ulp_hi = np.spacing(np.abs(hi[nz]).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(lo[nz]) < ulp_hi)
    # other inputs: the rounded float and the rounded remainder
    slow = ~fast
    hs = x[torch.from_numpy(slow).to(dev)].float()
    ls = (x[torch.from_numpy(slow).to(dev)] - hs.double()).float()
    assert np.array_equal(hi[slow], hs.double().cpu().numpy())
    assert np.array_equal(lo[slow], ls.double().cpu().numpy())


def test_double_single_to_double(dev):
    rng = np.random.default_rng(4)
    n = 200000
    hi = (rng.choice([-1.0, 1.0], n) * np.ldexp(rng.uniform(1, 2, n), rng.integers(-100, 100, n))).astype(np.float32)
    lo = (hi.astype(np.float64) * rng.uniform(-2.0 ** -24, 2.0 ** -24, n)).astype(np.float32)
    pairs = np.stack([hi, lo], axis=1)
    pairs = np.concatenate([pairs, np.array([[0.0, 0.0], [-0.0, 0.0], [1.0, -0.0], [np.inf, 0.0],
                                             [1e-40, 1e-45], [3.0e38, 1.0e31]], dtype=np.float32)])
    p = torch.from_numpy(pairs).to(dev)
    ref = p[:, 0].double() + p[:, 1].double()
    assert same_bits(S.sisdc_convert(3, p), ref)


def test_convert_rejects_bad_arguments(dev):
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    assert S.load().sisdc_convert(7, x.data_ptr(), 4, x.data_ptr(), None) == S.SISDC_E_ARG
    assert S.load().sisdc_convert(0, None, 4, x.data_ptr(), None) == S.SISDC_E_ARG
    assert S.load().sisdc_convert(0, x.data_ptr(), -1, x.data_ptr(), None) == S.SISDC_E_ARG
    assert S.load().sisdc_convert(0, None, 0, None, None) == S.SISDC_OK
