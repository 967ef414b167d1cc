"""The reciprocal of the native FP64 flux kernels, 1/(2 rho) by one
third-order Newton-Raphson step from an FP32 seed, against CUDA's IEEE
double quotient 0.5 / x on the same GPU: within one unit in the last place
over the whole exponent range it covers (exponent field 1..2040, both
signs), and bit for bit where it defers to the IEEE quotient (zero,
subnormal, above 2^1017, infinite, NaN)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ulp_distance(a, b):
    """|a - b| in units in the last place, for finite doubles of one sign."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def rcp(ml, x):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ml.mp_rcp_half_test(xd, yd)
    ref = 0.5 / xd                                       # CUDA's IEEE division
    torch.cuda.synchronize()
    return yd.cpu().numpy(), ref.cpu().numpy()


def test_rcp_half_within_one_ulp_over_the_exponent_range():
    import paper_1802_03749_gb300 as ml
    rng = np.random.default_rng(17)
    # every exponent field 1..2040, several significands each, both signs
    ex = np.repeat(np.arange(1, 2041, dtype=np.int64), 64)
    mant = rng.integers(0, 1 << 52, ex.size, dtype=np.int64)
    mant[::64] = 0                                        # powers of two
    mant[1::64] = (1 << 52) - 1                           # largest significands
    mant[2::64] = 1                                       # just above a power of two
    mant[3::64] = (1 << 52) - (1 << 32)                   # seed truncation edge
    bits = (ex << 52) | mant
    x = bits.view(np.float64).copy()
    x[1::2] = -x[1::2]
    y, ref = rcp(ml, x)
    assert np.all(np.isfinite(y)) and np.all(np.sign(y) == np.sign(ref))
    d = ulp_distance(y, ref)
    assert d.max() <= 1, (d.max(), x[d.argmax()])
    # most are the correctly rounded quotient
    assert np.mean(d == 0) > 0.9


def test_rcp_half_defers_to_ieee_outside_its_range():
    import paper_1802_03749_gb300 as ml
    sub = np.array([1, 3, (1 << 52) - 1, 1 << 40], dtype=np.int64).view(np.float64)   # subnormals
    big = (np.array([2041, 2045, 2046], dtype=np.int64) << 52).view(np.float64)         # >= 2^1018
    x = np.concatenate([[0.0, -0.0, np.inf, -np.inf, np.nan], sub, -sub, big, -big,
                        [np.finfo(np.float64).max, np.finfo(np.float64).tiny / 2]])
    y, ref = rcp(ml, x)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan].view(np.int64), ref[~nan].view(np.int64))


def test_rcp_half_arguments():
    import paper_1802_03749_gb300 as ml
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ml.MeshLoopError):
        ml.mp_rcp_half_test(x, torch.ones(4, dtype=torch.float64))          # host tensor
    with pytest.raises(ml.MeshLoopError):
        ml.mp_rcp_half_test(x.float(), x.float())                         # not float64
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    ml.mp_rcp_half_test(e, e)                                              # n = 0: nothing to do
