"""The FP64 helpers of the native flux kernels against CUDA's own
arithmetic on the same GPU: the reciprocals 1/rho and 1/(2 rho), by one
third-order Newton-Raphson step from an FP32 seed, within one unit in the
last place of the IEEE quotients 1 / x and 0.5 / x over the whole exponent
range they cover (exponent field 1..2040, both signs), and bit for bit
where they defer to the IEEE quotient (zero, subnormal, above 2^1017,
infinite, NaN); the halving by an exponent decrement bit for bit equal to
0.5 * x for every class of double."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ulp_distance(a, b):
    """|a - b| in units in the last place, for finite doubles of one sign."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def rcp(ml, x, half):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ml.mp_recip_test(xd, yd, mode=1 if half else 0)
    ref = (0.5 if half else 1.0) / xd                    # CUDA's IEEE division
    torch.cuda.synchronize()
    return yd.cpu().numpy(), ref.cpu().numpy()


@pytest.mark.parametrize("half", [True, False])
def test_rcp_within_one_ulp_over_the_exponent_range(half):
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
    y, ref = rcp(ml, x, half)
    assert np.all(np.isfinite(y)) and np.all(np.sign(y) == np.sign(ref))
    d = ulp_distance(y, ref)
    assert d.max() <= 1, (d.max(), x[d.argmax()])
    # most are the correctly rounded quotient
    assert np.mean(d == 0) > 0.9


@pytest.mark.parametrize("half", [True, False])
def test_rcp_defers_to_ieee_outside_its_range(half):
    import paper_1802_03749_gb300 as ml
    sub = np.array([1, 3, (1 << 52) - 1, 1 << 40], dtype=np.int64).view(np.float64)   # subnormals
    big = (np.array([2041, 2045, 2046], dtype=np.int64) << 52).view(np.float64)         # >= 2^1018
    x = np.concatenate([[0.0, -0.0, np.inf, -np.inf, np.nan], sub, -sub, big, -big,
                        [np.finfo(np.float64).max, np.finfo(np.float64).tiny / 2]])
    y, ref = rcp(ml, x, half)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan].view(np.int64), ref[~nan].view(np.int64))


def test_rcp_arguments():
    import paper_1802_03749_gb300 as ml
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ml.MeshLoopError):
        ml.mp_recip_test(x, torch.ones(4, dtype=torch.float64))            # host tensor
    with pytest.raises(ml.MeshLoopError):
        ml.mp_recip_test(x.float(), x.float())                           # not float64
    h = torch.ones(4, dtype=torch.float64).pin_memory()
    assert ml.lib().mp_recip_test(ml._ptr(h), ml._ptr(x), 4, 0, None) == -1    # host pointer: MP_EINVAL
    assert ml.lib().mp_recip_test(ml._ptr(x), ml._ptr(x), 4, 3, None) == -1    # mode not 0..2
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    ml.mp_recip_test(e, e)                                                 # n = 0: nothing to do


def test_half_of_is_exact():
    import paper_1802_03749_gb300 as ml
    rng = np.random.default_rng(19)
    ex = np.repeat(np.arange(0, 2048, dtype=np.int64), 16)           # every exponent field
    bits = (ex << 52) | rng.integers(0, 1 << 52, ex.size, dtype=np.int64)
    x = bits.view(np.float64).copy()
    x[1::2] = -x[1::2]
    x = np.concatenate([x, [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, np.finfo(np.float64).tiny]])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ml.mp_recip_test(xd, yd, mode=2)
    ref = (0.5 * xd).cpu().numpy()
    y = yd.cpu().numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(y), nan)
    assert np.array_equal(y[~nan].view(np.int64), ref[~nan].view(np.int64))
