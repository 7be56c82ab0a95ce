"""The reciprocal every kernel uses in place of a division (the hardware approximation refined by
one third-order Newton-Raphson step, y (1 + e + e^2) with e = 1 - x y) against the correctly
rounded IEEE quotient 1 / x computed on the host: within one unit in the last place for normal,
finite, non-zero x, over the whole exponent range the kernels can meet and densely around the
magnitudes they do meet (cell widths, their sums and products, depths above the dry threshold,
indicator sums), and NaN for the arguments it does not take (zero, infinities, subnormals).
Called through the C ABI (swale_check_recip)."""
import numpy as np
import pytest

from paper_2208_06588_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_06588_gb300 import build
    build.build()
    B.lib()


def kernels_recip(x):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.empty_like(xd)
    s = torch.cuda.current_stream()
    B.swale_check_recip(s.cuda_stream, xd.numel(), xd, yd)
    s.synchronize()
    return yd.cpu().numpy()


def ulp_distance(a, b):
    """Distance in units in the last place between doubles of the same sign."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def arguments(seed=20220812):
    rng = np.random.default_rng(seed)
    parts = [
        # log-uniform over the normal range whose reciprocals stay normal
        np.exp2(rng.uniform(-1000.0, 1000.0, 1 << 21)),
        # the magnitudes of the kernels' arguments: widths down to 1e-8, depths from 1e-6
        np.exp(rng.uniform(np.log(1e-12), np.log(1e4), 1 << 21)),
        # every mantissa pattern near the ends of a binade
        1.0 + np.arange(1 << 16) * 2.0 ** -52,
        2.0 - np.arange(1, 1 << 16) * 2.0 ** -52,
        np.exp2(np.arange(-1000, 1001).astype(np.float64)),
        # near-ties of the quotient: x = 1 + k / 2^26 (1 / x close to a rounding midpoint more often)
        1.0 + rng.integers(1, 1 << 26, 1 << 16) * 2.0 ** -26,
    ]
    x = np.concatenate(parts)
    sign = np.where(rng.random(x.size) < 0.5, -1.0, 1.0)
    return x * sign


def test_reciprocal_within_one_ulp_of_the_correctly_rounded_quotient():
    x = arguments()
    y = kernels_recip(x)
    ref = 1.0 / x  # IEEE division on the host: correctly rounded
    assert np.all(np.isfinite(y))
    assert np.all(np.sign(y) == np.sign(ref))
    d = ulp_distance(np.abs(y), np.abs(ref))
    assert d.max() <= 1, (d.max(), x[np.argmax(d)])
    # the refinement leaves a relative error far below half a unit before the final rounding,
    # so all but a small share of the results are the correctly rounded quotient itself
    assert (d == 0).mean() > 0.95, (d == 0).mean()


def test_reciprocal_of_arguments_it_does_not_take_is_nan():
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -1e-310, 2.0 ** -1030])
    y = kernels_recip(x)
    assert np.all(np.isnan(y)), y


def test_reciprocal_in_place_and_empty():
    import torch
    x = torch.linspace(0.5, 4.0, 1001, dtype=torch.float64, device="cuda")
    ref = 1.0 / x.cpu().numpy()
    s = torch.cuda.current_stream()
    B.swale_check_recip(s.cuda_stream, x.numel(), x, x)
    B.swale_check_recip(s.cuda_stream, 0, x, x)
    s.synchronize()
    assert ulp_distance(x.cpu().numpy(), ref).max() <= 1
    with pytest.raises(B.SwaleError):
        B.swale_check_recip(s.cuda_stream, 4, np.ones(4), np.ones(4))  # host arrays are refused
