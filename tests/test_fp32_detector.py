"""The device's FP32 test of the smooth class (no GPU): a host build of the same function
(swale_cell.cuh, sure_smooth_f32 on inputs truncated to FP32 by f32_trunc) against the FP64
class of the same indicators (shared_beta + hybrid_phi, Step 2 of Sec. 2.2 with the shared
indicators of Eq. alphamodified).

The FP32 test may only say "smooth" where the FP64 detector finds gamma <= 1/2: it is a shortcut,
never a second opinion. It must also say so for most clearly smooth cells, or it saves nothing.
"""
import numpy as np
import pytest

from paper_2208_06588_gb300 import cellcheck as C


def _gamma(b, eps):
    return abs(b[0] - b[2]) / (b.mean() + eps)


def _random_cell(rng, scale_spread=6.0):
    """Mesh factors and divided differences over many orders of magnitude, with cancellation
    between D2 and D3 F (q = D2 + D3 F small while both terms are large)."""
    dx = 10.0 ** rng.uniform(-6, 2)
    h2 = dx * rng.uniform(0.2, 1.0)
    F = h2 * rng.uniform(-2.0, 2.0, 3)
    c4 = 4.0 * dx * h2
    c3 = (3.0 * h2 * h2 + 36.0 * dx * dx) * dx * h2
    s = 10.0 ** rng.uniform(-scale_spread, scale_spread)
    D3h = s / h2 * rng.normal(size=3)
    D3m = s / h2 * rng.normal(size=3)
    D2h = s * rng.normal(size=3)
    D2m = s * rng.normal(size=3)
    kind = rng.integers(4)
    if kind == 1:  # near cancellation in q
        D2h = -D3h * F * (1.0 + 1e-6 * rng.normal(size=3))
    elif kind == 2:  # smooth data: third differences small
        D3h *= 1e-3
        D3m *= 1e-3
        D2h = D2h[0] + 1e-3 * D2h
        D2m = D2m[0] + 1e-3 * D2m
    elif kind == 3:  # still water: exact zeros
        D2m = np.zeros(3)
        D3m = np.zeros(3)
    return F, c4, c3, D2h, D3h, D2m, D3m


def test_fp32_smooth_implies_fp64_smooth_on_random_cells():
    rng = np.random.default_rng(20220812)
    sure_n = smooth_n = 0
    for _ in range(20000):
        args = _random_cell(rng)
        eps = 10.0 ** rng.uniform(-12, -4)
        sure, flag, b = C.smooth_test(*args, eps=eps)
        if sure:
            sure_n += 1
            assert flag == 0, (args, eps, b, _gamma(b, eps))
        if flag == 0:
            smooth_n += 1
    # the shortcut decides most of the smooth cells
    assert sure_n > 0.9 * smooth_n, (sure_n, smooth_n)


@pytest.mark.parametrize("seed", range(6))
def test_fp32_test_stays_off_near_the_threshold(seed):
    """Scale one difference so that the FP64 gamma crosses 1/2: just above it (class 1) the
    FP32 test must never claim the smooth class, just below it it may decline."""
    rng = np.random.default_rng(seed)
    F, c4, c3, D2h, D3h, D2m, D3m = _random_cell(rng, scale_spread=2.0)
    eps = 1e-6
    base = D2h.copy()

    def at(s):
        d = base.copy()
        d[0] = base[0] * s
        return C.smooth_test(F, c4, c3, d, D3h, D2m, D3m, eps=eps)

    g = lambda s: _gamma(at(s)[2], eps)
    lo, hi = 0.0, 1.0
    # find a scale with gamma above 1/2, then bisect to the crossing
    for _ in range(60):
        if g(hi) > 0.5:
            break
        hi *= 2.0
    if g(hi) <= 0.5 or g(lo) > 0.5:
        pytest.skip("this draw does not cross the threshold along the scaled direction")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.5:
            hi = mid
        else:
            lo = mid
    for s in np.linspace(lo, hi, 9):
        sure, flag, b = at(s)
        if flag != 0:
            assert not sure
    # a little inside the smooth range the shortcut still declines (it keeps a margin)
    sure, flag, b = at(lo)
    assert flag == 0 and not sure


def test_fp32_test_on_still_water_and_non_finite_data():
    F, c4, c3 = np.array([1e-3, 5e-4, -5e-4]), 4e-6, 4e-12
    z = np.zeros(3)
    assert C.smooth_test(F, c4, c3, z, z, z, z, 1e-6)[:2] == (True, 0)
    nan = np.array([np.nan, 0.0, 0.0])
    assert C.smooth_test(F, c4, c3, nan, z, z, z, 1e-6)[0] is False
    big = np.array([1e200, 0.0, 0.0])
    assert C.smooth_test(F, c4, c3, big, z, z, z, 1e-6)[0] is False


def test_f32_trunc_matches_the_float_conversion_toward_zero():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.uniform(-30, 30, 1000), [0.0, -0.0, 1.0, -2.5]])
    got = np.array([C.f32_trunc(v) for v in x], dtype=np.float32)
    ref = x.astype(np.float32)  # round to nearest
    # truncation: |got| <= |x|, within one float ulp of the rounded value, same sign
    assert np.all(np.abs(got.astype(np.float64)) <= np.abs(x))
    assert np.all(np.abs(got - ref) <= np.spacing(np.abs(ref)))
    assert np.all(np.signbit(got) == np.signbit(x))
    assert C.f32_trunc(1e300) == np.inf and C.f32_trunc(-1e300) == -np.inf and C.f32_trunc(1e-50) == 0.0
