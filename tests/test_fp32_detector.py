"""The device's FP32 test of the smooth class (no GPU): a host build of the same function
(swale_cell.cuh, sure_smooth_f32 on inputs truncated to FP32 by f32_trunc) against the FP64
class of the same indicators (shared_beta + hybrid_phi, Step 2 of Sec. 2.2 with the shared
indicators of Eq. alphamodified).

The FP32 test may only say "smooth" where the FP64 detector finds gamma <= 1/2: it is a shortcut,
never a second opinion. It must also say so for most clearly smooth cells, or it saves nothing.
"""
import numpy as np
import pytest

from tests import cellcheck as C


def _gamma(b, eps):
    return abs(b[0] - b[2]) / (b.mean() + eps)


def _random_cell(rng, scale_spread=6.0):
    """A 5-cell stencil over many orders of magnitude of widths and data: the mesh factors of
    the indicators (F, c4, c3 as the cell geometry forms them), the pair differences D2 of h and
    hu on its four pairs and the reciprocal sums of its three triples. Kinds: random data, near
    cancellation between D2 and D3 F, smooth data (small second differences), still water."""
    dx = 10.0 ** rng.uniform(-6, 2)
    w = dx * rng.uniform(0.2, 1.0, 5)  # widths J_{j-2..j+2}
    F = np.array([1.5 * w[2] + w[0] + 2 * w[1], 0.5 * w[2] + w[1], -(0.5 * w[2] + w[3])])  # for the cancellations
    it = 1.0 / (w[:3] + w[1:4] + w[2:])
    s = 10.0 ** rng.uniform(-scale_spread, scale_spread)
    kind = rng.integers(4)
    D2h, D2m = s * rng.normal(size=4), s * rng.normal(size=4)
    if kind == 1:  # q = D2 + D3 F nearly cancels on one sub-stencil
        a = rng.integers(3)
        D2h[a] = -(D2h[a + 1] * it[a] * F[a]) / (1.0 - it[a] * F[a]) * (1.0 + 1e-6 * rng.normal())
    elif kind == 2:  # smooth data: nearly equal pair differences
        D2h = D2h[0] * (1.0 + 1e-3 * rng.normal(size=4))
        D2m = D2m[0] * (1.0 + 1e-3 * rng.normal(size=4))
    elif kind == 3:  # still water: no discharge
        D2m = np.zeros(4)
    return w, dx, D2h, D2m, it


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


@pytest.mark.parametrize("seed", range(8))
def test_fp32_test_stays_off_near_the_threshold(seed):
    """Blend a smooth stencil (gamma near 0) into a rough one (gamma above 1) and bisect the
    blend to where the FP64 gamma crosses 1/2: above it (class 1) the FP32 test must never claim
    the smooth class, and a hair below it (gamma = 0.5 (1 - 1e-8)) it declines too: it keeps a
    margin of about 1e-5 relative."""
    rng = np.random.default_rng(seed)
    w5, dx, _, _, it = _random_cell(rng, scale_spread=2.0)
    eps = 1e-6
    sh, sm = 10.0 ** rng.uniform(-2, 2, 2)
    smooth_h = sh * (1.0 + 1e-3 * rng.normal(size=4))
    smooth_m = sm * (1.0 + 1e-3 * rng.normal(size=4))
    for _ in range(100):
        rough_h, rough_m = sh * rng.normal(size=4) * 10.0, sm * rng.normal(size=4) * 10.0
        if C.smooth_test(w5, dx, rough_h, rough_m, it, eps=eps)[1] == 2:
            break
    at = lambda t: C.smooth_test(w5, dx, (1 - t) * smooth_h + t * rough_h, (1 - t) * smooth_m + t * rough_m, it,
                                 eps=eps)
    g = lambda t: _gamma(at(t)[2], eps)

    def crossing(level):
        lo, hi = 0.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if g(mid) > level:
                hi = mid
            else:
                lo = mid
        return lo, hi

    assert g(0.0) < 0.4 and g(1.0) > 1.0
    lo, hi = crossing(0.5)
    for t in np.linspace(lo, 1.0, 33):
        sure, flag, b = at(t)
        if flag != 0:
            assert not sure
    for rel in (1e-12, 1e-9, 1e-7, 1e-6, 1e-5):  # just above the threshold: class 1
        _, hi = crossing(0.5 * (1.0 + rel))
        sure, flag, b = at(hi)
        assert flag == 1 and not sure, rel
    lo, _ = crossing(0.5 * (1.0 - 1e-8))
    sure, flag, b = at(lo)
    assert flag == 0 and not sure
    # well inside the smooth class the test decides
    assert at(0.0)[0]


def test_fp32_test_on_still_water_and_non_finite_data():
    w5, dx, it = np.full(5, 1e-3), 1e-3, np.full(3, 1.0 / 3e-3)
    z = np.zeros(4)
    assert C.smooth_test(w5, dx, z, z, it, 1e-6)[:2] == (True, 0)
    nan = np.array([np.nan, 0.0, 0.0, 0.0])
    assert C.smooth_test(w5, dx, nan, z, it, 1e-6)[0] is False
    big = np.array([1e200, 0.0, 0.0, 0.0])
    assert C.smooth_test(w5, dx, big, z, it, 1e-6)[0] is False
    # widths far beyond the FP32 range: the factors overflow, the test declines
    assert C.smooth_test(np.full(5, 1e30), 1e30, z + 1.0, z, np.full(3, 1e-30), 1e-6)[0] is False


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


def _random_field_cell(rng):
    """Projection rows of a wet cell (u, c) and the stencil data of eta, hu, h."""
    w5, dx, D2h, D2m, it = _random_cell(rng)
    s = np.abs(D2h).max() + np.abs(D2m).max() + 1e-300
    D2e = D2h + s * (1e-3 * rng.normal(size=4) if rng.random() < 0.5 else rng.normal(size=4))
    u, c = rng.normal(), 10.0 ** rng.uniform(-1, 1.5)
    if rng.random() < 0.2:  # a dry cell: identity rows
        proj = np.array([1.0, 0.0, 0.0, 1.0])
    else:
        i2c = 0.5 / c
        proj = np.array([(u + c) * i2c, -i2c, (c - u) * i2c, i2c])
    return proj, D2e, D2m, D2h, it, w5, dx


def test_field_fp32_smooth_implies_fp64_smooth():
    """The non-well-balanced scheme's test of each characteristic field and of the bottom."""
    rng = np.random.default_rng(7)
    sure_n = smooth_n = 0
    for _ in range(15000):
        args = _random_field_cell(rng)
        eps = 10.0 ** rng.uniform(-12, -4)
        sure, cls, _ = C.smooth1_test(*args, eps=eps)
        for s_, c_ in zip(sure, cls):
            if s_:
                sure_n += 1
                assert c_ == 0, (args, eps)
            smooth_n += c_ == 0
    assert sure_n > 0.9 * smooth_n, (sure_n, smooth_n)


@pytest.mark.parametrize("seed", range(6))
def test_field_fp32_test_stays_off_near_the_threshold(seed):
    """Blend smooth stencil data into rough data and bisect the blend to where a field's FP64
    gamma crosses 1/2: just above it the field's FP32 test never claims the smooth class, a hair
    below it it declines too."""
    rng = np.random.default_rng(100 + seed)
    proj, _, _, _, it, w5, dx = _random_field_cell(rng)
    eps = 1e-6
    s = 10.0 ** rng.uniform(-2, 2)
    smooth = [s * (1.0 + 1e-3 * rng.normal(size=4)) for _ in range(3)]
    for _ in range(100):
        rough = [s * 10.0 * rng.normal(size=4) for _ in range(3)]
        if min(C.smooth1_test(proj, *rough, it, w5, dx, eps)[1]) == 2:
            break
    at = lambda t: C.smooth1_test(proj, *[(1 - t) * a + t * b for a, b in zip(smooth, rough)], it, w5, dx, eps)
    g0, g1 = at(0.0)[2], at(1.0)[2]
    crossed = 0
    for f in range(3):
        if not (g0[f] < 0.4 and g1[f] > 1.0):
            continue
        crossed += 1

        def crossing(level):
            lo, hi = 0.0, 1.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if at(mid)[2][f] > level:
                    hi = mid
                else:
                    lo = mid
            return lo, hi

        for rel in (1e-12, 1e-9, 1e-7, 1e-6, 1e-5):
            _, hi = crossing(0.5 * (1.0 + rel))
            sure, cls, g = at(hi)
            assert cls[f] == 1 and not sure[f], (f, rel)
        lo, _ = crossing(0.5 * (1.0 - 1e-8))
        sure, cls, g = at(lo)
        assert cls[f] == 0 and not sure[f]
    assert crossed >= 1
