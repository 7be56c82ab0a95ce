"""The allocation-free entry point swale_rhs_noalloc against the ordinary swale_rhs.

swale_rhs_noalloc serves callers that cannot call cudaMalloc (code inside another
framework's memory pool, or work that must not grow device memory): its scratch is one fixed
device array shared by every call. This file is collected last so that a failure here comes
after every other test has run; it passes both alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

from paper_2208_06588_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _inputs(N, seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([[0.0], np.cumsum(rng.uniform(0.6, 1.4, N))]) / N
    J = np.diff(x)
    xc = 0.5 * (x[1:] + x[:-1])
    Bv = 0.5 + 0.3 * np.sin(5 * xc) + 0.2 * (xc > 0.6)
    h = 1.0 + 0.4 * np.cos(3 * xc) + 0.5 * (xc < 0.3)
    h[N // 2:N // 2 + 3] = 0.0
    E = h + Bv
    M = h * (0.3 * np.sin(7 * xc) + 0.5 * (xc > 0.45))
    w = rng.normal(size=N + 1) * 0.05
    w[0] = w[-1] = 0.0
    return E, M, Bv, J, w


@pytest.mark.parametrize("scheme,bc", [("hydrostatic", "reflective"), ("hydrostatic", "periodic"),
                                       ("nonwb", "transmissive"), ("special", "reflective")])
def test_noalloc_matches_swale_rhs_on_two_calls(scheme, bc):
    torch = pytest.importorskip("torch")
    from paper_2208_06588_gb300 import build
    build.build()
    cfg = B.make_config(bc=bc, scheme=scheme)
    stream = torch.cuda.current_stream().cuda_stream
    alpha = 7.5
    # Two calls in a row: the second is smaller and reuses the scratch left by the first.
    for N, seed in ((3000, 11), (1000, 12)):
        E, M, Bv, J, w = _inputs(N, seed)
        ctx = B.swale_create(cfg)
        RE, RM, RB = np.zeros(N), np.zeros(N), np.zeros(N)
        fl = np.zeros(N, dtype=np.uint8)
        A_ref, _ = B.swale_rhs(ctx, N, E, M, Bv, J, w, alpha, RE, RM, RB, fl)
        B.swale_destroy(ctx)

        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (E, M, Bv, J, w)]
        out = [torch.full((N,), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
        gfl = torch.full((N,), 9, dtype=torch.uint8, device="cuda")
        A = B.swale_rhs_noalloc(cfg, stream, N, *dev, alpha, *out, gfl)
        torch.cuda.synchronize()
        scale = max(np.abs(RE).max(), np.abs(RM).max(), np.abs(RB).max())
        for g, r in zip(out, (RE, RM, RB)):
            assert np.abs(g.cpu().numpy() - r).max() <= 1e-11 * scale
        assert np.array_equal(gfl.cpu().numpy(), fl)
        assert abs(A - A_ref) <= 1e-14 * A_ref


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    N = B.NOALLOC_MAX_CELLS + 1
    z = [torch.zeros(N + 1, dtype=torch.float64, device="cuda") for _ in range(8)]
    with pytest.raises(B.SwaleError) as e:
        B.swale_rhs_noalloc(B.make_config(), None, N, *z[:5], 1.0, *z[5:8])
    assert e.value.code == -1
