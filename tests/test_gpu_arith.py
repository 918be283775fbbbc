"""The FP64 arithmetic the kernels use in place of FP64 divisions and comparisons, checked on the GPU
against CUDA's own operations through mgfld_arith_check: the seeded quotient and the two-step
reciprocal within an ulp of CUDA's correctly rounded results, the one-step seed within 2^-45, and the
integer-pipe comparisons (order keys, the zero test) giving exactly the FP64 comparisons' outcomes,
subnormals and infinities included (the order key alone puts -0 below +0)."""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

M = None


@pytest.fixture(scope='module', autouse=True)
def _lib():
    global M
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1809_05608_gb300 import mgfld
    M = mgfld
    M.lib()


def _random_doubles(rng, n, emin, emax):
    """Mantissas uniform in [1, 2), exponents uniform in [emin, emax], random signs."""
    m = rng.uniform(1.0, 2.0, n)
    e = rng.integers(emin, emax + 1, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def _run(a, b):
    out = M.arith_check(torch.as_tensor(a, device='cuda'), torch.as_tensor(b, device='cuda'))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ulps(x, ref):
    """|x - ref| in units of the last place of ref."""
    return np.abs(x - ref) / np.spacing(np.abs(ref))


def test_quotients_and_reciprocals_within_an_ulp():
    rng = np.random.default_rng(1809)
    n = 1 << 18
    a = _random_doubles(rng, n, -400, 400)
    b = _random_doubles(rng, n, -400, 400)
    # near-equal pairs and exact multiples, where rounding decisions are closest
    a[: n // 8] = b[: n // 8] * (1.0 + rng.uniform(-1e-12, 1e-12, n // 8))
    a[n // 8: n // 4] = b[n // 8: n // 4] * rng.integers(1, 1000, n // 8)
    o = _run(a, b)
    q_lib, q_cuda, r2_lib, r_cuda, r1_lib = o[:, 0], o[:, 1], o[:, 2], o[:, 3], o[:, 4]
    normal = (np.abs(q_cuda) > 1e-300) & (np.abs(q_cuda) < 1e300)
    assert normal.mean() > 0.9
    uq = _ulps(q_lib[normal], q_cuda[normal])
    ur = _ulps(r2_lib, r_cuda)
    print(f'quotient: max {uq.max():.2f} ulp, {np.mean(uq == 0):.4f} equal to the correctly rounded; '
          f'reciprocal: max {ur.max():.2f} ulp, {np.mean(ur == 0):.4f} equal')
    assert uq.max() <= 1.0 and ur.max() <= 1.0
    rel = np.abs(r1_lib / r_cuda - 1.0)
    assert rel.max() <= 2.0 ** -45
    # exact cases: n / 1, n / n, powers of two
    o = _run(np.array([3.0, 7.5, -2.0, 1.0, 6.0]), np.array([1.0, 7.5, 0.5, 4.0, -3.0]))
    assert np.array_equal(o[:, 0], o[:, 1])


def test_quotients_at_the_edges_of_the_range():
    """Divisors whose reciprocal the seed cannot form (zero, subnormal, huge, non-finite) take a
    plain division: CUDA's results, infinities and NaNs in the same places."""
    b = np.array([0.0, -0.0, 5e-324, 1e-310, 1e308, -1e308, np.inf, -np.inf, np.nan, 2.0 ** 1023])
    a = np.ones_like(b)
    o = _run(a, b)
    for col_lib, col_cuda in ((0, 1), (2, 3), (4, 3)):
        x, y = o[:, col_lib], o[:, col_cuda]
        same = (x == y) | (np.isnan(x) & np.isnan(y)) | (_ulps(np.where(np.isfinite(y), x, 0.0),
                                                              np.where(np.isfinite(y), y, 1.0)) <= 1.0)
        assert np.all(same), (col_lib, x, y)


def test_integer_pipe_comparisons_match_fp64():
    rng = np.random.default_rng(5608)
    n = 1 << 18
    a = _random_doubles(rng, n, -1074, 1023)
    b = _random_doubles(rng, n, -1074, 1023)
    specials = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2e-308, -2.2e-308, 1.0, -1.0, np.inf, -np.inf, 1e-300])
    sa, sb = np.meshgrid(specials, specials)
    a = np.concatenate([a, b[:1000], sa.ravel()])
    b = np.concatenate([b, b[:1000], sb.ravel()])       # equal pairs too
    o = _run(a, b)
    # the order key puts -0 just below +0 (the kernels compare by it only where a tie of zeros
    # cannot change the outcome); every other pair orders as the FP64 comparison does
    zz = (a == 0.0) & (b == 0.0)
    assert np.array_equal(o[~zz, 5], o[~zz, 6])
    assert np.array_equal(o[zz, 5], (np.signbit(a[zz]) & ~np.signbit(b[zz])).astype(np.float64))
    assert np.array_equal(o[:, 7], (a == 0.0).astype(np.float64))
