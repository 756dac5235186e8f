"""Pins of the oracle's stencil geometry against closed forms and printed values.

Each check fixes a fact the paper or plain mathematics determines independently of the
oracle's code: exactness of interpolation on bilinear functions, the interpolation-error
term on x1^2, the consistency equations of the truncated weights (Eqs. 2.5, 2.6), the
growth bounds of Corollary 2.3, and the printed stencil lengths / radius.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import lisl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _const_problem(n, sig, lo=-2.0, hi=2.0, drift=None):
    sig = np.asarray(sig, dtype=np.float64)
    if sig.ndim == 2:
        sig = sig[None]
    p = W.Problem(name="t", n=n, lo=lo, hi=hi, T=1.0, n_steps=1, sigma=sig, phi=None, G=None,
                  tau_kind=None, tau_rate=None, g=np.zeros((n, n)),
                  psi_fn=lambda t: np.zeros((n, n)))
    if drift is not None:
        p.drift = np.asarray(drift, dtype=np.float64)[None]
    return p


def _lhat_of(p, k, q):
    """Interpolated truncated operator applied to q, at all interior nodes."""
    n = p.n
    i1, i2, flat = lisl.interior_flat(n)
    X1, X2 = p.coords()
    tp = lisl.control_taps(p, k, i1, i2)
    return lisl.apply_lhat(tp, q(X1, X2), flat), tp


SIGMAS = [
    [[0.3, 0.0], [0.2 * 0.5, 0.2 * math.sqrt(0.75)]],      # config-like, no truncation at 33^2
    [[1.2, 0.0], [1.2 * -0.8, 1.2 * 0.6]],                   # truncation-heavy, two-sided at corners
    [[0.7, -0.4], [0.9, 1.1]],                                # generic oblique columns
]


@pytest.mark.parametrize("sig", SIGMAS)
@pytest.mark.parametrize("n", [17, 33])
def test_bilinear_functions_are_differentiated_exactly(sig, n):
    """Bilinear interpolation reproduces span{1, x1, x2, x1 x2}, and the truncated weights are
    exact on quadratics along each direction (Eqs. 2.5, 2.6), so L q = tr(a D^2 q) exactly
    for these q at every row, truncated or not: 0 for 1, x1, x2 and (sigma sigma^T)_12 for x1 x2."""
    p = _const_problem(n, sig)
    S = np.asarray(sig)
    a12x2 = (S @ S.T)[0, 1]
    for q, expect in [(lambda x, y: np.ones_like(x), 0.0), (lambda x, y: x, 0.0),
                      (lambda x, y: y, 0.0), (lambda x, y: x * y, a12x2)]:
        v, tp = _lhat_of(p, 0, q)
        scale = np.max(tp.W) * 4.0
        assert np.max(np.abs(v - expect)) <= 1e-13 * max(1.0, scale)


def test_truncation_occurs_in_heavy_case():
    p = _const_problem(33, SIGMAS[1])
    i1, i2, _ = lisl.interior_flat(33)
    tp = lisl.control_taps(p, 0, i1, i2)
    M = 2
    truncated = tp.W > M / p.h * (1 + 1e-14)
    assert truncated.sum() > 100
    assert (~truncated).sum() > 100


@pytest.mark.parametrize("sig", [SIGMAS[0], SIGMAS[2]])
def test_interpolation_error_term_on_x1_squared(sig):
    """Linear interpolation of x^2 at fractional position t adds h^2 t (1 - t); at untruncated
    rows L x1^2 = (sigma sigma^T)_11 + h sum_p t_p (1 - t_p), t_p = frac(sigma_p1 / sqrt h)."""
    n = 65
    p = _const_problem(n, sig)
    S = np.asarray(sig)
    h = p.h
    v, tp = _lhat_of(p, 0, lambda x, y: x * x)
    untrunc = np.abs(tp.W - 2 / h) <= 1e-12 / h
    t = [math.modf(abs(S[0, j]) / math.sqrt(h))[0] for j in range(2)]
    expect = (S @ S.T)[0, 0] + h * sum(tj * (1 - tj) for tj in t)
    assert untrunc.sum() > 0
    assert np.max(np.abs(v[untrunc] - expect)) <= 1e-10


def test_truncated_weights_consistency_and_bounds():
    """A s+ + B s- = 0 and A s+ s+^T + B s- s-^T = 2 s s^T (Eqs. 2.5, 2.6 in index units,
    s = sigma / sqrt(dx)), A, B >= 1 (Corollary 2.3 a), A = B = 1 without truncation."""
    n = 33
    i1, i2 = lisl.interior_nodes(n)
    rng = np.random.default_rng(7)
    for _ in range(20):
        s = rng.normal(size=2) * rng.uniform(0.5, 12.0)
        s1 = np.full_like(i1, s[0])
        s2 = np.full_like(i1, s[1])
        mup, zp1, zp2 = lisl.truncate(i1, i2, s1, s2, n)
        mum, zm1, zm2 = lisl.truncate(i1, i2, -s1, -s2, n)
        A = 2.0 / (mup * mup + mup * mum)
        B = 2.0 / (mum * mum + mum * mup)
        yp = np.stack([zp1 - i1, zp2 - i2])
        ym = np.stack([zm1 - i1, zm2 - i2])
        scale = np.max(np.abs(s)) ** 2
        assert np.max(np.abs(A * yp + B * ym)) <= 1e-12 * np.max(np.abs(s)) * np.max(A + B)
        for a in range(2):
            for b in range(2):
                lhs = A * yp[a] * yp[b] + B * ym[a] * ym[b]
                assert np.max(np.abs(lhs - 2 * s[a] * s[b])) <= 1e-11 * scale * np.max(A + B)
        assert np.all(A >= 1 - 1e-15) and np.all(B >= 1 - 1e-15)
        un = (mup == 1.0) & (mum == 1.0)
        assert np.all(A[un] == 1.0) and np.all(B[un] == 1.0)
        # endpoints stay in the closed domain
        for z in (zp1, zp2, zm1, zm2):
            assert np.all(z >= 0.0) and np.all(z <= n - 1)


@pytest.mark.parametrize("sig", SIGMAS)
def test_exact_endpoint_scheme_is_exact_on_quadratics(sig):
    """Remark 2.2 variant (exact values at the truncated endpoints): by Eqs. 2.5/2.6 the
    truncated diffusion part is exact for every quadratic, including rows with two-sided
    overstepping."""
    n = 33
    p = _const_problem(n, sig)
    i1, i2 = lisl.interior_nodes(n)
    S = np.asarray(sig)
    a = 0.5 * S @ S.T
    rng = np.random.default_rng(3)
    c = rng.normal(size=6)

    def q(x, y):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y

    D2 = np.array([[2 * c[3], c[4]], [c[4], 2 * c[5]]])
    expect = np.trace(a @ D2)
    got = lisl.lhat_apply_exact_endpoints(p, 0, i1, i2, q)
    assert np.max(np.abs(got - expect)) <= 1e-9 * (1 + abs(expect))


def test_truncated_drift_is_exact_on_linear_functions():
    """Drift direction with A = B = 1/mu (Eqs. 2.2 / 2.4): the truncated one-sided
    difference reproduces b . Dq exactly for linear q, also where x + dx b oversteps."""
    n = 17
    drift = [7.5, -3.2]            # index units: 7.5 cells, so rows near the boundary truncate
    p = _const_problem(n, [[0.0, 0.0], [0.0, 0.0]], drift=drift)
    i1, i2 = lisl.interior_nodes(n)
    q = lambda x, y: 0.3 + 1.7 * x - 2.9 * y
    got = lisl.lhat_apply_exact_endpoints(p, 0, i1, i2, q)
    assert np.max(np.abs(got - (1.7 * 7.5 + 2.9 * 3.2))) <= 1e-11
    # with interpolation as well (bilinear interpolation is exact on linear functions)
    X1, X2 = p.coords()
    i1f, i2f, flat = lisl.interior_flat(n)
    tp = lisl.control_taps(p, 0, i1f, i2f)
    assert np.max(tp.W) > 1.01 * np.min(tp.W)          # some rows are truncated
    v = lisl.apply_lhat(tp, q(X1, X2), flat)
    assert np.max(np.abs(v - (1.7 * 7.5 + 2.9 * 3.2))) <= 1e-10


def test_weight_growth_rates():
    """Corollary 2.3 b: one-sided truncation at distance dx gives A ~ 2 dx^{-1/2} and
    B -> 2 (both with O(sqrt dx) relative corrections); two-sided truncation gives
    A, B ~ dx^{-1}."""
    for n in (65, 257, 1025, 4097):
        h = 1.0 / (n - 1)
        s = 1.0 / math.sqrt(h)          # sigma = 1 along x1
        i1 = np.array([1.0])
        i2 = np.array([(n - 1) / 2.0])
        mup, _, _ = lisl.truncate(i1, i2, np.array([-s]), np.array([0.0]), n)
        mum, _, _ = lisl.truncate(i1, i2, np.array([s]), np.array([0.0]), n)
        A = 2 / (mup ** 2 + mup * mum)
        B = 2 / (mum ** 2 + mum * mup)
        assert abs(A[0] * math.sqrt(h) - 2.0) <= 2.5 * math.sqrt(h)
        assert abs(B[0] - 2.0) <= 2.5 * math.sqrt(h)
    for n in (65, 257, 1025):
        h = 1.0 / (n - 1)
        s = 1.0 / math.sqrt(h)          # direction (1, -1) through the node next to a corner:
        i = np.array([1.0])             # both ends overstep at mu = 1/s = sqrt(dx)
        mup, _, _ = lisl.truncate(i, i, np.array([s]), np.array([-s]), n)
        mum, _, _ = lisl.truncate(i, i, np.array([-s]), np.array([s]), n)
        A = 2 / (mup ** 2 + mup * mum)
        B = 2 / (mum ** 2 + mum * mup)
        assert mup[0] < 1.0 and mum[0] < 1.0
        assert abs(A[0] * h - 1.0) <= 1e-12 and abs(B[0] * h - 1.0) <= 1e-12
    n = 9
    mup, _, _ = lisl.truncate(np.array([1.0]), np.array([1.0]), np.array([20.0]), np.array([20.0]), n)
    mum, _, _ = lisl.truncate(np.array([1.0]), np.array([1.0]), np.array([-20.0]), np.array([-20.0]), n)
    assert mup[0] < 1 and mum[0] < 1


def test_stencil_length_table_3_1():
    """Stencil length of Eq. 3.2: for sigma = s I the nearest positive-weight tap of the
    oracle's stencil along x1 sits m = floor(s / sqrt(dx)) cells from the node (Table 3.1)."""
    gold = json.load(open(os.path.join(GOLD, "table_3_1_stencil_length.json")))
    for key, sig in (("sigma_2", 2.0), ("sigma_sqrt5", math.sqrt(5.0))):
        for l, m in gold[key].items():
            n = 2 ** int(l) + 1
            p = _const_problem(n, [[sig, 0.0], [0.0, sig]], lo=0.0, hi=1.0)
            c = (n - 1) // 2
            tp = lisl.control_taps(p, 0, np.array([float(c)]), np.array([float(c)]))
            col1 = tp.cols % n - c
            col2 = tp.cols // n - c
            along = (col2 == 0) & (tp.w > 0) & (col1 > 0)
            assert int(col1[along].min()) == m


def test_stencil_radius_figure_2_2():
    """Radius ||sigma|| / sqrt(dx) = 14.27 of the Problem B stencil on the 641 x 641 grid."""
    gold = json.load(open(os.path.join(GOLD, "figure_2_2_radius.json")))
    p = W.problem_B(641)
    c = 320.0
    radii = []
    for k in range(p.K):
        sig = lisl.control_sigma(p, k, np.array([c]), np.array([c]))
        s = sig[:, :, 0] / math.sqrt(p.h)
        _, z1, z2 = lisl.truncate(np.array([c]), np.array([c]), s[:, 0], s[:, 1], p.n)
        radii.append(math.hypot(z1[0] - c, z2[0] - c))
    assert max(radii) - min(radii) < 1e-9
    assert abs(radii[0] - gold["radius"]) < 0.005


@pytest.mark.parametrize("make", [lambda: W.oracle_scale(), lambda: W.oracle_scale(truncation_heavy=True),
                                  lambda: W.problem_A(33), lambda: W.problem_B(33)],
                         ids=["plain", "truncated", "problemA", "problemB"])
def test_tap_weights_sum_to_W(make):
    """Every row's tap weights add up to its W: each of the scheme's points is split over the
    corners of its cell with bilinear weights that sum to one (Section 2.1), and W is the sum
    of the point weights.  The FP64 residual kernel relies on this identity: it forms
    sum_t w_t (X_t - X_j) as sum_t w_t x'_t - W x'_j on a tile centred at one value."""
    p = make()
    n = p.n
    i1, i2 = np.meshgrid(np.arange(1, n - 1), np.arange(1, n - 1))
    i1, i2 = i1.ravel(), i2.ravel()
    K = p.sigma.shape[0] if p.sigma is not None else 8
    for k in range(min(K, 8)):
        tp = lisl.control_taps(p, k, i1, i2)
        s = np.bincount(tp.rows, weights=tp.w, minlength=len(i1))
        assert np.all(tp.W > 0)
        np.testing.assert_allclose(s, tp.W, rtol=4 * np.finfo(float).eps, atol=0)
