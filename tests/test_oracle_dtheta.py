"""Pins of the oracle's closed-form derivative of the truncated Scheme-2 operator in sigma
(oracle/adjoint.py, dlhat_dtheta), which the oracle's dJ/dtheta is built on.

* Bilinear data, every row (truncated or not): bilinear interpolation reproduces
  span{1, x1, x2, x1 x2} and the truncated weights satisfy Eqs. 2.5 and 2.6 identically in sigma,
  so L q = sum_p sigma_p1 sigma_p2 c for q = a + b1 x1 + b2 x2 + c x1 x2, and therefore
  dL q / dtheta = c sum_p (dsigma_p1 sigma_p2 + sigma_p1 dsigma_p2).  A wrong dA, dB, d mu or
  endpoint motion on a truncated row breaks the cancellation of the linear terms.
* x1^2 at untruncated rows: L x1^2 = (sigma sigma^T)_11 + h sum_p t_p (1 - t_p) with
  t_p = frac(sigma_p1 / sqrt h), so dL x1^2 / dtheta = sum_p (2 sigma_p1 + sqrt(h) (1 - 2 t_p)) dsigma_p1.
* Generic data and truncation: a fourth-order central difference of the operator in theta,
  on the rows whose taps keep their cells over the stencil of the difference.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj
from oracle import lisl

SIGMAS = [
    [[0.3, 0.0], [0.2 * 0.5, 0.2 * math.sqrt(0.75)]],
    [[1.2, 0.0], [1.2 * -0.8, 1.2 * 0.6]],      # truncation-heavy, two-sided at corners
    [[0.7, -0.4], [0.9, 1.1]],                   # generic oblique columns
]
DSIGMAS = [
    [[1.0, 0.0], [0.0, 0.0]],
    [[0.0, 0.0], [-0.8, 0.6]],
    [[0.3, -0.7], [0.5, 0.2]],
]


def _problem(n, sig):
    sig = np.asarray(sig, dtype=np.float64)[None]
    return W.Problem(name="t", n=n, lo=-2.0, hi=2.0, T=1.0, n_steps=1, sigma=sig, phi=None, G=None,
                     tau_kind=None, tau_rate=None, g=np.zeros((n, n)),
                     psi_fn=lambda t: np.zeros((n, n)))


def _truncated_rows(p):
    i1, i2, _ = lisl.interior_flat(p.n)
    tp = lisl.control_taps(p, 0, i1, i2)
    return tp.W > p.sigma.shape[2] / p.h * (1 + 1e-14)   # W = P / h without truncation


@pytest.mark.parametrize("sig", SIGMAS)
@pytest.mark.parametrize("dsig", DSIGMAS)
@pytest.mark.parametrize("n", [17, 33])
def test_bilinear_data_every_row(sig, dsig, n):
    p = _problem(n, sig)
    S, dS = np.asarray(sig), np.asarray(dsig)
    X1, X2 = p.coords()
    rng = np.random.default_rng(n)
    a, b1, b2, c = rng.normal(size=4)
    q = a + b1 * X1 + b2 * X2 + c * X1 * X2
    i1, i2, _ = lisl.interior_flat(n)
    d = adj.dlhat_dtheta(p, 0, dS, q, i1, i2)
    expect = c * float(np.sum(dS[0] * S[1] + S[0] * dS[1]))
    scale = 4.0 * float(np.max(np.abs(q))) / p.h
    assert np.max(np.abs(d - expect)) <= 1e-12 * scale
    if sig is SIGMAS[1]:
        assert _truncated_rows(p).sum() > 50


@pytest.mark.parametrize("sig", [SIGMAS[0], SIGMAS[2]])
@pytest.mark.parametrize("dsig", DSIGMAS)
def test_x1_squared_untruncated_rows(sig, dsig):
    n = 65
    p = _problem(n, sig)
    S, dS = np.asarray(sig), np.asarray(dsig)
    X1, _ = p.coords()
    i1, i2, _ = lisl.interior_flat(n)
    if np.any((S[0] == 0.0) & (dS[0] != 0.0)):
        pytest.skip("moves an offset component that is exactly zero: a kink of the operator")
    d = adj.dlhat_dtheta(p, 0, dS, X1 * X1, i1, i2)
    rh = math.sqrt(p.h)
    expect = 0.0
    for j in range(S.shape[1]):
        s = S[0, j] / rh
        t = s - math.floor(s)
        expect += (2.0 * S[0, j] + rh * (1.0 - 2.0 * t)) * dS[0, j]
    untrunc = ~_truncated_rows(p)
    assert untrunc.sum() > 0
    assert np.max(np.abs(d[untrunc] - expect)) <= 1e-10


def _lhat(p, sigma, U, i1, i2, flat):
    q = W.Problem(name="t", n=p.n, lo=p.lo, hi=p.hi, T=1.0, n_steps=1, sigma=sigma[None], phi=None,
                  G=None, tau_kind=None, tau_rate=None, g=p.g, psi_fn=p.psi_fn)
    tp = lisl.control_taps(q, 0, i1, i2)
    return lisl.apply_lhat(tp, U, flat), tp


@pytest.mark.parametrize("sig", SIGMAS)
@pytest.mark.parametrize("dsig", DSIGMAS)
def test_fourth_order_difference_on_smooth_rows(sig, dsig):
    n = 33
    p = _problem(n, sig)
    S, dS = np.asarray(sig), np.asarray(dsig)
    if np.any((S[0] == 0.0) & (dS[0] != 0.0)):
        pytest.skip("moves an offset component that is exactly zero: a kink of the operator")
    X1, X2 = p.coords()
    U = np.sin(1.3 * X1 + 0.4) * np.cos(0.7 * X2 - 0.2) + 0.3 * X1 * X1
    i1, i2, flat = lisl.interior_flat(n)
    d = adj.dlhat_dtheta(p, 0, dS, U, i1, i2)
    eps = 1e-4
    vals, cols = [], []
    for k in (2, 1, -1, -2):
        v, tp = _lhat(p, S + k * eps * dS, U, i1, i2, flat)
        vals.append(v)
        cols.append(tp.cols)
    fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * eps)
    # rows whose taps keep their cells between -2 eps and +2 eps (the tap lists are stacked
    # endpoint by endpoint in the same order for every sigma)
    same = np.ones(len(i1), dtype=bool)
    R = len(i1)
    changed = cols[0] != cols[3]
    tp_rows = np.tile(np.arange(R), len(changed) // R)
    same[np.unique(tp_rows[changed])] = False
    assert same.sum() > 0.8 * R
    scale = float(np.max(np.abs(d[same])))
    assert np.max(np.abs(d[same] - fd[same])) <= 1e-7 * max(1.0, scale)
