"""Fourier-mode pin of the oracle (single control, periodic grid, no truncation).

Grid functions exp(i theta . j) are eigenfunctions of any constant-coefficient stencil
(Section 3.2).  Interpolating such a mode at the offset s of a diffusion direction gives the
factor G(s) = prod_d g(theta_d, gamma_d, m_d) with g(theta, gamma, m) =
gamma e^{i m theta} + (1 - gamma) e^{i (m+1) theta}, m = floor(|s_d|), gamma = m + 1 - |s_d|,
conjugated on components where s_d < 0 (the symbol of Section 3.2 and its oblique-direction
variant).  Hence L cos(theta . j) = lambda cos(theta . j) with
lambda = sum_p (Re G(s_p) - 1) / dx, and n implicit Euler steps scale the mode by
(1 - dt lambda)^{-n}.  The test evaluates this closed form with complex arithmetic of its own
and compares it with the oracle's real-space bilinear stencil.
"""
import cmath
import math

import numpy as np
import pytest

import workloads as W
from oracle import lisl


def g_sym(theta, s):
    m = math.floor(abs(s))
    gamma = m + 1 - abs(s)
    val = gamma * cmath.exp(1j * m * theta) + (1 - gamma) * cmath.exp(1j * (m + 1) * theta)
    return val.conjugate() if s < 0 else val


@pytest.mark.parametrize("sig", [
    [[0.7, -0.4], [0.9, 1.1]],
    [[0.5, 0.0], [0.0, 0.8]],
    [[0.6, 0.3], [-0.45, 0.2]],
])
@pytest.mark.parametrize("kmode", [(1, 0), (2, 3), (5, -7), (11, 4)])
def test_periodic_mode_decay(sig, kmode):
    n = 32
    h = 0.01
    p = W.Problem(name="per", n=n, lo=0.0, hi=(n - 1) * h, T=1.0, n_steps=1,
                  sigma=np.asarray(sig, dtype=np.float64)[None], phi=None, G=None,
                  tau_kind=None, tau_rate=None, g=np.zeros((n, n)),
                  psi_fn=lambda t: np.zeros((n, n)))
    th = (2 * math.pi * kmode[0] / n, 2 * math.pi * kmode[1] / n)
    S = np.asarray(sig)
    lam = 0.0
    for col in range(S.shape[1]):
        s = S[:, col] / math.sqrt(h)
        G = g_sym(th[0], s[0]) * g_sym(th[1], s[1])
        lam += (G.real - 1.0) / h
    i2, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mode = np.cos(th[0] * i1 + th[1] * i2)
    dt, steps = 0.002, 5
    M = lisl.periodic_step_matrix(p, 0, dt)
    x = mode.ravel().copy()
    for _ in range(steps):
        x = lisl.direct_solve(M, x)
    expect = (1.0 - dt * lam) ** (-steps) * mode.ravel()
    assert np.max(np.abs(x - expect)) <= 1e-12
    # the eigenvalue itself
    V = lisl.control_values(p, mode, 0.0, f_full=np.zeros((1, n, n)), periodic=True)[0]
    assert np.max(np.abs(V - lam * mode.ravel())) <= 1e-9 * max(1.0, abs(lam))
