"""Pins of the oracle's multigrid pieces.

* Bilinear prolongation equals SciPy's piecewise-linear interpolation of the coarse data.
* Full weighting equals the textbook 9-point stencil (1/16)[1 2 1; 2 4 2; 1 2 1].
* The V-cycle with damped Jacobi (omega = 0.8, two pre- and two post-sweeps) on the 5-point
  Laplacian, which is the LISL stencil with grid-aligned unit offsets, contracts the error
  by a mesh-independent factor below 0.2 (local Fourier analysis: smoothing factor 0.6 per
  sweep, 0.6^4 = 0.13 for four sweeps).
* A one-level hierarchy is a direct solve; a two-level cycle without smoothing is exactly the
  coarse-grid correction P A_c^{-1} R.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.interpolate import RegularGridInterpolator

import workloads as W
from oracle import lisl, multigrid as mg


def test_prolongation_is_bilinear_interpolation():
    nc = 9
    nf = 2 * nc - 1
    rng = np.random.default_rng(0)
    vc = np.zeros((nc, nc))
    vc[1:-1, 1:-1] = rng.normal(size=(nc - 2, nc - 2))
    xc = np.linspace(0, 1, nc)
    xf = np.linspace(0, 1, nf)
    interp = RegularGridInterpolator((xc, xc), vc, method="linear")
    Y2, Y1 = np.meshgrid(xf, xf, indexing="ij")
    ref = interp(np.stack([Y2.ravel(), Y1.ravel()], axis=1)).reshape(nf, nf)
    got = (mg.prolongation(nc) @ vc[1:-1, 1:-1].ravel()).reshape(nf - 2, nf - 2)
    assert np.max(np.abs(got - ref[1:-1, 1:-1])) <= 1e-14


def test_full_weighting_stencil():
    nc = 9
    nf = 2 * nc - 1
    rng = np.random.default_rng(1)
    vf = np.zeros((nf, nf))
    vf[1:-1, 1:-1] = rng.normal(size=(nf - 2, nf - 2))
    w = {-1: 0.25, 0: 0.5, 1: 0.25}
    ref = np.zeros((nc - 2, nc - 2))
    for I2 in range(1, nc - 1):
        for I1 in range(1, nc - 1):
            ref[I2 - 1, I1 - 1] = sum(w[a] * w[b] * vf[2 * I2 + a, 2 * I1 + b]
                                      for a in (-1, 0, 1) for b in (-1, 0, 1))
    got = (mg.restriction(nc) @ vf[1:-1, 1:-1].ravel()).reshape(nc - 2, nc - 2)
    assert np.max(np.abs(got - ref)) <= 1e-15


def _five_point(n):
    h = 1.0 / (n - 1)
    p = W.Problem(name="fp", n=n, lo=0.0, hi=1.0, T=1.0, n_steps=1,
                  sigma=np.array([[[math.sqrt(h), 0.0], [0.0, math.sqrt(h)]]]), phi=None,
                  G=None, tau_kind=None, tau_rate=None, g=np.zeros((n, n)),
                  psi_fn=lambda t: np.zeros((n, n)))
    i1, i2, flat = lisl.interior_flat(n)
    tp = lisl.control_taps(p, 0, i1, i2)
    unk = -np.ones(n * n, dtype=np.int64)
    unk[flat] = np.arange(len(flat))
    cu = unk[tp.cols]
    m = cu >= 0
    N = len(flat)
    L = sp.csr_matrix((tp.w[m], (tp.rows[m], cu[m])), shape=(N, N)) - sp.diags(tp.W)
    A = (-L).tocsr()
    A.eliminate_zeros()
    return A


def test_lisl_unit_offsets_is_five_point_laplacian():
    n = 17
    A = _five_point(n)
    h = 1.0 / (n - 1)
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n - 2, n - 2))
    I = sp.identity(n - 2)
    ref = (sp.kron(I, T) + sp.kron(T, I)) / (2 * h)
    assert abs(A - ref).max() <= 1e-12 / h


def test_vcycle_contraction_is_mesh_independent():
    rates = []
    for l in (5, 6, 7):
        n = 2 ** l + 1
        A = _five_point(n)
        H = mg.galerkin_hierarchy(A, n, l - 1)
        rng = np.random.default_rng(l)
        x = rng.normal(size=A.shape[0])
        b = np.zeros_like(x)
        e0 = np.linalg.norm(x)
        for _ in range(8):
            x = x + mg.vcycle(H, b - A @ x, 2, 2, 0.8)
        rates.append((np.linalg.norm(x) / e0) ** (1 / 8))
    assert max(rates) < 0.2, rates
    assert max(rates) - min(rates) < 0.05, rates


def test_vcycle_limits():
    n = 17
    A = _five_point(n) + sp.identity((n - 2) ** 2)
    rng = np.random.default_rng(3)
    b = rng.normal(size=A.shape[0])
    H1 = mg.galerkin_hierarchy(A, n, 1)
    assert np.allclose(mg.vcycle(H1, b), np.linalg.solve(A.toarray(), b), atol=1e-13)
    H2 = mg.galerkin_hierarchy(A, n, 2)
    cgc = H2.P[0] @ np.linalg.solve(H2.A[1].toarray(), H2.R[0] @ b)
    assert np.allclose(mg.vcycle(H2, b, 0, 0), cgc, atol=1e-13)
