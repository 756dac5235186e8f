"""Pins of the oracle's discrete adjoint (oracle/adjoint.py).

* Single control (K = 1): the march is linear in g and affine in the source tables G, so
  J(g + dg) - J(g) = <dJ/dg, dg> and J(G + dG) - J(G) = <dJ/dG, dG> hold exactly (up to
  rounding) for any perturbation, however large.  These identities fix the transposed
  recursion, its time indexing and the source factors dt tau_q(t_n) phi.
* Several controls: central finite differences of the full forward solve (direct solves,
  Howard to convergence) in g, in G and in scalar parameters of sigma, at perturbations
  small enough that no step's policy changes (checked).  The sigma directions cover the
  truncated rows (large offsets) and a non-zero Dirichlet boundary, whose values enter
  dL/dtheta U through the taps that reach the boundary.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj
from oracle import lisl


def _weights(n, seed):
    rng = np.random.default_rng(seed)
    w = np.zeros((n, n))
    w[1:-1, 1:-1] = rng.uniform(0.0, 1.0, (n - 2, n - 2))
    return w


def _J(p, w, **kw):
    return adj.objective(p, w, **kw)


def test_single_control_linear_in_g():
    p = W.with_dirichlet(W.manufactured(17, 1, 0.4, 0.4, 0.9, 0.7, T=0.25, n_steps=5))
    w = _weights(17, 1)
    r = adj.adjoint(p, w)
    rng = np.random.default_rng(3)
    dg = rng.normal(size=(17, 17))
    q = copy.copy(p)
    q.g = p.g + dg
    J0, _ = _J(p, w)
    J1, _ = _J(q, w)
    lhs, rhs = J1 - J0, float(np.sum(r.dJ_dg * dg))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(J0))
    # g's boundary values never enter the march
    assert np.all(r.dJ_dg[0, :] == 0) and np.all(r.dJ_dg[:, -1] == 0)


def test_single_control_affine_in_source_tables():
    p = W.manufactured(17, 1, -0.3, -0.3, 1.1, 0.6, T=0.3, n_steps=4)
    w = _weights(17, 2)
    r = adj.adjoint(p, w)
    rng = np.random.default_rng(4)
    dG = rng.normal(size=p.G.shape)
    q = copy.copy(p)
    q.G = p.G + dG
    J0, _ = _J(p, w)
    J1, _ = _J(q, w)
    assert abs((J1 - J0) - float(np.sum(r.dJ_dG * dG))) <= 1e-12 * max(1.0, abs(J0))


@pytest.mark.parametrize("s1,s2,bnd", [(0.9, 0.7, False), (1.3, 1.1, True)])
def test_sigma_gradient_matches_central_differences(s1, s2, bnd):
    p = W.manufactured(17, 5, -0.6, 0.6, s1, s2, T=0.25, n_steps=4)
    if bnd:
        p = W.with_dirichlet(p)
    w = _weights(17, 5)
    dirs = list(W.sigma_directions(p))
    r = adj.adjoint(p, w, dirs)
    eps = 1e-5
    for i, ds in enumerate(dirs):
        pp, pm = copy.copy(p), copy.copy(p)
        pp.sigma = p.sigma + eps * ds
        pm.sigma = p.sigma - eps * ds
        Jp, polp = _J(pp, w)
        Jm, polm = _J(pm, w)
        assert all(np.array_equal(a, b) for a, b in zip(polp, polm)), "policy switched: move eps"
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - r.dJ_dtheta[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, r.dJ_dtheta[i])


def test_g_and_source_gradients_match_central_differences_with_several_controls():
    p = W.manufactured(17, 5, -0.6, 0.6, 0.9, 0.7, T=0.25, n_steps=4)
    w = _weights(17, 6)
    r = adj.adjoint(p, w)
    rng = np.random.default_rng(7)
    dg = np.zeros((17, 17))
    dg[1:-1, 1:-1] = rng.normal(size=(15, 15))
    dG = rng.normal(size=p.G.shape)
    eps = 1e-6
    for name, pert, grad in (("g", dg, r.dJ_dg), ("G", dG, r.dJ_dG)):
        pp, pm = copy.copy(p), copy.copy(p)
        if name == "g":
            pp.g, pm.g = p.g + eps * pert, p.g - eps * pert
        else:
            pp.G, pm.G = p.G + eps * pert, p.G - eps * pert
        Jp, polp = _J(pp, w)
        Jm, polm = _J(pm, w)
        assert all(np.array_equal(a, b) for a, b in zip(polp, polm))
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - float(np.sum(grad * pert))) <= 1e-7 * max(1.0, abs(fd)), name


def test_policies_recorded_are_those_of_the_final_solves():
    p = W.manufactured(17, 5, -0.6, 0.6, 0.9, 0.7, T=0.25, n_steps=4)
    w = _weights(17, 8)
    r = adj.adjoint(p, w)
    # re-solving each step at its recorded policy reproduces the march
    U = p.g.copy()
    dt = p.T / p.n_steps
    for s, pol in enumerate(r.policies, start=1):
        A, F = lisl.assemble(p, pol, U, s * dt, dt)
        X = np.linalg.solve(A.toarray(), F)
        U2 = U.copy()
        U2[1:-1, 1:-1] = np.asarray(X).reshape(15, 15)
        U2[0, :], U2[-1, :], U2[:, 0], U2[:, -1] = 0.0, 0.0, 0.0, 0.0
        U = U2
    assert np.max(np.abs(U - r.U)) <= 1e-12
