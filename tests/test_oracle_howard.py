"""Pins of the oracle's Howard policy iteration.

* Brute force: on a 5 x 5 grid (9 unknowns) with 3 controls and truncation-heavy diffusion,
  the discrete HJB solution is the componentwise minimum over all 3^9 policies of
  (A^alpha)^{-1} F^alpha (the system matrices are inverse-positive M-matrices with row-wise
  independent controls), and Howard's iteration must reach it.
* Monotonicity of Howard's iterates: X^{m+1} <= X^m componentwise.
* At convergence max_k (A^k X - F^k) = 0 row by row (Eq. 1.10).
"""
import itertools

import numpy as np

import workloads as W
from oracle import lisl


def _tiny_problem():
    p = W.manufactured(5, 3, -0.7, 0.9, 1.3, 1.1, T=0.5, n_steps=1)
    return p


def test_brute_force_policy_enumeration():
    p = _tiny_problem()
    dt = 0.5
    U = p.g.copy()
    rng = np.random.default_rng(2)
    U[1:-1, 1:-1] += rng.uniform(-0.3, 0.3, size=(3, 3))
    N = 9
    best = np.full(N, np.inf)
    for pol in itertools.product(range(p.K), repeat=N):
        A, F = lisl.assemble(p, np.array(pol), U, dt, dt)
        X = np.linalg.solve(A.toarray(), F)
        best = np.minimum(best, X)
    res = lisl.howard_step(p, U, dt, dt, policy0=np.zeros(N, dtype=np.int64))
    X = res.X[1:-1, 1:-1].ravel()
    assert res.converged
    assert np.max(np.abs(X - best)) <= 1e-13 * max(1.0, np.abs(best).max())
    # and the minimum is attained by the final policy
    A, F = lisl.assemble(p, res.policy, U, dt, dt)
    assert np.max(np.abs(np.linalg.solve(A.toarray(), F) - best)) <= 1e-13


def test_howard_iterates_decrease_and_residual_vanishes():
    p = W.oracle_scale(True)
    dt = p.dt
    res = lisl.howard_step(p, p.g, dt, dt, policy0=np.zeros((p.n - 2) ** 2, dtype=np.int64),
                           keep_iterates=True)
    assert res.converged and res.pi_iters >= 2
    for a, b in zip(res.iterates, res.iterates[1:]):
        assert np.all(b <= a + 1e-13)
    r = lisl.hjb_residual(p, res.X, p.g, dt, dt)
    assert np.max(np.abs(r)) <= 1e-12


def test_improvement_tie_break_lowest_index():
    # rows are controls, columns are nodes
    V = np.array([[1.0 + 5e-13, 2.0, 0.5 + 1e-9, -7.0 + 6e-12],
                  [1.0, 1.0, 0.5, -7.0],
                  [3.0, 1.0 - 1e-15, 0.5, -7.0 - 1e-11]])
    pol = lisl.improve(V)
    assert list(pol) == [0, 1, 1, 2]
