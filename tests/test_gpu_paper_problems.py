"""The paper's test problems on the GPU (Section 2.4): Problem A (x-dependent diffusion
sigma = sqrt(2) (sin(x1 + x2), cos(x1 + x2)), drift control on the unit circle) and Problem B
(diffusion control sqrt(2) alpha), 40 controls, implicit scheme with stencil truncation,
one step Delta t = T = 1/2.

* The L-infinity errors at t = T reproduce Tables 2.4 and A.4 as printed (3 digits), with the
  same allowance as the oracle's own pins.
* The GPU solution equals the oracle's element by element (1e-10 FP64, 1e-8 mixed).
* Problem A runs the general fine level (per-row tables assembled for the policy): its
  argmin and its operators on every multigrid level are checked against the oracle.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import lisl, multigrid as mg
from tests._gpu_util import TOL_FP64, TOL_MIXED, policies_agree, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TABLES = {"A": ("table_2_4_problem_A.json", W.problem_A), "B": ("table_A_4_problem_B.json", W.problem_B)}
# printed with 3 digits; Problem B has exactly tied controls, so its digits also depend on the
# tie rule (see the oracle's pins); the 161 entry of Table A.4 is not a pin (reading 4)
ALLOW = {("A", 41): 0.006, ("A", 81): 0.006, ("A", 161): 0.006, ("B", 41): 0.006, ("B", 81): 0.015}


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("prob,n", [("A", 41), ("A", 81), ("A", 161), ("B", 41), ("B", 81), ("B", 161)])
def test_paper_tables_on_the_gpu(prob, n, precision):
    S = _lib()
    fname, make = TABLES[prob]
    gold = json.load(open(os.path.join(GOLD, fname)))
    p = make(n, n_alpha=gold["n_alpha"])
    ref = lisl.solve(p)
    sol = S.solver_from_problem(p, precision=precision, argmin_screen=precision)
    assert sol.general == (prob == "A")
    u = to_dev(p.g)
    sol.solve(u, 0.0, p.T, p.n_steps)
    U = u.cpu().numpy()
    assert rel_maxnorm(U, ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)
    if (prob, n) in ALLOW:
        err = np.max(np.abs(U - p.exact(p.T)))
        want = gold["error_linf"][str(n)]
        assert abs(err - want) <= ALLOW[(prob, n)] * want, (err, want)
    sol.close()


def test_general_argmin_matches_oracle():
    import torch
    S = _lib()
    p = W.problem_A(81)
    sol = S.solver_from_problem(p)
    rng = np.random.default_rng(4)
    X = p.exact(0.2).copy()
    X[1:-1, 1:-1] += 0.01 * rng.standard_normal((p.n - 2, p.n - 2))
    pol = torch.zeros((p.n - 2) ** 2, dtype=torch.uint8, device="cuda")
    sol.improve(to_dev(X), 0.2, pol)
    V = lisl.control_values(p, X, 0.2)
    ok, nd = policies_agree(pol.cpu().numpy(), lisl.improve(V), V)
    assert ok, nd
    sol.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_general_operators_on_every_level(precision):
    import torch
    S = _lib()
    p = W.problem_A(81)
    sol = S.solver_from_problem(p, precision=precision)
    dt = p.dt
    m = p.n - 2
    pol = (np.arange(m)[None, :] // 9 + np.arange(m)[:, None] // 13).ravel() % p.K
    sol.set_policy(to_dev(pol, torch.uint8))
    sol.build_hierarchy(dt)
    A, _ = lisl.assemble(p, pol, p.g, 0.0, dt)
    H = mg.galerkin_hierarchy(A, p.n, sol.num_levels())
    rng = np.random.default_rng(5)
    dtype = torch.float64 if precision == 0 else torch.float32
    tol = 1e-12 if precision == 0 else 2e-6
    for level in range(sol.num_levels()):
        nl = H.n[level]
        x = np.zeros((nl, nl))
        x[1:-1, 1:-1] = rng.standard_normal((nl - 2, nl - 2))
        y = torch.zeros((nl, nl), dtype=dtype, device="cuda")
        sol.apply(level, to_dev(x, dtype), y)
        ref = H.A[level] @ x[1:-1, 1:-1].ravel()
        got = y.double().cpu().numpy()[1:-1, 1:-1].ravel()
        assert rel_maxnorm(got, ref) <= tol, f"level {level}"
    sol.close()


def test_general_adjoint_gradient_in_g_matches_oracle():
    """The adjoint runs on the general fine level too (dJ/dg and dJ/dG; no sigma parameters)."""
    import torch
    from oracle import adjoint as adj
    S = _lib()
    p = W.problem_A(41, n_steps=2)
    w = W.gaussian_bump(p.n, p.lo, p.hi, seed=2)
    ref = adj.adjoint(p, w)
    sol = S.solver_from_problem(p)
    u = to_dev(p.g)
    sol.solve_record(u, 0.0, p.T, p.n_steps, 1)
    dg = torch.zeros_like(u)
    dG = torch.zeros_like(sol._G)
    sol.adjoint(to_dev(w), dg, dG)
    assert rel_maxnorm(dg.cpu().numpy(), ref.dJ_dg) <= 1e-9
    assert rel_maxnorm(dG.cpu().numpy(), ref.dJ_dG) <= 1e-9
    with pytest.raises(S.SLError):   # sigma parameters need the constant-per-control form
        sol.adjoint(to_dev(w), dg, None, np.zeros((1, p.K, 2, 1)))
    sol.close()
