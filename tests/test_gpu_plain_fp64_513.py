"""The plain FP64 GPU workload against the oracle's full march: 513 x 513 grid, 33 controls
rho in [-0.9, 0.9], s1 = 0.3, s2 = 0.2, T = 1, 64 implicit steps, Howard iteration with
BiCGSTAB preconditioned by an 8-level V(2,2) damped-Jacobi (omega = 0.8) V-cycle, FP64.

The oracle's march (sparse direct solve per Howard iteration, about 60 s per factorisation
here) is stored in tests/golden/plain_fp64_513.npz by tests/golden/make_plain_fp64_513.py,
which calls only the oracle.  Checks, element by element: U after step 1 and at t = T to 1e-10
relative max-norm; the policies after step 1 and at T equal up to near-ties within 1e-12
(decided with the oracle's control values at the nodes where they differ); the Howard
iteration count of every step (with the oracle's Howard iteration: sl_opts.howard_init = 0
and howard_loose_tol = 0).
At 513^2 the stencil offsets reach 3.4-3.8 cells, so the truncation band of Section 2.1 is
exercised along the whole boundary.  A second march with howard_init = 1 (each step's policy
first improved at its extrapolated first iterate) must reach the same U(T) and policy, in no
more Howard iterations in total.  The default loose first solve (howard_loose_tol) is covered
by the marches of the device-step tests.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import lisl
from tests._gpu_util import TIE, TOL_FP64, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "plain_fp64_513.npz")


def _policies_agree_at(p, X_full, t, p_gpu, p_orc):
    """Equal policies except at near-ties of the oracle's control values at X_full."""
    diff = np.nonzero(p_gpu != p_orc)[0]
    if len(diff) == 0:
        return True, 0
    m = p.n - 2
    i1 = (diff % m + 1).astype(np.float64)
    i2 = (diff // m + 1).astype(np.float64)
    V = lisl.control_values_at(p, X_full, t, i1, i2)
    cols = np.arange(len(diff))
    vg = V[p_gpu[diff], cols]
    vo = V[p_orc[diff], cols]
    ok = np.abs(vg - vo) <= 2 * TIE * np.maximum(1.0, np.abs(vo))
    return bool(np.all(ok)), len(diff)


def test_plain_fp64_513_matches_the_oracle_march():
    if not os.path.exists(GOLD):
        pytest.skip("tests/golden/plain_fp64_513.npz not generated")
    import paper_1605_04821_gb300 as S
    S.load()
    gold = np.load(GOLD)
    p = W.plain_fp64()
    # the oracle's Howard iteration: each step starts from the previous step's policy and every
    # linear solve is tight, so that the Howard counts can be compared step by step
    sol = S.solver_from_problem(p, precision=0, nu1=2, nu2=2, omega=0.8, howard_init=0,
                                howard_loose_tol=0.0)
    assert sol.num_levels() == 8
    u = to_dev(p.g)
    m = p.n - 2
    pol = torch.empty(m * m, dtype=torch.uint8, device="cuda")
    dt = p.T / p.n_steps
    pis = []
    for i in range(1, p.n_steps + 1):
        st = sol.step(u, i * dt, dt, policy_out=pol)
        pis.append(st["pi_iters"])
        if i == 1:
            U1 = u.cpu().numpy()
            assert rel_maxnorm(U1, gold["U_1"]) <= TOL_FP64
            ok, nd = _policies_agree_at(p, gold["U_1"], dt, pol.cpu().numpy().astype(np.int64),
                                        gold["policy_1"].astype(np.int64))
            assert ok, f"step 1: {nd} policy entries differ beyond the tie window"
    sol.close()
    U = u.cpu().numpy()
    err = rel_maxnorm(U, gold["U_T"])
    assert err <= TOL_FP64, err
    ok, nd = _policies_agree_at(p, gold["U_T"], p.T, pol.cpu().numpy().astype(np.int64),
                                gold["policy_T"].astype(np.int64))
    assert ok, f"t = T: {nd} policy entries differ beyond the tie window"
    assert pis == [int(x) for x in gold["pi_iters"]]


def test_plain_fp64_513_predictor_start_reaches_the_same_march():
    if not os.path.exists(GOLD):
        pytest.skip("tests/golden/plain_fp64_513.npz not generated")
    import paper_1605_04821_gb300 as S
    S.load()
    gold = np.load(GOLD)
    p = W.plain_fp64()
    sol = S.solver_from_problem(p, precision=0, nu1=2, nu2=2, omega=0.8, howard_init=1,
                                howard_loose_tol=0.0)
    u = to_dev(p.g)
    m = p.n - 2
    pol = torch.empty(m * m, dtype=torch.uint8, device="cuda")
    st = sol.solve(u, 0.0, p.T, p.n_steps, policy_out=pol)
    sol.close()
    assert rel_maxnorm(u.cpu().numpy(), gold["U_T"]) <= TOL_FP64
    ok, nd = _policies_agree_at(p, gold["U_T"], p.T, pol.cpu().numpy().astype(np.int64),
                                gold["policy_T"].astype(np.int64))
    assert ok, f"t = T: {nd} policy entries differ beyond the tie window"
    assert st["pi_iters"] <= int(gold["pi_iters"].sum())
