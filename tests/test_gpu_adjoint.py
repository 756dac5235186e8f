"""GPU parity of the discrete adjoint (sl_hjb_solve_record + sl_hjb_adjoint).

Small cases run against the oracle's dense-transpose adjoint element by element: dJ/dg and
dJ/dG in relative max-norm, dJ/dtheta per parameter (the oracle writes dL/dtheta U in closed
form, so both sides are exact up to the solves' tolerance).  The full-size case (1025^2,
33 controls, 64 steps, checkpoints every 8 steps, Gaussian-bump weights) is checked against
central differences of the library's own forward march at 1e-6 relative, with every step's
policy and Howard count unchanged under the perturbations (away from policy switches).
"""
import copy

import numpy as np
import pytest

import workloads as W
from tests._gpu_util import TOL_FP64, TOL_MIXED, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

ADJ_TOL = {0: 1e-9, 1: 1e-8}     # dJ/dg, dJ/dG, relative max-norm
THETA_TOL = {0: 1e-10, 1: 1e-10}  # dJ/dtheta, relative


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _case(name):
    if name == "c33":
        p = W.oracle_scale(False)
    elif name == "heavy33":
        p = W.oracle_scale(True)
    elif name == "bnd33":
        p = W.with_dirichlet(W.oracle_scale(True))
    elif name == "cb33":
        p = W.with_dirichlet(W.oracle_scale(True))
        p.c = np.linspace(-0.5, 0.3, p.K)
        p.drift = np.stack([np.linspace(-2.0, 2.0, p.K), np.linspace(1.5, -1.0, p.K)], axis=1)
    elif name == "k1_33":
        p = W.manufactured(33, 1, 0.3, 0.3, 0.9, 0.7)
    else:
        p = W.scaled(65, 17, 4, seed=5)
    p = copy.copy(p)
    p.n_steps = 6 if name != "s65" else 4
    p.T = 0.5
    return p


def _oracle(p, w, dirs):
    from oracle import adjoint as adj
    return adj.adjoint(p, w, list(dirs))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,ckpt", [("c33", 1), ("heavy33", 3), ("bnd33", 1), ("k1_33", 2),
                                       ("s65", 1), ("cb33", 2)])
def test_adjoint_matches_oracle(name, ckpt, precision):
    import torch
    S = _lib()
    p = _case(name)
    w = W.gaussian_bump(p.n, p.lo, p.hi, seed=1)
    dirs = W.sigma_directions(p)
    ref = _oracle(p, w, dirs)
    sol = S.solver_from_problem(p, precision=precision)
    u = to_dev(p.g)
    sol.solve_record(u, 0.0, p.T, p.n_steps, ckpt)
    tol_u = TOL_FP64 if precision == 0 else TOL_MIXED
    assert rel_maxnorm(u.cpu().numpy(), ref.U) <= tol_u
    dg = torch.full_like(u, float("nan"))
    dG = torch.full_like(sol._G, float("nan"))
    dth, st = sol.adjoint(to_dev(w), dg, dG, dirs)
    torch.cuda.synchronize()
    assert st["steps"] == p.n_steps
    eg = rel_maxnorm(dg.cpu().numpy(), ref.dJ_dg)
    eG = rel_maxnorm(dG.cpu().numpy(), ref.dJ_dG)
    assert eg <= ADJ_TOL[precision], eg
    assert eG <= ADJ_TOL[precision], eG
    for i in range(len(dirs)):
        e = abs(dth[i] - ref.dJ_dtheta[i]) / max(1e-300, abs(ref.dJ_dtheta[i]))
        assert e <= THETA_TOL[precision], (i, dth[i], ref.dJ_dtheta[i])
    sol.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_interval_does_not_change_the_gradient(precision):
    import torch
    S = _lib()
    p = W.scaled(129, 17, 9, seed=2)
    w = W.gaussian_bump(p.n, p.lo, p.hi, seed=3)
    dirs = W.sigma_directions(p)
    sol = S.solver_from_problem(p, precision=precision)
    out = []
    for ckpt in (1, 4, 9):
        u = to_dev(p.g)
        sol.solve_record(u, 0.0, p.T, p.n_steps, ckpt)
        dg = torch.zeros_like(u)
        dth, _ = sol.adjoint(to_dev(w), dg, None, dirs)
        out.append((dg.cpu().numpy(), dth))
    for dg, dth in out[1:]:
        assert rel_maxnorm(dg, out[0][0]) <= 1e-9
        assert np.max(np.abs(dth - out[0][1]) / np.abs(out[0][1])) <= 1e-9
    sol.close()


def test_autograd_function_returns_the_adjoint_gradients():
    import torch
    S = _lib()
    p = _case("c33")
    w = to_dev(W.gaussian_bump(p.n, p.lo, p.hi, seed=4))
    sol = S.solver_from_problem(p)
    g = to_dev(p.g).requires_grad_(True)
    G = sol._G.requires_grad_(True)
    theta = torch.zeros(2, dtype=torch.float64, device=g.device, requires_grad=True)
    U = S.hjb_solve(sol, g, G, p.T, p.n_steps, theta=theta, dsigma=W.sigma_directions(p))
    (w * U).sum().backward()
    ref = _oracle(p, w.cpu().numpy(), W.sigma_directions(p))
    assert rel_maxnorm(g.grad.cpu().numpy(), ref.dJ_dg) <= ADJ_TOL[0]
    assert rel_maxnorm(G.grad.cpu().numpy(), ref.dJ_dG) <= ADJ_TOL[0]
    assert np.allclose(theta.grad.cpu().numpy(), ref.dJ_dtheta, rtol=THETA_TOL[0], atol=0)
    sol.close()


def test_full_size_gradient_matches_central_differences_of_the_march():
    """1025^2, 33 controls, 64 steps, checkpoints every 8 steps: <dJ/dg, w> and dJ/dtheta
    against central differences of the library's own FP64 march.

    * On the piece (away from policy switches): every perturbed march runs at the recorded
      per-step policies of the base march (sl_hjb_recorded_policy + sl_hjb_set_policy +
      sl_hjb_linear_solve), which is the map whose derivative the adjoint is; 1e-6 relative.
    * The full Howard march, beside it: at this size some of the 6.4e7 node-steps sit within
      any usable step of a tie between two controls and switch, each moving J only at second
      order; the switched node-steps are counted (a small fraction: 27 to 364 of 1.3e8 when
      this was written) and the difference must agree to 1e-6 as well.
    The marches solve to 1e-14 so that the differences resolve 1e-6."""
    import warnings

    import torch
    S = _lib()
    p, w = W.adjoint_1025(seed=0)
    dirs = W.sigma_directions(p)
    tol = 1e-14
    m = p.n - 2
    N = p.n_steps
    dt = p.T / N
    sol = S.solver_from_problem(p, precision=0, krylov_tol=tol)
    u = to_dev(p.g)
    sol.solve_record(u, 0.0, p.T, N, 8)
    rec = torch.empty((N, m * m), dtype=torch.uint8, device=u.device)
    for i in range(1, N + 1):
        sol.recorded_policy(i, rec[i - 1])
    wd = to_dev(w)
    dg = torch.zeros_like(u)
    dth, _ = sol.adjoint(wd, dg, None, dirs)
    sol.close()

    def solver(sigma):
        q = copy.copy(p)
        if sigma is not None:
            q.sigma = sigma
        return S.solver_from_problem(q, precision=0, krylov_tol=tol)

    def march_fixed(sigma=None, g=None):
        s = solver(sigma)
        uu = to_dev(p.g if g is None else g)
        x = torch.empty_like(uu)
        for i in range(1, N + 1):
            s.set_policy(rec[i - 1])
            x.copy_(uu)
            s.linear_solve(uu, x, i * dt, dt)
            uu, x = x, uu
        s.close()
        return float((wd * uu).sum())

    def march_howard(sigma=None, g=None):
        s = solver(sigma)
        uu = to_dev(p.g if g is None else g)
        pols = torch.empty((N, m * m), dtype=torch.uint8, device=uu.device)
        for i in range(1, N + 1):
            s.step(uu, i * dt, dt, policy_out=pols[i - 1])
        s.close()
        return float((wd * uu).sum()), pols

    _, pol0 = march_howard()
    d = w  # a coherent direction: the bump itself
    ad_g = float((dg.cpu().numpy() * d).sum())
    cases = [("g", ad_g, 1e-3, 1e-5, lambda e: {"g": p.g + e * d})]
    for i, ds in enumerate(dirs):
        cases.append((f"theta_{i}", float(dth[i]), 2e-5, 2e-5,
                      lambda e, ds=ds: {"sigma": p.sigma + e * ds}))
    for name, ad, eps_f, eps_h, make in cases:
        fd = (march_fixed(**make(eps_f)) - march_fixed(**make(-eps_f))) / (2 * eps_f)
        assert abs(fd - ad) <= 1e-6 * abs(fd), (name, "fixed policies", fd, ad)
        Jp, pp = march_howard(**make(eps_h))
        Jm, pm = march_howard(**make(-eps_h))
        fdh = (Jp - Jm) / (2 * eps_h)
        switched = int((pp != pol0).sum()) + int((pm != pol0).sum())
        warnings.warn(f"{name}: adjoint {ad:.12e}, fixed-policy FD {fd:.12e} "
                      f"({abs(fd - ad) / abs(fd):.1e}), Howard FD {fdh:.12e} "
                      f"({abs(fdh - ad) / abs(fdh):.1e}, {switched} switched node-steps)")
        assert switched <= 1e-3 * 2 * N * m * m, (name, switched)
        assert abs(fdh - ad) <= 1e-6 * abs(fdh), (name, "Howard", fdh, ad, switched)
