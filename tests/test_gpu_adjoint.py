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
    against central differences of the library's own FP64 forward march at 1e-6 relative.
    The perturbed marches must take the base march's policy and Howard count at every step,
    so that the differences stay on the piece of the piecewise-smooth map whose gradient the
    adjoint gives: the step of each difference is the largest of a short decreasing list for
    which that holds.  The marches solve to 1e-14 so that the differences resolve 1e-6."""
    import torch
    S = _lib()
    p, w = W.adjoint_1025(seed=0)
    dirs = W.sigma_directions(p)
    tol = 1e-14
    sol = S.solver_from_problem(p, precision=0, krylov_tol=tol)
    u = to_dev(p.g)
    sol.solve_record(u, 0.0, p.T, p.n_steps, 8)
    wd = to_dev(w)
    dg = torch.zeros_like(u)
    dth, _ = sol.adjoint(wd, dg, None, dirs)
    sol.close()
    m = p.n - 2
    dt = p.T / p.n_steps

    def march(sigma=None, g=None):
        q = copy.copy(p)
        if sigma is not None:
            q.sigma = sigma
        s = S.solver_from_problem(q, precision=0, krylov_tol=tol)
        uu = to_dev(p.g if g is None else g)
        pols = torch.empty((p.n_steps, m * m), dtype=torch.uint8, device=uu.device)
        its = []
        for i in range(1, p.n_steps + 1):
            st = s.step(uu, i * dt, dt, policy_out=pols[i - 1])
            its.append(st["pi_iters"])
        s.close()
        return float((wd * uu).sum()), pols, its

    _, pol0, it0 = march()

    def central(make, steps):
        for eps in steps:
            Jp, pp, ip = march(**make(eps))
            Jm, pm, im = march(**make(-eps))
            if torch.equal(pp, pol0) and torch.equal(pm, pol0) and ip == it0 and im == it0:
                return (Jp - Jm) / (2 * eps), eps
        pytest.fail("every step of the list switched a policy")

    d = w  # a coherent direction: the bump itself
    fd_g, eps_g = central(lambda e: {"g": p.g + e * d}, (1e-5, 2e-6, 5e-7))
    ad_g = float((dg.cpu().numpy() * d).sum())
    assert abs(fd_g - ad_g) <= 1e-6 * abs(fd_g), (fd_g, ad_g, eps_g)
    for i, ds in enumerate(dirs):
        fd, eps = central(lambda e: {"sigma": p.sigma + e * ds}, (2e-5, 5e-6, 1e-6))
        assert abs(fd - dth[i]) <= 1e-6 * abs(fd), (i, fd, dth[i], eps)
