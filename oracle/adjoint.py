"""Dense-transpose adjoint of the implicit Howard solve (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each step n defines U^n through the residual of the converged policy alpha_n (the policy of the
step's last linear solve):
    G_n(U^n, U^{n-1}; theta) = A^{alpha_n} U^n - F^{alpha_n} = U^n - U^{n-1} - dt (L U^n_ext + c U^n + f_n),
(Eq. 2.11 with theta = 1, boundary terms inside L U_ext).  For J = sum_x w(x) U^N(x), away
from policy switches (where alpha_n does not move under small perturbations) the Lagrangian
J - sum_n mu_n^T G_n gives the backward recursion
    A_N^T mu_N = w,   A_n^T mu_n = mu_{n+1}   (dG_{n+1}/dU^n = -I),
and the gradients
    dJ/dg           = mu_1,
    dJ/dG[m][q](x)  = sum_n dt tau_q(t_n) phi[alpha_n(x), m] mu_n(x)     (source tables),
    dJ/dtheta       = -sum_n mu_n^T dG_n/dtheta = sum_n dt mu_n^T (dL_n/dtheta U^n_ext)
for a scalar theta of the diffusion coefficients (d sigma / d theta given).  dL/dtheta U is
taken here as a central difference of this oracle's own control values in theta: inside one
interpolation cell the bilinear weights are linear in sigma, so the difference is exact up to
rounding wherever no tap crosses a cell edge within +-eps (truncated rows add an O(eps^2) term).
"""
from __future__ import annotations

import copy
import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse.linalg as spla

from . import lisl


@dataclasses.dataclass
class AdjointResult:
    U: np.ndarray                  # U^N (full grid)
    dJ_dg: np.ndarray              # full grid, zero on the boundary
    dJ_dG: Optional[np.ndarray]    # (nf, nq, n, n) or None
    dJ_dtheta: np.ndarray          # (nparam,)
    policies: List[np.ndarray]


def _perturbed(prob, dsigma, eps):
    p = copy.copy(prob)
    p.sigma = prob.sigma + eps * dsigma
    return p


def adjoint(prob, w: np.ndarray, dsigma: Sequence[np.ndarray] = (), n_steps: Optional[int] = None,
            T: Optional[float] = None, eps_rel: float = 1e-6) -> AdjointResult:
    n_steps = prob.n_steps if n_steps is None else n_steps
    T = prob.T if T is None else T
    dt = T / n_steps
    n = prob.n
    _, _, flat = lisl.interior_flat(n)
    # forward, recording U^n and the policy of each step's last solve
    Us = [prob.g.copy()]
    pols = []
    policy = None
    for s in range(1, n_steps + 1):
        r = lisl.howard_step(prob, Us[-1], s * dt, dt, policy0=policy)
        Us.append(r.X)
        pols.append(r.solve_policy)
        policy = r.policy
    lam = w.ravel()[flat].copy()
    dtheta = np.zeros(len(dsigma))
    dG = None if prob.G is None else np.zeros_like(prob.G)
    for s in range(n_steps, 0, -1):
        t = s * dt
        A, _ = lisl.assemble(prob, pols[s - 1], Us[s - 1], t, dt)
        mu = spla.spsolve(A.T.tocsc(), lam)
        U_ext = Us[s]
        for p, ds in enumerate(dsigma):
            eps = eps_rel * max(1.0, float(np.max(np.abs(prob.sigma))))
            vp = lisl.control_values(_perturbed(prob, ds, +eps), U_ext, t)
            vm = lisl.control_values(_perturbed(prob, ds, -eps), U_ext, t)
            idx = pols[s - 1]
            dL = (vp[idx, np.arange(len(idx))] - vm[idx, np.arange(len(idx))]) / (2 * eps)
            dtheta[p] += dt * float(mu @ dL)
        if dG is not None:
            tau = prob.tau(t)
            phi_a = prob.phi[pols[s - 1]]          # (N, nf)
            for m in range(prob.G.shape[0]):
                for q in range(prob.G.shape[1]):
                    dG[m, q].ravel()[flat] += dt * tau[q] * phi_a[:, m] * mu
        lam = mu
    dg = np.zeros((n, n))
    dg.ravel()[flat] = lam
    return AdjointResult(Us[-1], dg, dG, dtheta, pols)


def objective(prob, w: np.ndarray, n_steps: Optional[int] = None, T: Optional[float] = None):
    """J = sum_x w(x) U^N(x) from a full forward solve, and the per-step final policies."""
    r = lisl.solve(prob, n_steps=n_steps, T=T)
    return float(np.sum(w * r.U)), r.policies
