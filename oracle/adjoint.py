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
for a scalar theta of the diffusion coefficients (d sigma / d theta given).

dL/dtheta U is written out in closed form from the truncated scheme (Eq. 2.1, Proposition 2.2),
row by row, for the piece of its piecewise-smooth dependence on sigma that the data lie in:
    (L U)_j = sum_p [A_p (I U)(z+_p) - (A_p + B_p) U_j + B_p (I U)(z-_p)] / (2 dx),
    z+-_p = x_j + mu+-_p (+-sqrt(dx) sigma_p)   (index units: s_p = sigma_p / sqrt(dx)),
    A_p = 2 / (mu+^2 + mu+ mu-),  B_p = 2 / (mu-^2 + mu- mu+)                      (Eq. 2.3),
so with ds = d sigma_p / d theta / sqrt(dx):
  * mu = 1 (no truncation): d mu = 0 and dz = +-ds;
  * mu < 1, bound by component c (mu = (edge_c - i_c) / s_c): d mu = -mu ds_c / s_c, the bound
    component stays on its boundary line (dz_c = 0) and the other moves by d mu s + mu ds;
  * dA = -(A^2 / 2) (2 mu+ dmu+ + dmu+ mu- + mu+ dmu-), dB likewise with + and - swapped;
  * d (I U)(z) = grad(I U)(z) . dz with the gradient of the bilinear interpolant (Eq. 1.7) on
    the cell that holds z (the cell the value itself uses);
    (dL U)_j = sum_p [dA (I U)(z+) + A d(I U)(z+) - (dA + dB) U_j + dB (I U)(z-) + B d(I U)(z-)] / (2 dx).
"""
from __future__ import annotations

import dataclasses
import math
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


def _truncate_d(i1, i2, s1, s2, d1, d2, n):
    """truncate() of the oracle and its derivative along ds = (d1, d2) (index units).

    Returns mu, z1, z2 (exactly those of lisl.truncate) and dmu, dz1, dz2.  A component that
    binds the truncation stays on its boundary line; when both bind (a corner), the derivative
    of mu is taken from component 1 (a kink: either one-sided value is a derivative there).
    """
    mu, z1, z2 = lisl.truncate(i1, i2, s1, s2, n)
    top = float(n - 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        b1 = np.where(s1 > 0, (top - i1) / s1, np.where(s1 < 0, (0.0 - i1) / s1, np.inf))
        b2 = np.where(s2 > 0, (top - i2) / s2, np.where(s2 < 0, (0.0 - i2) / s2, np.inf))
        trunc = mu < 1.0
        hit1 = trunc & (b1 == mu)
        hit2 = trunc & (b2 == mu)
        dmu = np.where(hit1, -mu * d1 / s1, np.where(hit2, -mu * d2 / s2, 0.0))
    dmu = np.where(trunc, dmu, 0.0)
    dz1 = np.where(hit1, 0.0, dmu * s1 + mu * d1)
    dz2 = np.where(hit2, 0.0, dmu * s2 + mu * d2)
    return mu, z1, z2, dmu, dz1, dz2


def _bilinear_value_grad(U, z1, z2, n):
    """(I U)(z) and its gradient in z (index units) on the cell that holds z (Eq. 1.7)."""
    c1 = np.clip(np.floor(z1), 0, n - 2)
    c2 = np.clip(np.floor(z2), 0, n - 2)
    t1, t2 = z1 - c1, z2 - c2
    c1 = c1.astype(np.int64)
    c2 = c2.astype(np.int64)
    u00, u10 = U[c2, c1], U[c2, c1 + 1]
    u01, u11 = U[c2 + 1, c1], U[c2 + 1, c1 + 1]
    val = (1 - t1) * (1 - t2) * u00 + t1 * (1 - t2) * u10 + (1 - t1) * t2 * u01 + t1 * t2 * u11
    g1 = (1 - t2) * (u10 - u00) + t2 * (u11 - u01)
    g2 = (1 - t1) * (u01 - u00) + t1 * (u11 - u10)
    return val, g1, g2


def dlhat_dtheta(prob, k: int, dsig_k: np.ndarray, U_full: np.ndarray, i1, i2) -> np.ndarray:
    """(dL^k / dtheta U)_j at the interior nodes (i1, i2), closed form (see the module doc).

    dsig_k: (2, P) derivative of control k's diffusion columns.  The drift and the discount do
    not depend on theta.
    """
    if prob.sigma is None:
        raise ValueError("dL/dtheta needs x-independent diffusion columns")
    n, h = prob.n, prob.h
    rh = math.sqrt(h)
    i1 = np.asarray(i1, dtype=np.float64)
    i2 = np.asarray(i2, dtype=np.float64)
    U = np.asarray(U_full, dtype=np.float64)
    Uj = U[i2.astype(np.int64), i1.astype(np.int64)]
    sig = prob.sigma[k]
    out = np.zeros(len(i1))
    for p in range(sig.shape[1]):
        s1 = np.full_like(i1, sig[0, p] / rh)
        s2 = np.full_like(i1, sig[1, p] / rh)
        d1 = np.full_like(i1, dsig_k[0, p] / rh)
        d2 = np.full_like(i1, dsig_k[1, p] / rh)
        mup, zp1, zp2, dmup, dzp1, dzp2 = _truncate_d(i1, i2, s1, s2, d1, d2, n)
        mum, zm1, zm2, dmum, dzm1, dzm2 = _truncate_d(i1, i2, -s1, -s2, -d1, -d2, n)
        A = 2.0 / (mup * mup + mup * mum)
        B = 2.0 / (mum * mum + mum * mup)
        dA = -0.5 * A * A * (2.0 * mup * dmup + dmup * mum + mup * dmum)
        dB = -0.5 * B * B * (2.0 * mum * dmum + dmum * mup + mum * dmup)
        vp, gp1, gp2 = _bilinear_value_grad(U, zp1, zp2, n)
        vm, gm1, gm2 = _bilinear_value_grad(U, zm1, zm2, n)
        out += (dA * vp + A * (gp1 * dzp1 + gp2 * dzp2) - (dA + dB) * Uj
                + dB * vm + B * (gm1 * dzm1 + gm2 * dzm2)) / (2.0 * h)
    return out


def adjoint(prob, w: np.ndarray, dsigma: Sequence[np.ndarray] = (), n_steps: Optional[int] = None,
            T: Optional[float] = None) -> AdjointResult:
    n_steps = prob.n_steps if n_steps is None else n_steps
    T = prob.T if T is None else T
    dt = T / n_steps
    n = prob.n
    i1, i2, flat = lisl.interior_flat(n)
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
        idx = pols[s - 1]
        for p, ds in enumerate(dsigma):
            dL = np.empty(len(idx))
            for k in np.unique(idx):
                sel = idx == k
                dL[sel] = dlhat_dtheta(prob, int(k), ds[k], U_ext, i1[sel], i2[sel])
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
