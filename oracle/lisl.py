"""FP64 oracle of the truncated LISL Scheme 2, implicit Euler, Howard policy iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring): a plain, slow, vectorised-NumPy
restatement of the paper's scheme, used to check the CUDA library.

What is computed, with the passage each piece follows
-----------------------------------------------------
* Scheme 2 stencil (Section 1, "Examples of LISL schemes"): directions
  y_p^{+-} = +-sqrt(dx) sigma_p for p <= P and y_{P+1} = dx b, M = P + 1 (drift present) or P.
* Truncation (Section 2.1 and Proposition 2.2): mu^{+-}_p is the largest value in (0, 1]
  with x + mu y in the closed domain; the truncated endpoint is x + mu y.
* Truncated weights (Proposition 2.2, Eqs. 2.2 / 2.3):
  A_p = 2 / (mu+^2 + mu+ mu-), B_p = 2 / (mu-^2 + mu- mu+) for diffusion directions and
  A = B = 1 / mu for the drift direction.
* Bilinear interpolation at the endpoints (Eqs. 1.7, 2.10).
* Graph-Laplacian form of the truncated operator (Eq. 2.9):
  (L U)_j = sum_i l_{j,i} (U_i - U_j),
  l_{j,i} = sum_p [A_p w_i(x_j + y+_p) + B_p w_i(x_j + y-_p)] / (2 dx).
* Fully implicit step (Eq. 2.11 with theta = 1): row j of A has diagonal
  1 + dt (sum_p (A_p + B_p)/(2 dx) - l_{j,j} - c_j) and off-diagonals -dt l_{j,i} on interior
  columns; boundary columns move to the right-hand side as +dt l_{j,i} psi_i (Remark 2.2).
  F_j = U^{n-1}_j + dt f_j.
* Nonlinear system max_alpha (A^alpha X - F^alpha) = 0 (Eq. 1.10), solved by Howard
  policy iteration (Section 1, policy iteration of Bokanowski et al.): solve at a fixed policy,
  then improve row by row by linear search over the discrete control set.

Readings where the paper is silent (each is listed with its reason in the design notes):
* Coordinates are handled in grid-index units: node j sits at integer index (i1, i2), and a
  displacement y becomes s = y / dx.  For a diffusion column, s = sigma_p / sqrt(dx), which is
  the stencil length of Eq. 3.2.  Truncation then asks that i + mu s stays in
  [0, n-1]^2, which is the same condition as x + mu y in the closed rectangle.
* A truncated endpoint is placed exactly on the boundary line of the binding component.
* The boundary value at a truncated endpoint is interpolated from the boundary nodes
  (Eq. 2.9); `lhat_apply_exact_endpoints` gives the exact-value variant of Remark 2.2.
* Policy improvement picks the lowest control index whose value is within
  1e-12 * max(1, |v_min|) of the minimum.
* Howard iteration starts from the previous step's final policy (the first step starts from
  an improvement on X = U^0); it stops when the policy is unchanged or when
  ||X^m - X^{m-1}||_inf <= 1e-10 max(1, ||X^m||_inf), with X^0 = U^{n-1}; at most 100 iterations.

Array conventions: full-grid arrays have shape (n, n) indexed [i2, i1]; the unknowns are the
(n-2)^2 interior nodes, ordered row-major (flat interior index = (i2-1)*(n-2) + (i1-1)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

TIE_REL = 1e-12
PI_TOL = 1e-10
PI_MAX = 100


# --------------------------------------------------------------------------- geometry

def interior_nodes(n: int):
    """Index coordinates (i1, i2) of the interior nodes, row-major, as float64 arrays."""
    i2, i1 = np.meshgrid(np.arange(1, n - 1), np.arange(1, n - 1), indexing="ij")
    return i1.ravel().astype(np.float64), i2.ravel().astype(np.float64)


def truncate(i1, i2, s1, s2, n):
    """Truncation factor and endpoint for displacement s (index units) from node i.

    Returns mu, z1, z2: mu is the largest value in (0, 1] such that i + mu' s lies in
    [0, n-1]^2 for all mu' in [0, mu] (Proposition 2.2); z = i + mu s, with a binding
    component placed exactly on its boundary line.
    """
    top = float(n - 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        b1 = np.where(s1 > 0, (top - i1) / s1, np.where(s1 < 0, (0.0 - i1) / s1, np.inf))
        b2 = np.where(s2 > 0, (top - i2) / s2, np.where(s2 < 0, (0.0 - i2) / s2, np.inf))
    mu = np.minimum(1.0, np.minimum(b1, b2))
    z1 = i1 + mu * s1
    z2 = i2 + mu * s2
    trunc = mu < 1.0
    hit1 = trunc & (b1 == mu)
    hit2 = trunc & (b2 == mu)
    z1 = np.where(hit1, np.where(s1 > 0, top, 0.0), z1)
    z2 = np.where(hit2, np.where(s2 > 0, top, 0.0), z2)
    return mu, z1, z2


def bilinear(z1, z2, n):
    """Bilinear interpolation nodes and weights at index-space points z (Eq. 1.7).

    Returns four (col, weight) pairs, col = flat full-grid index i2 * n + i1.
    """
    c1 = np.clip(np.floor(z1), 0, n - 2)
    c2 = np.clip(np.floor(z2), 0, n - 2)
    t1 = z1 - c1
    t2 = z2 - c2
    c1 = c1.astype(np.int64)
    c2 = c2.astype(np.int64)
    return [
        (c2 * n + c1, (1.0 - t1) * (1.0 - t2)),
        (c2 * n + c1 + 1, t1 * (1.0 - t2)),
        ((c2 + 1) * n + c1, (1.0 - t1) * t2),
        ((c2 + 1) * n + c1 + 1, t1 * t2),
    ]


@dataclasses.dataclass
class Taps:
    """Truncated Scheme-2 operator of one control on a set of rows, in graph-Laplacian form.

    rows: row number (position in the row set) of each tap; cols: full-grid flat column;
    w: l-weight of the tap (already divided by 2 dx); W: (nrows,) sum_p (A_p + B_p) / (2 dx).
    """
    rows: np.ndarray
    cols: np.ndarray
    w: np.ndarray
    W: np.ndarray


def scheme2_taps(i1, i2, sig, drift, n, h, periodic=False) -> Taps:
    """Taps of the truncated Scheme 2 at nodes (i1, i2).

    sig: (R, 2, P) diffusion columns at each node; drift: (R, 2) or None.
    With periodic=True there is no boundary: nothing is truncated and indices wrap mod n
    (used only for the Fourier-mode check).
    """
    R = len(i1)
    P = sig.shape[2]
    rows_l, cols_l, w_l = [], [], []
    W = np.zeros(R)
    rid = np.arange(R)
    sqrt_h = math.sqrt(h)

    def add(z1, z2, scale):
        if periodic:
            c1 = np.floor(z1)
            c2 = np.floor(z2)
            t1 = z1 - c1
            t2 = z2 - c2
            c1 = c1.astype(np.int64)
            c2 = c2.astype(np.int64)
            pts = [(c1, c2, (1 - t1) * (1 - t2)), (c1 + 1, c2, t1 * (1 - t2)),
                   (c1, c2 + 1, (1 - t1) * t2), (c1 + 1, c2 + 1, t1 * t2)]
            for a1, a2, wt in pts:
                rows_l.append(rid)
                cols_l.append((a2 % n) * n + (a1 % n))
                w_l.append(wt * scale)
        else:
            for col, wt in bilinear(z1, z2, n):
                rows_l.append(rid)
                cols_l.append(col)
                w_l.append(wt * scale)

    for p in range(P):
        s1 = sig[:, 0, p] / sqrt_h
        s2 = sig[:, 1, p] / sqrt_h
        if periodic:
            mup = mum = np.ones(R)
            zp1, zp2, zm1, zm2 = i1 + s1, i2 + s2, i1 - s1, i2 - s2
        else:
            mup, zp1, zp2 = truncate(i1, i2, s1, s2, n)
            mum, zm1, zm2 = truncate(i1, i2, -s1, -s2, n)
        A = 2.0 / (mup * mup + mup * mum)
        B = 2.0 / (mum * mum + mum * mup)
        add(zp1, zp2, A / (2.0 * h))
        add(zm1, zm2, B / (2.0 * h))
        W += (A + B) / (2.0 * h)
    if drift is not None:
        # y_{P+1} = dx b, i.e. b itself in index units; A = B = 1/mu (Eq. 2.2).
        s1 = drift[:, 0]
        s2 = drift[:, 1]
        if periodic:
            mu = np.ones(R)
            z1, z2 = i1 + s1, i2 + s2
        else:
            mu, z1, z2 = truncate(i1, i2, s1, s2, n)
        AB = 2.0 / mu
        add(z1, z2, AB / (2.0 * h))
        W += AB / (2.0 * h)
    return Taps(np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(w_l), W)


# --------------------------------------------------------------------------- problem access

def control_sigma(prob, k, i1, i2):
    """(R, 2, P) diffusion columns of control k at nodes i."""
    if prob.sigma_fn is not None:
        return prob.sigma_fn(k, prob.lo + prob.h * i1, prob.lo + prob.h * i2)
    return np.broadcast_to(prob.sigma[k], (len(i1),) + prob.sigma[k].shape)


def control_drift(prob, k, i1, i2):
    if prob.drift_fn is not None:
        return prob.drift_fn(k, prob.lo + prob.h * i1, prob.lo + prob.h * i2)
    if prob.drift is not None:
        return np.broadcast_to(prob.drift[k], (len(i1), 2))
    return None


def control_c(prob, k):
    return 0.0 if prob.c is None else float(prob.c[k])


def control_taps(prob, k, i1, i2, periodic=False) -> Taps:
    return scheme2_taps(i1, i2, control_sigma(prob, k, i1, i2), control_drift(prob, k, i1, i2),
                        prob.n, prob.h, periodic=periodic)


def apply_lhat(taps: Taps, X_full: np.ndarray, rows_full: np.ndarray) -> np.ndarray:
    """(L U)_j = sum_i l_{j,i} (U_i - U_j) for the rows of `taps` (Eq. 2.9)."""
    x = X_full.ravel()
    contrib = taps.w * (x[taps.cols] - x[rows_full[taps.rows]])
    return np.bincount(taps.rows, weights=contrib, minlength=len(taps.W))


def lhat_apply_exact_endpoints(prob, k, i1, i2, q: Callable) -> np.ndarray:
    """Truncated scheme (Eq. 2.1) with exact function values at the endpoints.

    No interpolation: sum_p [A q(x + y+) - (A + B) q(x) + B q(x + y-)] / (2 dx), the form
    Remark 2.2 allows at boundary endpoints.  Used to check the weights' consistency.
    """
    n, h = prob.n, prob.h
    sig = control_sigma(prob, k, i1, i2)
    drift = control_drift(prob, k, i1, i2)
    sqrt_h = math.sqrt(h)

    def val(z1, z2):
        return q(prob.lo + h * z1, prob.lo + h * z2)

    q0 = val(i1, i2)
    out = np.zeros(len(i1))
    for p in range(sig.shape[2]):
        s1 = sig[:, 0, p] / sqrt_h
        s2 = sig[:, 1, p] / sqrt_h
        mup, zp1, zp2 = truncate(i1, i2, s1, s2, n)
        mum, zm1, zm2 = truncate(i1, i2, -s1, -s2, n)
        A = 2.0 / (mup * mup + mup * mum)
        B = 2.0 / (mum * mum + mum * mup)
        out += (A * val(zp1, zp2) - (A + B) * q0 + B * val(zm1, zm2)) / (2.0 * h)
    if drift is not None:
        mu, z1, z2 = truncate(i1, i2, drift[:, 0], drift[:, 1], n)
        out += (2.0 / mu) * (val(z1, z2) - q0) / (2.0 * h)
    return out


# --------------------------------------------------------------------------- assembly

def interior_flat(n):
    i1, i2 = interior_nodes(n)
    return i1, i2, (i2.astype(np.int64) * n + i1.astype(np.int64))


def assemble(prob, policy: np.ndarray, U_prev: np.ndarray, t: float, dt: float,
             f_full: Optional[np.ndarray] = None, psi_full: Optional[np.ndarray] = None):
    """System A^alpha X = F^alpha of the implicit step at time t for a fixed policy.

    Row j (Eq. 2.11, theta = 1): diagonal 1 + dt (W_j - l_{j,j} - c_j), interior
    off-diagonals -dt l_{j,i}; F_j = U^{n-1}_j + dt f_j + dt sum_{i on boundary} l_{j,i} psi_i.
    Returns (A as CSR over the interior unknowns, F).
    """
    n = prob.n
    i1, i2, flat = interior_flat(n)
    N = len(flat)
    if f_full is None:
        f_full = prob.f_tables(t)
    if psi_full is None:
        psi_full = prob.psi_fn(t)
    # map full-grid flat index -> interior unknown number (-1 on the boundary)
    unk = -np.ones(n * n, dtype=np.int64)
    unk[flat] = np.arange(N)
    rows_all, cols_all, vals_all = [], [], []
    diag = np.ones(N)
    F = U_prev.ravel()[flat].copy()
    for k in np.unique(policy):
        sel = np.nonzero(policy == k)[0]
        tp = control_taps(prob, int(k), i1[sel], i2[sel])
        r = sel[tp.rows]
        diag[sel] += dt * (tp.W - control_c(prob, int(k)))
        F[sel] += dt * f_full[k].ravel()[flat[sel]]
        cu = unk[tp.cols]
        inner = cu >= 0
        rows_all.append(r[inner])
        cols_all.append(cu[inner])
        vals_all.append(-dt * tp.w[inner])
        bnd = ~inner
        np.add.at(F, r[bnd], dt * tp.w[bnd] * psi_full.ravel()[tp.cols[bnd]])
    rows_all.append(np.arange(N))
    cols_all.append(np.arange(N))
    vals_all.append(diag)
    A = sp.csr_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                      shape=(N, N))
    A.sum_duplicates()
    return A, F


def control_values(prob, X_full: np.ndarray, t: float, f_full: Optional[np.ndarray] = None,
                   periodic: bool = False) -> np.ndarray:
    """v_k(j) = (L^k X)_j + c^k X_j + f^k_j for every control k and interior node j.

    A^k X - F^k = X - U^{n-1} - dt v_k once the boundary terms sit inside L X (X carries psi
    on the boundary), so the row-wise maximisation of Eq. 1.10 is the row-wise
    minimisation of v_k.
    """
    n = prob.n
    if periodic:
        i2, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        i1 = i1.ravel().astype(np.float64)
        i2 = i2.ravel().astype(np.float64)
        flat = (i2 * n + i1).astype(np.int64)
    else:
        i1, i2, flat = interior_flat(n)
    if f_full is None:
        f_full = prob.f_tables(t)
    V = np.empty((prob.K, len(flat)))
    x = X_full.ravel()
    for k in range(prob.K):
        tp = control_taps(prob, k, i1, i2, periodic=periodic)
        V[k] = apply_lhat(tp, X_full, flat) + control_c(prob, k) * x[flat] + f_full[k].ravel()[flat]
    return V


def control_values_at(prob, X_full: np.ndarray, t: float, i1: np.ndarray, i2: np.ndarray) -> np.ndarray:
    """v_k(j) of control_values at the interior nodes (i1, i2) only, shape (K, len(i1)).

    The same formulas restricted to the listed rows; the source is evaluated at those nodes
    only (f^k = sum_m phi[k, m] sum_q tau_q(t) G[m, q]), so grids too large for the full
    (K, n, n) source table can be sampled.
    """
    n = prob.n
    i1 = np.asarray(i1, dtype=np.float64)
    i2 = np.asarray(i2, dtype=np.float64)
    flat = (i2.astype(np.int64) * n + i1.astype(np.int64))
    if prob.f_fn is not None:
        f_at = prob.f_fn(t).reshape(prob.K, -1)[:, flat]
    else:
        Fm = np.einsum("q,mqs->ms", prob.tau(t), prob.G.reshape(prob.G.shape[0], prob.G.shape[1], -1)[:, :, flat])
        f_at = prob.phi @ Fm
    V = np.empty((prob.K, len(flat)))
    x = X_full.ravel()
    for k in range(prob.K):
        tp = control_taps(prob, k, i1, i2)
        V[k] = apply_lhat(tp, X_full, flat) + control_c(prob, k) * x[flat] + f_at[k]
    return V


def improve(V: np.ndarray) -> np.ndarray:
    """Row-wise linear search: lowest k with v_k <= v_min + 1e-12 max(1, |v_min|)."""
    vmin = V.min(axis=0)
    eps = TIE_REL * np.maximum(1.0, np.abs(vmin))
    return np.argmax(V <= vmin + eps, axis=0).astype(np.int64)


# --------------------------------------------------------------------------- solves

def direct_solve(A, F):
    return spla.splu(A.tocsc()).solve(F)


@dataclasses.dataclass
class StepResult:
    X: np.ndarray            # full grid, psi(t_n) on the boundary
    policy: np.ndarray       # (N,) final policy of the step
    pi_iters: int
    iterates: List[np.ndarray]
    converged: bool
    solve_policy: Optional[np.ndarray] = None   # policy of the last linear solve (defines A_n)


def howard_step(prob, U_prev: np.ndarray, t: float, dt: float, policy0=None,
                pi_tol: float = PI_TOL, pi_max: int = PI_MAX,
                keep_iterates: bool = False) -> StepResult:
    """One implicit step: Howard policy iteration on max_k (A^k X - F^k) = 0."""
    n = prob.n
    _, _, flat = interior_flat(n)
    f_full = prob.f_tables(t)
    psi = prob.psi_fn(t)
    X_full = U_prev.copy()
    bmask = np.ones((n, n), dtype=bool)
    bmask[1:-1, 1:-1] = False
    X_full[bmask] = psi[bmask]
    if policy0 is None:
        policy = improve(control_values(prob, X_full, t, f_full))
    else:
        policy = np.asarray(policy0, dtype=np.int64).copy()
    X_prev = U_prev.ravel()[flat].copy()
    iterates = []
    for it in range(1, pi_max + 1):
        A, F = assemble(prob, policy, U_prev, t, dt, f_full, psi)
        X = direct_solve(A, F)
        X_full.ravel()[flat] = X
        if keep_iterates:
            iterates.append(X.copy())
        new_policy = improve(control_values(prob, X_full, t, f_full))
        same = bool(np.all(new_policy == policy))
        small = np.max(np.abs(X - X_prev)) <= pi_tol * max(1.0, np.max(np.abs(X)))
        used = policy
        policy = new_policy
        X_prev = X
        if same or small:
            return StepResult(X_full, policy, it, iterates, True, used)
    return StepResult(X_full, policy, pi_max, iterates, False, used)


@dataclasses.dataclass
class SolveResult:
    U: np.ndarray
    policies: List[np.ndarray]
    pi_iters: List[int]
    converged: bool


def solve(prob, n_steps: Optional[int] = None, T: Optional[float] = None,
          U0: Optional[np.ndarray] = None, t0: float = 0.0) -> SolveResult:
    """Implicit Euler over n_steps uniform steps from U0 = g (Section 1, theta = 1)."""
    n_steps = prob.n_steps if n_steps is None else n_steps
    T = prob.T if T is None else T
    dt = T / n_steps
    U = (prob.g if U0 is None else U0).copy()
    policy = None
    policies, iters = [], []
    ok = True
    for s in range(1, n_steps + 1):
        t = t0 + s * dt
        res = howard_step(prob, U, t, dt, policy0=policy)
        U, policy = res.X, res.policy
        policies.append(policy.copy())
        iters.append(res.pi_iters)
        ok = ok and res.converged
    return SolveResult(U, policies, iters, ok)


def hjb_residual(prob, X_full, U_prev, t, dt):
    """max_k (A^k X - F^k)_j = max_k (X_j - U^{n-1}_j - dt v_k(j)) for every interior j."""
    _, _, flat = interior_flat(prob.n)
    V = control_values(prob, X_full, t)
    return X_full.ravel()[flat] - U_prev.ravel()[flat] - dt * V.min(axis=0)


# --------------------------------------------------------------------------- periodic mode

def periodic_step_matrix(prob, k: int, dt: float):
    """I - dt L^k on the periodic n x n grid (all n^2 nodes unknown, no truncation)."""
    n = prob.n
    i2, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i1 = i1.ravel().astype(np.float64)
    i2 = i2.ravel().astype(np.float64)
    tp = control_taps(prob, k, i1, i2, periodic=True)
    N = n * n
    L = sp.csr_matrix((tp.w, (tp.rows, tp.cols)), shape=(N, N)) - sp.diags(tp.W)
    return (sp.identity(N) - dt * L).tocsr()
