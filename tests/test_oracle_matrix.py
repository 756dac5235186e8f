"""Pins of the oracle's assembled system against invariants the paper proves.

Positive type / M-matrix structure (Corollary 2.3 a, Eq. 2.11), row sums (Section 3.4:
1 + dt (M/dx - c) - dt M/dx >= 0, including the boundary columns), the lower bound
sum_i l_{j,i} >= M/dx with equality exactly when nothing is truncated (after Eq. 2.9),
column sums under the step-size condition of Proposition 3.1, and the discrete maximum
principle that monotonicity implies.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import lisl


def _full_rows(prob, policy, dt):
    """Rows including boundary columns: (A_int, boundary-column weights, W)."""
    n = prob.n
    i1, i2, flat = lisl.interior_flat(n)
    N = len(flat)
    Bcols = sp.lil_matrix((N, n * n))
    Wrow = np.zeros(N)
    unk = -np.ones(n * n, dtype=np.int64)
    unk[flat] = np.arange(N)
    for k in np.unique(policy):
        sel = np.nonzero(policy == k)[0]
        tp = lisl.control_taps(prob, int(k), i1[sel], i2[sel])
        Wrow[sel] = tp.W
        r = sel[tp.rows]
        bnd = unk[tp.cols] < 0
        for rr, cc, ww in zip(r[bnd], tp.cols[bnd], tp.w[bnd]):
            Bcols[rr, cc] += dt * ww
    return Bcols.tocsr(), Wrow


CASES = [
    ("config33", lambda: W.oracle_scale(False)),
    ("heavy33", lambda: W.oracle_scale(True)),
    ("problemA21", lambda: W.problem_A(21, n_alpha=8)),
]


@pytest.mark.parametrize("name,mk", CASES)
def test_m_matrix_structure_and_row_sums(name, mk):
    p = mk()
    rng = np.random.default_rng(11)
    N = (p.n - 2) ** 2
    policy = rng.integers(0, p.K, size=N)
    dt = 0.05
    A, F = lisl.assemble(p, policy, p.g, 0.1, dt)
    A = A.tocsr()
    d = A.diagonal()
    off = A - sp.diags(d)
    assert np.all(d > 0)
    assert off.data.max(initial=0.0) <= 0.0
    Bc, Wrow = _full_rows(p, policy, dt)
    # row sum over interior and boundary columns (a boundary column would carry -dt l_{j,i})
    # equals 1 - dt c  (c = 0 here)
    rs = np.asarray(A.sum(axis=1)).ravel() - np.asarray(Bc.sum(axis=1)).ravel()
    assert np.max(np.abs(rs - 1.0)) <= 1e-12 * (1 + dt * Wrow.max())
    # sum_i l_{j,i} = sum_p (A_p + B_p)/(2 dx) >= M / dx, equality iff untruncated
    # Problem A: one diffusion column plus the drift direction; the others: two columns
    M = 2
    assert np.all(Wrow >= M / p.h * (1 - 1e-14))


def test_sum_of_lhat_weights_equality_iff_untruncated():
    p = W.oracle_scale(True)
    i1, i2, _ = lisl.interior_flat(p.n)
    for k in range(p.K):
        tp = lisl.control_taps(p, k, i1, i2)
        S = np.bincount(tp.rows, weights=tp.w, minlength=len(tp.W))
        assert np.max(np.abs(S - tp.W)) <= 1e-12 * tp.W.max()   # partition of unity
        s = p.sigma[k] / np.sqrt(p.h)
        reach = np.abs(s).sum(axis=1)                           # |s_1| + |s_2| per axis (loose)
        far = (i1 - 1 >= reach[0] + 1) & (p.n - 2 - i1 >= reach[0] + 1) & \
              (i2 - 1 >= reach[1] + 1) & (p.n - 2 - i2 >= reach[1] + 1)
        assert np.allclose(tp.W[far], 2 / p.h, rtol=0, atol=1e-12 / p.h)


def test_column_sums_nonnegative_under_prop_3_1():
    """Proposition 3.1 with constant coefficients: dt <= dx / ((3^d - 1)(P + 1)) gives
    non-negative column sums (here c = 0, d = 2, P = 2)."""
    for heavy in (False, True):
        p = W.oracle_scale(heavy)
        rng = np.random.default_rng(5)
        N = (p.n - 2) ** 2
        for policy in (np.zeros(N, dtype=np.int64), rng.integers(0, p.K, size=N)):
            dt = p.h / ((3 ** 2 - 1) * (2 + 1))
            A, _ = lisl.assemble(p, policy, p.g, 0.0, dt)
            cs = np.asarray(A.sum(axis=0)).ravel()
            if np.all(policy == 0):
                assert cs.min() >= -1e-12


@pytest.mark.parametrize("heavy", [False, True])
def test_discrete_maximum_principle(heavy):
    """Inverse positivity: F >= 0 gives X >= 0; with c = f = 0 one implicit step keeps
    min(psi, U) <= X <= max(psi, U); ||X||_inf <= ||F||_inf."""
    p = W.oracle_scale(heavy)
    rng = np.random.default_rng(1)
    N = (p.n - 2) ** 2
    policy = rng.integers(0, p.K, size=N)
    A, _ = lisl.assemble(p, policy, p.g, 0.0, 0.1)
    for _ in range(5):
        F = rng.uniform(0, 1, size=N)
        X = lisl.direct_solve(A, F)
        assert X.min() >= -1e-13
        assert np.abs(X).max() <= np.abs(F).max() * (1 + 1e-12)
    # c = f = 0 with random boundary data and previous values
    U = rng.uniform(-1, 1, size=(p.n, p.n))
    psi = rng.uniform(-1, 1, size=(p.n, p.n))
    A, F = lisl.assemble(p, policy, U, 0.0, 0.1, f_full=np.zeros((p.K, p.n, p.n)), psi_full=psi)
    X = lisl.direct_solve(A, F)
    bmask = np.ones((p.n, p.n), dtype=bool)
    bmask[1:-1, 1:-1] = False
    lo = min(psi[bmask].min(), U[1:-1, 1:-1].min())
    hi = max(psi[bmask].max(), U[1:-1, 1:-1].max())
    assert X.min() >= lo - 1e-12 and X.max() <= hi + 1e-12


@pytest.mark.parametrize("heavy", [False, True])
def test_bilinear_discrete_solution_with_boundary_data_and_discount(heavy):
    """A bilinear q is differentiated exactly by every row (interpolation reproduces it and the
    truncated weights are consistent), so with psi = q on the boundary, discount c, f = 0 and
    U^{n-1} = q - dt (L q + c q), the implicit step's solution is X = q exactly.  This fixes
    the boundary right-hand side (Remark 2.2) and the -dt c diagonal term (Eq. 2.11)."""
    p = W.oracle_scale(heavy)
    rng = np.random.default_rng(9)
    p.c = rng.uniform(0.0, 2.0, size=p.K)
    coef = rng.normal(size=4)
    X1, X2 = p.coords()
    q = coef[0] + coef[1] * X1 + coef[2] * X2 + coef[3] * X1 * X2
    dt = 0.07
    N = (p.n - 2) ** 2
    policy = rng.integers(0, p.K, size=N)
    i1, i2, flat = lisl.interior_flat(p.n)
    Lq = np.empty(N)
    cq = np.empty(N)
    for k in range(p.K):
        sel = policy == k
        S = p.sigma[k]
        Lq[sel] = (S @ S.T)[0, 1] * coef[3]          # tr(a D^2 q) for bilinear q
        cq[sel] = p.c[k] * q.ravel()[flat[sel]]
    U = q.copy()
    U.ravel()[flat] = q.ravel()[flat] - dt * (Lq + cq)
    A, F = lisl.assemble(p, policy, U, 0.0, dt, f_full=np.zeros((p.K, p.n, p.n)), psi_full=q)
    X = lisl.direct_solve(A, F)
    assert np.max(np.abs(X - q.ravel()[flat])) <= 1e-11 * (1 + np.abs(q).max())
    # the same holds through the control values used by the policy improvement
    V = lisl.control_values(p, q, 0.0, f_full=np.zeros((p.K, p.n, p.n)))
    chosen = V[policy, np.arange(N)]
    assert np.max(np.abs(chosen - (Lq + cq))) <= 1e-10 * (1 + np.abs(q).max()) / p.h


@pytest.mark.parametrize("heavy", [False, True])
def test_sampled_control_values_equal_the_full_evaluation(heavy):
    """control_values_at (used to check full-size GPU steps node by node) restricted to every
    interior node, and to a shuffled subset, reproduces control_values, including a non-zero
    boundary, a discount and a drift."""
    p = W.with_dirichlet(W.oracle_scale(heavy))
    p.c = np.linspace(-0.5, 0.3, p.K)
    p.drift = np.stack([np.linspace(-2.0, 2.0, p.K), np.linspace(1.5, -1.0, p.K)], axis=1)
    rng = np.random.default_rng(0)
    X = p.g + rng.uniform(-0.1, 0.1, p.g.shape)
    t = 0.37
    V = lisl.control_values(p, X, t)
    i1, i2, _ = lisl.interior_flat(p.n)
    Va = lisl.control_values_at(p, X, t, i1, i2)
    assert np.max(np.abs(Va - V)) <= 1e-13 * max(1.0, np.abs(V).max())
    sel = rng.permutation(len(i1))[:50]
    Vs = lisl.control_values_at(p, X, t, i1[sel], i2[sel])
    assert np.max(np.abs(Vs - V[:, sel])) <= 1e-13 * max(1.0, np.abs(V).max())
