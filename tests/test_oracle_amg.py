"""Pins of the oracle's aggregation AMG (oracle/amg.py).

* fmix32 is MurmurHash3's finalizer: fmix32(1) = 0x514e28b7, and it inverts with the modular
  inverses of its two multipliers.
* Matching: pairs are mutual and strong from both ends; when the rounds stop, no two unmatched
  unknowns propose each other; the heaviest strong edge of the whole matrix is always paired;
  a 1-D chain with equal couplings is fully paired except possibly isolated ends.
* Galerkin: row sums of P^T A P are the aggregated row sums of A (P 1 = 1), and a symmetric A
  gives a symmetric coarse matrix.
* Cycle: on a two-level hierarchy the K-cycle equals the explicit two-grid operator
  (pre-smoothing, exact coarse correction, post-smoothing) written with dense matrices; a
  two-step coarse GCR leaves a residual orthogonal to both search directions, a one-step GCR
  (levels below k_levels) is the minimal-residual scaling of one cycle; as a BiCGSTAB
  preconditioner it converges in a mesh-independent number of iterations on the 2-D
  Laplacian.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import amg, lisl


def _lap2d(n):
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], (n, n))
    return (sp.kron(sp.eye(n), T) + sp.kron(T, sp.eye(n))).tocsr()


def _lisl(heavy, seed=0):
    p = W.oracle_scale(heavy)
    pol = np.random.default_rng(seed).integers(0, p.K, (p.n - 2) ** 2)
    A, _ = lisl.assemble(p, pol, p.g, p.dt, p.dt)
    return A.tocsr()


def test_union_pattern_coarsens_far_reaching_directional_stencils():
    """Problem A (x-dependent diffusion direction, offsets of about 3.6 cells at 41 nodes):
    couplings are rarely mutual, yet the symmetric part pairs most unknowns, so every level
    has at most half the unknowns of the one above."""
    p = W.problem_A(41)
    r = lisl.howard_step(p, p.g, p.T, p.T)
    A, _ = lisl.assemble(p, r.policy, p.g, p.T, p.T)
    H = amg.build(A.tocsr())
    sizes = [a.shape[0] for a in H.A]
    assert sizes[-1] <= 256
    assert all(b <= a // 2 for a, b in zip(sizes, sizes[1:])), sizes


def test_graded_chain_pairs_within_the_rounds():
    """A chain whose couplings grow by 0.2 % per edge (all within one octave): ranking by
    octave and hash pairs most unknowns within ROUNDS rounds, where exact strengths would
    pair about one edge per round."""
    n = 200
    c = 1.0 + 0.002 * np.arange(n - 1)
    A = sp.diags([-c, 2.1 * np.ones(n) + np.r_[c, 0] + np.r_[0, c], -c], [-1, 0, 1]).tocsr()
    partner = amg.pairwise_match(A)
    assert np.mean(partner >= 0) > 0.8


def test_octave_is_the_binary_exponent():
    for s_, e in ((1.0, 1), (0.5, 0), (0.75, 0), (0.4999, -1), (3.0, 2), (2.0 ** -30, -29)):
        assert amg.octave(s_) == e


def test_large_coarsest_level_uses_jacobi_sweeps(monkeypatch):
    """A hierarchy that stops above COARSEST unknowns solves its last level with
    COARSE_SWEEPS damped-Jacobi sweeps from zero (closed form written densely)."""
    A = _lap2d(40)
    monkeypatch.setattr(amg, "COARSEST", 100)
    H = amg.build(A, coarsest=100, max_levels=2)
    assert len(H.A) == 2 and H.A[1].shape[0] > 100
    Ac = H.A[1].toarray()
    d = np.diag(Ac)
    b = np.random.default_rng(7).standard_normal(Ac.shape[0])
    x = 0.8 * b / d
    for _ in range(amg.COARSE_SWEEPS - 1):
        x = x + 0.8 * (b - Ac @ x) / d
    got = amg.gcr(H, 1, b, 1, 1, 0.8)
    assert np.max(np.abs(got - x)) <= 1e-12 * np.abs(x).max()


def test_coarsening_and_convergence_on_a_129_grid():
    """Every level keeps at most 3/4 of the unknowns above it, and the K-cycle (with a Jacobi
    coarsest level where coarsening stalls above 256 unknowns) preconditions BiCGSTAB to
    1e-10 in a handful of iterations."""
    p = W.scaled(129, 33, 4, seed=0)
    pol = lisl.improve(lisl.control_values(p, p.g, p.dt))
    A, _ = lisl.assemble(p, pol, p.g, p.dt, p.dt)
    A = A.tocsr()
    H = amg.build(A)
    sizes = [a.shape[0] for a in H.A]
    assert all(b <= amg.MIN_REDUCTION * a for a, b in zip(sizes, sizes[1:])), sizes
    M = spla.LinearOperator(A.shape, matvec=lambda r: amg.kcycle(H, 0, r))
    b = np.random.default_rng(8).standard_normal(A.shape[0])
    cnt = [0]
    x, info = spla.bicgstab(A, b, M=M, rtol=1e-10, callback=lambda _: cnt.__setitem__(0, cnt[0] + 1))
    assert info == 0 and cnt[0] <= 12
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_fmix32_is_murmur3_finalizer():
    assert amg.fmix32(0) == 0
    assert amg.fmix32(1) == 0x514E28B7
    inv1, inv2 = pow(0x85EBCA6B, -1, 2 ** 32), pow(0xC2B2AE35, -1, 2 ** 32)

    def unxorshift(x, s):
        y = x
        for _ in range(32 // s + 1):
            y = x ^ (y >> s)
        return y & 0xFFFFFFFF

    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2 ** 32, 200, dtype=np.uint64):
        x = int(x)
        y = amg.fmix32(x)
        y = unxorshift(y, 16)
        y = (y * inv2) & 0xFFFFFFFF
        y = unxorshift(y, 13)
        y = (y * inv1) & 0xFFFFFFFF
        y = unxorshift(y, 16)
        assert y == x


@pytest.mark.parametrize("heavy", [False, True])
def test_matching_invariants(heavy):
    A = _lisl(heavy)
    S = amg.strength(A)
    n = A.shape[0]
    smax = np.array([S.data[S.indptr[i]:S.indptr[i + 1]].max(initial=0.0) for i in range(n)])
    partner = amg.pairwise_match(A)
    paired = np.nonzero(partner >= 0)[0]
    assert len(paired) > 0.6 * n
    for i in paired:
        j = partner[i]
        assert partner[j] == i and j != i
        for a, b in ((i, j), (j, i)):   # strong from both ends
            sab = S[a, b]
            assert sab > 0 and sab >= amg.BETA * smax[a]
    # terminal state: no two unmatched unknowns propose each other
    free = partner < 0

    def proposal(i):
        best, bkey = -1, None
        for p in range(S.indptr[i], S.indptr[i + 1]):
            j, s = S.indices[p], S.data[p]
            if not free[j] or not (s > 0) or s < amg.BETA * smax[i]:
                continue
            key = (amg.octave(s), amg.edge_hash(i, j), -j)
            if bkey is None or key > bkey:
                best, bkey = j, key
        return best

    prop = {i: proposal(i) for i in np.nonzero(free)[0]}
    assert not any(j >= 0 and prop.get(j) == i for i, j in prop.items())


def test_heaviest_strong_edge_is_paired():
    A = _lisl(True, seed=3)
    S = amg.strength(A)
    n = A.shape[0]
    smax = np.array([S.data[S.indptr[i]:S.indptr[i + 1]].max(initial=0.0) for i in range(n)])
    best, bkey = None, None
    Sc = S.tocoo()
    for i, j, s in zip(Sc.row, Sc.col, Sc.data):
        if s > 0 and s >= amg.BETA * smax[i] and S[j, i] >= amg.BETA * smax[j]:
            key = (amg.octave(s), amg.edge_hash(i, j))
            if bkey is None or key > bkey:
                best, bkey = (i, j), key
    partner = amg.pairwise_match(A)
    assert partner[best[0]] == best[1]


def test_equal_chain_pairs_almost_everything():
    n = 200
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], (n, n)).tocsr()
    partner = amg.pairwise_match(T)
    # only isolated unknowns (both neighbours already paired) may stay alone
    for i in np.nonzero(partner < 0)[0]:
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        assert all(partner[j] >= 0 for j in nb)
    assert np.mean(partner >= 0) > 0.8
    assert all(abs(partner[i] - i) == 1 for i in np.nonzero(partner >= 0)[0])


@pytest.mark.parametrize("which", ["lisl", "lap"])
def test_galerkin_row_sums_and_symmetry(which):
    A = _lisl(False) if which == "lisl" else _lap2d(24)
    H = amg.build(A)
    assert len(H.A) >= 2
    for l in range(len(H.A) - 1):
        Af, Ac, agg = H.A[l], H.A[l + 1], H.agg[l]
        fine_rows = np.asarray(Af.sum(axis=1)).ravel()
        want = np.bincount(agg, weights=fine_rows)
        assert np.max(np.abs(np.asarray(Ac.sum(axis=1)).ravel() - want)) <= 1e-12 * np.abs(want).max()
        sizes = np.bincount(agg)
        assert sizes.min() >= 1 and sizes.max() <= 4
        if which == "lap":
            assert abs(Ac - Ac.T).max() <= 1e-14 * abs(Ac).max()
    assert amg.complexity(H) < 2.0


def test_two_level_kcycle_is_the_two_grid_operator(monkeypatch):
    monkeypatch.setattr(amg, "COARSEST", 2000)   # an exact coarse solve on level 1
    A = _lisl(True)
    H = amg.build(A)
    H2 = amg.AmgHierarchy(H.A[:2], H.agg[:1], H.P[:1])
    Ad = A.toarray()
    P = H.P[0].toarray()
    Ac = P.T @ Ad @ P
    Dinv = np.diag(1.0 / np.diag(Ad))
    om = 0.8
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    x0 = om * Dinv @ b
    x1 = x0 + P @ np.linalg.solve(Ac, P.T @ (b - Ad @ x0))
    x2 = x1 + om * Dinv @ (b - Ad @ x1)
    got = amg.kcycle(H2, 0, b)
    assert np.max(np.abs(got - x2)) <= 1e-12 * np.abs(x2).max()


def test_edge_hash_is_symmetric():
    rng = np.random.default_rng(5)
    for i, j in rng.integers(0, 10 ** 6, (200, 2)):
        assert amg.edge_hash(i, j) == amg.edge_hash(j, i)


def test_coarse_gcr_two_steps_minimise_over_both_directions():
    """On a level with two steps, GCR leaves a residual orthogonal to A v1 and to the
    orthogonalised A v2 (the minimal residual over span{v1, v2})."""
    A = _lap2d(40)
    H = amg.build(A)
    assert len(H.A) >= 3
    l = 1
    Al = H.A[l]
    r = np.random.default_rng(2).standard_normal(Al.shape[0])
    e = amg.gcr(H, l, r, 1, 1, 0.8)
    v1 = amg.kcycle(H, l, r)
    w1 = Al @ v1
    a1 = (w1 @ r) / (w1 @ w1)
    r2 = r - a1 * w1
    w2 = Al @ amg.kcycle(H, l, r2)
    w2 = w2 - (w2 @ w1) / (w1 @ w1) * w1
    res = r - Al @ e
    for w in (w1, w2):
        assert abs(res @ w) <= 1e-10 * np.linalg.norm(res) * np.linalg.norm(w)
    assert np.linalg.norm(res) < np.linalg.norm(r2)


def test_coarse_gcr_below_k_levels_takes_one_step():
    A = _lap2d(64)
    H = amg.build(A, coarsest=16)
    assert len(H.A) >= amg.K_LEVELS + 3
    l = amg.K_LEVELS + 1
    Al = H.A[l]
    r = np.random.default_rng(4).standard_normal(Al.shape[0])
    v1 = amg.kcycle(H, l, r)
    w1 = Al @ v1
    e = amg.gcr(H, l, r, 1, 1, 0.8)
    assert np.array_equal(e, (w1 @ r) / (w1 @ w1) * v1)
    # and the residual after one step is orthogonal to A v1
    res = r - Al @ e
    assert abs(res @ w1) <= 1e-10 * np.linalg.norm(res) * np.linalg.norm(w1)
    # level k_levels itself still takes two steps
    lk = amg.K_LEVELS
    rk = np.random.default_rng(6).standard_normal(H.A[lk].shape[0])
    vk = amg.kcycle(H, lk, rk)
    wk = H.A[lk] @ vk
    ek = amg.gcr(H, lk, rk, 1, 1, 0.8)
    assert np.max(np.abs(ek - (wk @ rk) / (wk @ wk) * vk)) > 1e-6 * np.abs(ek).max()


def test_mesh_independent_iterations_on_the_laplacian():
    its = []
    for n in (32, 64):
        A = _lap2d(n)
        H = amg.build(A)
        M = spla.LinearOperator(A.shape, matvec=lambda r, H=H: amg.kcycle(H, 0, r))
        b = np.random.default_rng(3).standard_normal(A.shape[0])
        cnt = [0]
        x, info = spla.bicgstab(A, b, M=M, rtol=1e-10, callback=lambda _: cnt.__setitem__(0, cnt[0] + 1))
        assert info == 0
        its.append(cnt[0])
    assert max(its) <= 15 and its[1] <= its[0] + 4
