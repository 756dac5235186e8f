"""Aggregation-based algebraic multigrid with a K-cycle (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves the step systems with AGMG, aggregation AMG as a Krylov preconditioner in an
enhanced (Krylov-accelerated) cycle, and justifies it by the M-matrix property with
non-negative row and column sums of the LISL matrices (Section 3.4, Prop. 3.1; the method of
Notay's aggregation papers that it cites).  The paper gives no algorithm listing; this module
restates the published scheme in the following form, which the GPU path implements exactly:

Coarsening (one level = two pairwise passes, aggregates of at most four unknowns):
  * strength of the coupling i-j: the off-diagonal entries of the symmetric part,
    s_ij = -(a_ij + a_ji) / 2, on the union of the patterns of A and A^T (zero entries
    dropped).  The paper points to A + A^T as the matrix that carries the aggregation
    theory's assumptions for non-symmetric M-matrices (Section 3.4), and the union pattern
    matters: with far-reaching stencils whose direction depends on x (Problem A) a_ij != 0
    rarely comes with a_ji != 0, and a row-only pattern leaves almost nothing to pair.
    j is a strong neighbour of i when s_ij > 0 and s_ij >= beta * max_k s_ik, beta = 0.25;
  * pairwise matching in rounds: every unmatched unknown proposes its strong unmatched
    neighbour that is largest in the order of the edge keys (e(s_ij), h(i, j), -j), where
    e(s) is the binary exponent of s (s = m 2^e, m in [0.5, 1)), so strengths within a factor
    two rank equal and are ordered by the hash: on the nearly one-dimensional coarse graphs
    of anisotropic LISL operators, exactly graded strengths form chains along which a
    locally-dominant matching pairs one edge per round, while hashed ties pair a fixed
    fraction per round.  h(i, j)
    = fmix32(min(i, j) XOR fmix32(max(i, j))) and fmix32 is the 32-bit finalizer of
    MurmurHash3 (x ^= x >> 16; x *= 0x85ebca6b; x ^= x >> 13; x *= 0xc2b2ae35; x ^= x >> 16).
    The key of an edge is the same seen from either end, so this is a locally-dominant edge
    matching: the heaviest unmatched edge always pairs, and equal strengths (every interior
    row of a translation-invariant region) are ordered pseudo-randomly instead of forming
    proposal chains.  Two unknowns that propose each other form a pair.  Rounds repeat until
    none forms a pair (at most `rounds`); unknowns left unmatched stay alone;
  * aggregates are numbered in the order of their lowest member; the prolongation P is
    piecewise constant (P_iI = 1 for i in aggregate I), the coarse matrix is the Galerkin
    product P^T A P.  The second pass repeats the matching on that coarse matrix, and the
    level's aggregates are the unions.
  * coarsening stops at a level of at most 256 unknowns, or when a level would keep more than
    3/4 of the unknowns of the one above (or at 16 levels).  The last level is solved exactly
    (dense) when it has at most 256 unknowns, and otherwise approximately by COARSE_SWEEPS
    damped-Jacobi sweeps from zero.
Cycle (K-cycle, damped Jacobi, GCR acceleration of the coarse corrections):
  kcycle(l, b): x = omega D^-1 b, nu1 - 1 further sweeps x += omega D^-1 (b - A x);
                r = b - A x; e = gcr(l + 1, P^T r) (an exact solve on the coarsest level);
                x += P e; nu2 sweeps; return x.
  gcr(l, r):   v1 = kcycle(l, r); w1 = A v1; a1 = (w1.r)/(w1.w1); e = a1 v1;
               on levels l <= k_levels a second step follows: r2 = r - a1 w1;
               v2 = kcycle(l, r2); w2 = A v2; g = (w2.w1)/(w1.w1); w2 -= g w1; v2 -= g v1;
               a2 = (w2.r2)/(w2.w2); e += a2 v2.   (a zero denominator gives a zero step)
The number of GCR steps per level is fixed (two on the first k_levels coarse levels, one
below) instead of being decided by the size of the first step's residual: a data-dependent
exit would have to be decided on the device before launching the second step's subtree, and
with two steps on every level the launches grow as 2^l.  With k_levels = 2 the levels below
the second are visited four times per cycle.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

BETA = 0.25
ROUNDS = 8
K_LEVELS = 2
COARSEST = 256        # exact dense solve at or below this size
MIN_REDUCTION = 0.75  # a level must keep at most this fraction of the unknowns above it
COARSE_SWEEPS = 16


def strength(A: sp.csr_matrix) -> sp.csr_matrix:
    """Off-diagonal part of -(A + A^T) / 2 on the union pattern, zero entries dropped."""
    A = A.tocsr()
    S = (-(A + A.T) / 2.0).tocsr()
    S.setdiag(0.0)
    S.eliminate_zeros()
    S.sort_indices()
    return S


def fmix32(x: int) -> int:
    """MurmurHash3's 32-bit finalizer."""
    x &= 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & 0xFFFFFFFF
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def octave(s: float) -> int:
    """The binary exponent e of s = m 2^e, m in [0.5, 1) (exact, from the floating-point bits)."""
    return math.frexp(s)[1]


def edge_hash(i: int, j: int) -> int:
    i, j = int(i), int(j)
    a, b = (i, j) if i < j else (j, i)
    return fmix32(a ^ fmix32(b))


def pairwise_match(A: sp.csr_matrix, beta: float = BETA, rounds: int = ROUNDS) -> np.ndarray:
    """partner[i] = the unknown paired with i, or -1 (see the module docstring)."""
    A = A.tocsr()
    n = A.shape[0]
    S = strength(A)
    smax = np.zeros(n)
    for i in range(n):
        row = S.data[S.indptr[i]:S.indptr[i + 1]]
        smax[i] = row.max() if len(row) else 0.0
    partner = -np.ones(n, dtype=np.int64)
    for _ in range(rounds):
        prop = -np.ones(n, dtype=np.int64)
        for i in range(n):
            if partner[i] >= 0:
                continue
            best, bkey = -1, None
            for p in range(S.indptr[i], S.indptr[i + 1]):
                j, s = S.indices[p], S.data[p]
                if partner[j] >= 0 or not (s > 0.0) or s < beta * smax[i]:
                    continue
                key = (octave(s), edge_hash(i, j), -j)
                if bkey is None or key > bkey:
                    best, bkey = j, key
            prop[i] = best
        new = 0
        for i in range(n):
            j = prop[i]
            if j >= 0 and prop[j] == i:
                partner[i] = j
                new += 1
        if new == 0:
            break
    return partner


def aggregates_from_pairs(partner: np.ndarray) -> np.ndarray:
    """agg[i]: aggregates numbered in the order of their lowest member."""
    n = len(partner)
    agg = -np.ones(n, dtype=np.int64)
    nxt = 0
    for i in range(n):
        j = partner[i]
        if j < 0 or i < j:
            agg[i] = nxt
            if j >= 0:
                agg[j] = nxt
            nxt += 1
    return agg


def prolongation(agg: np.ndarray) -> sp.csr_matrix:
    n = len(agg)
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, int(agg.max()) + 1))


@dataclasses.dataclass
class AmgHierarchy:
    A: List[sp.csr_matrix]
    agg: List[np.ndarray]        # agg[l][i] = aggregate (unknown of level l+1) of unknown i of level l
    P: List[sp.csr_matrix]


def build(A: sp.csr_matrix, coarsest: int = COARSEST, max_levels: int = 16) -> AmgHierarchy:
    """Levels until the coarse matrix has at most `coarsest` unknowns, coarsening stalls
    (more than MIN_REDUCTION of the unknowns kept) or max_levels is reached."""
    As, aggs, Ps = [A.tocsr()], [], []
    while As[-1].shape[0] > coarsest and len(As) < max_levels:
        Al = As[-1]
        a1 = aggregates_from_pairs(pairwise_match(Al))
        P1 = prolongation(a1)
        A1 = (P1.T @ Al @ P1).tocsr()
        a2 = aggregates_from_pairs(pairwise_match(A1))
        agg = a2[a1]
        if int(agg.max()) + 1 > MIN_REDUCTION * Al.shape[0]:
            break
        P = prolongation(agg)
        As.append((P.T @ Al @ P).tocsr())
        aggs.append(agg)
        Ps.append(P)
    return AmgHierarchy(As, aggs, Ps)


def coarsest_solve(A: sp.csr_matrix, b: np.ndarray, omega: float) -> np.ndarray:
    """Exact for at most COARSEST unknowns, else COARSE_SWEEPS damped-Jacobi sweeps from 0."""
    if A.shape[0] <= COARSEST:
        return sla.solve(A.toarray(), b)
    d = A.diagonal()
    x = omega * b / d
    for _ in range(COARSE_SWEEPS - 1):
        x = x + omega * (b - A @ x) / d
    return x


def kcycle(H: AmgHierarchy, l: int, b: np.ndarray, nu1: int = 1, nu2: int = 1,
           omega: float = 0.8, k_levels: int = K_LEVELS) -> np.ndarray:
    A = H.A[l]
    if l == len(H.A) - 1:
        return coarsest_solve(A, b, omega)
    d = A.diagonal()
    x = omega * b / d
    for _ in range(nu1 - 1):
        x = x + omega * (b - A @ x) / d
    r = b - A @ x
    e = gcr(H, l + 1, H.P[l].T @ r, nu1, nu2, omega, k_levels)
    x = x + H.P[l] @ e
    for _ in range(nu2):
        x = x + omega * (b - A @ x) / d
    return x


def gcr(H: AmgHierarchy, l: int, r: np.ndarray, nu1: int, nu2: int, omega: float,
        k_levels: int = K_LEVELS) -> np.ndarray:
    A = H.A[l]
    if l == len(H.A) - 1:
        return coarsest_solve(A, r, omega)
    v1 = kcycle(H, l, r, nu1, nu2, omega, k_levels)
    w1 = A @ v1
    ww = w1 @ w1
    a1 = (w1 @ r) / ww if ww > 0.0 else 0.0     # r = 0 gives e = 0
    e = a1 * v1
    if l > k_levels:
        return e
    r2 = r - a1 * w1
    v2 = kcycle(H, l, r2, nu1, nu2, omega, k_levels)
    w2 = A @ v2
    g = (w2 @ w1) / ww if ww > 0.0 else 0.0
    w2 = w2 - g * w1
    v2 = v2 - g * v1
    w22 = w2 @ w2
    a2 = (w2 @ r2) / w22 if w22 > 0.0 else 0.0
    return e + a2 * v2


def complexity(H: AmgHierarchy) -> float:
    """Operator complexity c_A = sum_l nnz(A_l) / nnz(A_0)."""
    return sum(A.nnz for A in H.A) / H.A[0].nnz
