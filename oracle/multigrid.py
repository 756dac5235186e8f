"""Geometric multigrid pieces of the oracle: transfers, Galerkin hierarchy, V-cycle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Section 3.3 (performance of geometric multigrid): standard coarsening
Omega_{dx} -> Omega_{2 dx} on 2^l + 1 grids, bilinear prolongation P, restriction the
(scaled) transpose of P, and coarse operators built by the Galerkin principle
A_{l+1} = R A_l P.  Restriction is full weighting, R = P^T / 4; the preconditioner
P (R A P)^{-1} R does not depend on the scale of R, so this is the paper's R = P^T up to a
factor.  The smoother is damped Jacobi x <- x + omega D^{-1} (b - A x), and the coarsest
level is solved directly.  Grid and algebraic complexities follow Definitions 3.1 and 3.2.

The paper's geometric multigrid smooths with Gauss-Seidel (Section 3.3).  Its data-parallel
form here is the two-colour (red-black) Gauss-Seidel sweep: the interior nodes with i1 + i2
even, then those with i1 + i2 odd, each colour updated at once from the current values of all
nodes, x_c <- x_c + omega D_c^{-1} (b - A x)_c.  For the 5-point Laplacian, whose nodes of one
colour do not couple, this is Gauss-Seidel in red-black order exactly; the wide LISL stencils
couple nodes of one colour too, which the simultaneous update of a colour treats as Jacobi does.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def prolongation(nc: int) -> sp.csr_matrix:
    """Bilinear interpolation from the interior of an nc x nc grid to the interior of the
    (2 nc - 1) x (2 nc - 1) grid; boundary values are zero (Dirichlet), so coarse boundary
    nodes carry no column."""
    nf = 2 * nc - 1
    mf, mc = nf - 2, nc - 2
    # 1-D: fine index i (1..nf-2) takes coarse I = i/2 (weight 1) if i even, else
    # (i-1)/2 and (i+1)/2 (weight 1/2 each); coarse 0 and nc-1 are boundary (dropped).
    rows, cols, vals = [], [], []
    for i in range(1, nf - 1):
        if i % 2 == 0:
            pairs = [(i // 2, 1.0)]
        else:
            pairs = [((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5)]
        for I, w in pairs:
            if 1 <= I <= nc - 2:
                rows.append(i - 1)
                cols.append(I - 1)
                vals.append(w)
    P1 = sp.csr_matrix((vals, (rows, cols)), shape=(mf, mc))
    # unknowns are ordered (i2, i1) row-major, so the 2-D operator is kron(P_x2, P_x1)
    return sp.kron(P1, P1, format="csr")


def restriction(nc: int) -> sp.csr_matrix:
    """Full weighting, R = P^T / 4 (stencil [1 2 1; 2 4 2; 1 2 1] / 16)."""
    return (0.25 * prolongation(nc).T).tocsr()


@dataclasses.dataclass
class Hierarchy:
    A: List[sp.csr_matrix]
    P: List[sp.csr_matrix]
    R: List[sp.csr_matrix]
    n: List[int]             # nodes per dimension (boundary included) on each level


def galerkin_hierarchy(A0: sp.csr_matrix, n0: int, levels: int) -> Hierarchy:
    """A_{l+1} = R_l A_l P_l for l = 0 .. levels-2 (Galerkin principle)."""
    A = [A0.tocsr()]
    Ps, Rs, ns = [], [], [n0]
    n = n0
    for _ in range(levels - 1):
        if (n - 1) % 2 != 0 or n < 5:
            raise ValueError("grid does not coarsen: need n = 2^k + 1")
        nc = (n + 1) // 2
        P = prolongation(nc)
        R = restriction(nc)
        Ac = (R @ A[-1] @ P).tocsr()
        Ac.sum_duplicates()
        A.append(Ac)
        Ps.append(P)
        Rs.append(R)
        ns.append(nc)
        n = nc
    return Hierarchy(A, Ps, Rs, ns)


def jacobi(A, b, x, omega, sweeps):
    d = A.diagonal()
    for _ in range(sweeps):
        x = x + omega * (b - A @ x) / d
    return x


def colours(n: int) -> np.ndarray:
    """(i1 + i2) mod 2 of the interior nodes of an n x n grid, in the unknowns' row-major order."""
    i2, i1 = np.meshgrid(np.arange(1, n - 1), np.arange(1, n - 1), indexing="ij")
    return ((i1 + i2) % 2).ravel()


def rbgs(A, b, x, omega, sweeps, n):
    """Two-colour Gauss-Seidel sweeps: colour 0 (i1 + i2 even), then colour 1, each updated at once."""
    d = A.diagonal()
    col = colours(n)
    for _ in range(sweeps):
        for c in (0, 1):
            sel = col == c
            r = b - A @ x
            x = x.copy()
            x[sel] += omega * r[sel] / d[sel]
    return x


def vcycle(H: Hierarchy, b: np.ndarray, nu1: int = 2, nu2: int = 2, omega: float = 0.8,
           level: int = 0, smoother: str = "jacobi") -> np.ndarray:
    """One V(nu1, nu2) cycle for A_level x = b from x = 0; exact solve on the coarsest level.
    smoother: "jacobi" (damped Jacobi) or "rbgs" (two-colour Gauss-Seidel, relaxation omega)."""
    A = H.A[level]
    if level == len(H.A) - 1:
        return spla.spsolve(A.tocsc(), b)

    def smooth(x, sweeps):
        if smoother == "rbgs":
            return rbgs(A, b, x, omega, sweeps, H.n[level])
        return jacobi(A, b, x, omega, sweeps)

    x = smooth(np.zeros_like(b), nu1)
    r = b - A @ x
    ec = vcycle(H, H.R[level] @ r, nu1, nu2, omega, level + 1, smoother)
    x = x + H.P[level] @ ec
    return smooth(x, nu2)


def complexities(H: Hierarchy):
    """Grid complexity c_G and algebraic complexity c_A (Definitions 3.1, 3.2)."""
    N = [A.shape[0] for A in H.A]
    nnz = [A.count_nonzero() for A in H.A]
    return sum(N) / N[0], sum(nnz) / nnz[0]
