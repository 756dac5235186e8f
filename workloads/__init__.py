"""Seeded synthetic inputs for the implicit LISL HJB solver (shared by tests, bench and smoke).

This module only *describes problems*: grids, control sets, diffusion columns, source
terms, boundary and initial data, and closed-form solutions.  It holds none of the
scheme's arithmetic (no stencils, truncation, interpolation, assembly or solves); both the
CPU oracle and the CUDA library receive the arrays built here as plain inputs.

Problem family (uncertain-correlation HJB, the 2-D shape of the paper's benchmarks):

    u_t - inf_{rho in {rho_k}} { L^rho u + f^rho } = 0   on (0, T] x [-2, 2]^2     (Eq. 1.1)
    L^rho u = tr(a^rho D^2 u),  a^rho = 1/2 sigma^rho sigma^rho^T                   (def of L)
    sigma^rho = [[s1, 0], [s2 rho, s2 sqrt(1 - rho^2)]]  (columns sigma_1, sigma_2; P = 2)
    b = 0, c = 0, psi = 0 on the boundary, g = u(0, .)

with the manufactured solution u = exp(-t) cos(pi x1 / 4) cos(pi x2 / 4) and
f^rho = u_t - L^rho u + 5 (rho - rho*(x))^2, rho*(x) = 0.8 tanh(x1 x2).  The source is
passed in the library's separable form  f^k(t, x) = sum_m phi[k, m] sum_q tau_q(t) G[m, q, x]
with phi[k] = (1, rho_k, rho_k^2) and time factors tau = (1, exp(-t)).

Problems A and B of Section 2.4 (x-dependent diffusion, drift control, controls on the unit
circle) are also described here for the oracle's printed-value checks (Tables 2.4 / A.4).

Arrays of grid values have shape (n, n) and are indexed [i2, i1]: x1 runs along the fast
(last) axis, x = lo + h * (i1, i2), h = (hi - lo) / (n - 1).
"""
from __future__ import annotations

import copy
import dataclasses
import math
from typing import Callable, Optional

import numpy as np

# Time factor kinds understood by the library's separable source/boundary model.
TAU_ONE = 0      # tau(t) = 1
TAU_EXP = 1      # tau(t) = exp(rate * t)
TAU_LINEAR = 2   # tau(t) = t


@dataclasses.dataclass
class Problem:
    """One HJB instance on a square grid.

    sigma:  (K, 2, P) constant diffusion columns per control, or None when sigma_fn is given.
    sigma_fn: optional callable (k, X1, X2) -> (..., 2, P) for x-dependent diffusion.
    drift:  (K, 2) constant drift per control or None.
    c:      (K,) constant discount per control or None.
    phi:    (K, nf) control factors of the source; G: (nf, nq, n, n) spatial tables;
            tau_kind / tau_rate: (nq,) time factors, f^k(t) = sum_m phi[k,m] sum_q tau_q(t) G[m,q].
    f_fn:   optional callable (t) -> (K, n, n) used instead of (phi, G) by problems whose
            source is not separable (Problems A and B); only the oracle consumes it.
    psi_fn: callable (t) -> (n, n) boundary values (interior entries ignored).
    g:      (n, n) initial data.
    exact:  optional callable (t) -> (n, n) closed-form solution.
    """

    name: str
    n: int
    lo: float
    hi: float
    T: float
    n_steps: int
    sigma: Optional[np.ndarray]
    phi: Optional[np.ndarray]
    G: Optional[np.ndarray]
    tau_kind: Optional[np.ndarray]
    tau_rate: Optional[np.ndarray]
    g: np.ndarray
    psi_fn: Callable[[float], np.ndarray]
    exact: Optional[Callable[[float], np.ndarray]] = None
    drift: Optional[np.ndarray] = None
    c: Optional[np.ndarray] = None
    sigma_fn: Optional[Callable] = None
    drift_fn: Optional[Callable] = None
    f_fn: Optional[Callable[[float], np.ndarray]] = None
    rho: Optional[np.ndarray] = None
    s1: float = 0.0
    s2: float = 0.0

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / (self.n - 1)

    @property
    def K(self) -> int:
        if self.sigma is not None:
            return self.sigma.shape[0]
        return self.phi.shape[0] if self.phi is not None else int(self._K)

    @property
    def dt(self) -> float:
        return self.T / self.n_steps

    def coords(self):
        x = self.lo + self.h * np.arange(self.n, dtype=np.float64)
        X1, X2 = np.meshgrid(x, x, indexing="xy")  # X1[i2, i1] = x[i1]
        return X1, X2

    def tau(self, t: float) -> np.ndarray:
        out = np.empty(len(self.tau_kind))
        for q, (kind, rate) in enumerate(zip(self.tau_kind, self.tau_rate)):
            out[q] = 1.0 if kind == TAU_ONE else (math.exp(rate * t) if kind == TAU_EXP else t)
        return out

    def f_tables(self, t: float) -> np.ndarray:
        """Source values f^k(t, x) on the full grid, shape (K, n, n)."""
        if self.f_fn is not None:
            return self.f_fn(t)
        F = np.einsum("q,mqij->mij", self.tau(t), self.G)
        return np.einsum("km,mij->kij", self.phi, F)


def correlation_sigma(rho: np.ndarray, s1: float, s2: float) -> np.ndarray:
    """sigma^rho with columns sigma_1 = (s1, s2 rho), sigma_2 = (0, s2 sqrt(1 - rho^2)); shape (K, 2, 2)."""
    K = len(rho)
    sig = np.zeros((K, 2, 2))
    sig[:, 0, 0] = s1
    sig[:, 1, 0] = s2 * rho
    sig[:, 0, 1] = 0.0
    sig[:, 1, 1] = s2 * np.sqrt(1.0 - rho * rho)
    return sig


def manufactured(n: int, K: int, rho_lo: float, rho_hi: float, s1: float, s2: float,
                 T: float = 1.0, n_steps: int = 16, control_exact: bool = False) -> Problem:
    """Uncertain-correlation problem on [-2, 2]^2 with u = exp(-t) cos(pi x1/4) cos(pi x2/4).

    control_exact=True subtracts min_k 5 (rho_k - rho*)^2 from f, so that the discrete control
    set attains the continuum infimum and the only error left is the scheme's O(h) + O(dt).
    """
    lo, hi = -2.0, 2.0
    rho = np.linspace(rho_lo, rho_hi, K)
    x = lo + (hi - lo) / (n - 1) * np.arange(n, dtype=np.float64)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    a = math.pi / 4.0
    Phi = np.cos(a * X1) * np.cos(a * X2)
    S12 = np.sin(a * X1) * np.sin(a * X2)
    rstar = 0.8 * np.tanh(X1 * X2)
    G = np.zeros((3, 2, n, n))
    G[0, 0] = 5.0 * rstar * rstar
    G[0, 1] = (0.5 * a * a * (s1 * s1 + s2 * s2) - 1.0) * Phi
    G[1, 0] = -10.0 * rstar
    G[1, 1] = -s1 * s2 * a * a * S12
    G[2, 0] = 5.0
    if control_exact:
        gap = np.min(5.0 * (rho[:, None, None] - rstar[None]) ** 2, axis=0)
        G[0, 0] -= gap
    phi = np.stack([np.ones(K), rho, rho * rho], axis=1)
    g = Phi.copy()
    # psi = u on the boundary, which is exactly 0 there (cos(+-pi/2) rounds to 6e-17 in FP64).
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 0.0

    def psi_fn(t, n=n):
        return np.zeros((n, n))

    def exact(t, Phi=Phi):
        u = math.exp(-t) * Phi
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = 0.0
        return u

    return Problem(name=f"manufactured{n}", n=n, lo=lo, hi=hi, T=T, n_steps=n_steps,
                   sigma=correlation_sigma(rho, s1, s2), phi=phi, G=G,
                   tau_kind=np.array([TAU_ONE, TAU_EXP]), tau_rate=np.array([0.0, -1.0]),
                   g=g, psi_fn=psi_fn, exact=exact, rho=rho, s1=s1, s2=s2)


# Named workloads ------------------------------------------------------------------------

def oracle_scale(truncation_heavy: bool = False) -> Problem:
    """33 x 33 grid, 9 controls rho in [-0.8, 0.8], s1 = 0.3, s2 = 0.2, T = 1, 16 steps.

    The truncation-heavy twin uses s1 = s2 = 1.2 (offsets of about 3.4 cells), so that
    one- and two-sided overstepping of the boundary occurs.
    """
    s = (1.2, 1.2) if truncation_heavy else (0.3, 0.2)
    return manufactured(33, 9, -0.8, 0.8, s[0], s[1], T=1.0, n_steps=16)


def plain_fp64() -> Problem:
    """513 x 513 grid, 33 controls rho in [-0.9, 0.9], s1 = 0.3, s2 = 0.2, T = 1, 64 steps."""
    return manufactured(513, 33, -0.9, 0.9, 0.3, 0.2, T=1.0, n_steps=64)


def mixed_2049(seed: int = 0) -> Problem:
    """2049 x 2049 grid, 65 controls rho in [-0.95, 0.95], (s1, s2) ~ U[0.15, 0.4]^2, 128 steps."""
    rng = np.random.default_rng(seed)
    s1, s2 = rng.uniform(0.15, 0.4, size=2)
    return manufactured(2049, 65, -0.95, 0.95, float(s1), float(s2), T=1.0, n_steps=128)


def scaled(n: int, K: int, n_steps: int, seed: Optional[int] = None, s=(0.3, 0.2),
           rho_range=(-0.9, 0.9), T: float = 1.0) -> Problem:
    """Same family at another size (parity cases between the oracle scale and the full size)."""
    if seed is not None:
        rng = np.random.default_rng(seed)
        s = tuple(rng.uniform(0.15, 0.4, size=2))
    return manufactured(n, K, rho_range[0], rho_range[1], float(s[0]), float(s[1]),
                        T=T, n_steps=n_steps)


def with_dirichlet(p: Problem) -> Problem:
    """The same problem with a non-zero, time-independent Dirichlet boundary
    psi = 0.3 + 0.1 x1 - 0.05 x1 x2 (g takes psi on the boundary)."""
    q = copy.copy(p)
    x = np.linspace(p.lo, p.hi, p.n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    psi = 0.3 + 0.1 * X1 - 0.05 * X2 * X1
    q.psi_fn = lambda t, psi=psi: psi.copy()
    g = p.g.copy()
    g[0, :], g[-1, :], g[:, 0], g[:, -1] = psi[0, :], psi[-1, :], psi[:, 0], psi[:, -1]
    q.g = g
    return q


def gaussian_bump(n: int, lo: float, hi: float, seed: int = 0) -> np.ndarray:
    """Weights of J = sum_x w(x) U(T, x): exp(-|x - c|^2 / (2 r^2)) with centre c ~ U[-1, 1]^2
    and width r ~ U[0.2, 0.5] (seeded), zero on the boundary."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, size=2)
    r = rng.uniform(0.2, 0.5)
    x = np.linspace(lo, hi, n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    w = np.exp(-((X1 - c[0]) ** 2 + (X2 - c[1]) ** 2) / (2.0 * r * r))
    w[0, :] = w[-1, :] = w[:, 0] = w[:, -1] = 0.0
    return w


def sigma_directions(p: Problem) -> np.ndarray:
    """d sigma / d theta for theta = (s1, s2) of the correlation family
    sigma^rho = [[s1, 0], [s2 rho, s2 sqrt(1 - rho^2)]]: shape (2, K, 2, 2)."""
    d = np.zeros((2,) + p.sigma.shape)
    d[0, :, 0, 0] = 1.0
    d[1, :, 1, 0] = p.rho
    d[1, :, 1, 1] = np.sqrt(1.0 - p.rho ** 2)
    return d


def adjoint_1025(seed: int = 0):
    """1025 x 1025 grid, 33 controls rho in [-0.9, 0.9], s1 = 0.3, s2 = 0.2, T = 1, 64 steps,
    and Gaussian-bump weights w (centre and width drawn from `seed`).  Returns (problem, w)."""
    p = manufactured(1025, 33, -0.9, 0.9, 0.3, 0.2, T=1.0, n_steps=64)
    return p, gaussian_bump(p.n, p.lo, p.hi, seed)


def batched(n_inst: int = 256, seed: int = 0, sizes=(65, 129, 257, 513), k_range=(17, 65),
            n_steps: int = 32, T: float = 1.0):
    """Independent instances of the uncertain-correlation family: grid size uniform over
    `sizes`, (s1, s2) ~ U[0.15, 0.4]^2, K ~ U{k_range}, rho in [-0.9, 0.9], n_steps steps."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        n = int(rng.choice(sizes))
        s1, s2 = rng.uniform(0.15, 0.4, size=2)
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        out.append(manufactured(n, K, -0.9, 0.9, float(s1), float(s2), T=T, n_steps=n_steps))
    return out


def unit_circle_controls(n_alpha: int) -> np.ndarray:
    """N_alpha equally spaced points on the unit circle, angles 2 pi k / N_alpha."""
    ang = 2.0 * math.pi * np.arange(n_alpha) / n_alpha
    return np.stack([np.cos(ang), np.sin(ang)], axis=1)


def problem_A(n: int, n_alpha: int = 40, n_steps: int = 1) -> Problem:
    """Problem A of Section 2.4: u = (3/2 - t) sin x1 sin x2 on [-pi, pi]^2, T = 1/2.

    sigma = sqrt(2) (sin(x1 + x2), cos(x1 + x2))^T (P = 1, x-dependent), drift b = alpha on
    the unit circle, c = 0.  The source does not depend on the control; the dangling term in
    the printed source is read as
    (1/2 - t) S1 S2 + (3/2 - t) [sqrt(C1^2 S2^2 + S1^2 C2^2) - 2 sin(x1+x2) cos(x1+x2) C1 C2],
    which satisfies the PDE exactly with inf_alpha alpha . Du = -|Du|.
    """
    lo, hi = -math.pi, math.pi
    alphas = unit_circle_controls(n_alpha)
    x = lo + (hi - lo) / (n - 1) * np.arange(n, dtype=np.float64)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    S1, S2, C1, C2 = np.sin(X1), np.sin(X2), np.cos(X1), np.cos(X2)
    sp, cp = np.sin(X1 + X2), np.cos(X1 + X2)
    K = n_alpha

    def f_fn(t):
        f = (0.5 - t) * S1 * S2 + (1.5 - t) * (np.sqrt(C1 ** 2 * S2 ** 2 + S1 ** 2 * C2 ** 2)
                                             - 2.0 * sp * cp * C1 * C2)
        return np.broadcast_to(f, (K, n, n)).copy()

    def sigma_fn(k, Y1, Y2):
        s = np.empty(Y1.shape + (2, 1))
        s[..., 0, 0] = math.sqrt(2.0) * np.sin(Y1 + Y2)
        s[..., 1, 0] = math.sqrt(2.0) * np.cos(Y1 + Y2)
        return s

    def drift_fn(k, Y1, Y2):
        b = np.empty(Y1.shape + (2,))
        b[..., 0] = alphas[k, 0]
        b[..., 1] = alphas[k, 1]
        return b

    def exact(t):
        u = (1.5 - t) * S1 * S2
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = 0.0
        return u

    g = exact(0.0)
    # The same source in the separable form (phi = 1, tau = (1, t)): with
    # Q = sqrt(C1^2 S2^2 + S1^2 C2^2) - 2 sin(x1+x2) cos(x1+x2) C1 C2,
    # f = (0.5 S1 S2 + 1.5 Q) * 1 - (S1 S2 + Q) * t.  The oracle evaluates f_fn.
    Q = np.sqrt(C1 ** 2 * S2 ** 2 + S1 ** 2 * C2 ** 2) - 2.0 * sp * cp * C1 * C2
    G = np.zeros((1, 2, n, n))
    G[0, 0] = 0.5 * S1 * S2 + 1.5 * Q
    G[0, 1] = -(S1 * S2 + Q)
    p = Problem(name=f"problemA{n}", n=n, lo=lo, hi=hi, T=0.5, n_steps=n_steps, sigma=None,
                phi=np.ones((K, 1)), G=G, tau_kind=[TAU_ONE, TAU_LINEAR], tau_rate=[0.0, 0.0], g=g,
                psi_fn=lambda t: np.zeros((n, n)), exact=exact, sigma_fn=sigma_fn,
                drift_fn=drift_fn, f_fn=f_fn)
    p._K = K
    return p


def problem_B(n: int, n_alpha: int = 40, n_steps: int = 1) -> Problem:
    """Problem B of Section 2.4: u = (2 - t) sin x1 sin x2 on [-pi, pi]^2, T = 1/2.

    sigma = sqrt(2) alpha (P = 1), alpha on the unit circle, b = 0, c = 0,
    f^alpha = (1 - t) S1 S2 - 2 alpha_1 alpha_2 (2 - t) C1 C2.
    """
    lo, hi = -math.pi, math.pi
    alphas = unit_circle_controls(n_alpha)
    x = lo + (hi - lo) / (n - 1) * np.arange(n, dtype=np.float64)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    S1, S2, C1, C2 = np.sin(X1), np.sin(X2), np.cos(X1), np.cos(X2)
    K = n_alpha
    sig = np.zeros((K, 2, 1))
    sig[:, 0, 0] = math.sqrt(2.0) * alphas[:, 0]
    sig[:, 1, 0] = math.sqrt(2.0) * alphas[:, 1]

    def f_fn(t):
        return ((1.0 - t) * S1 * S2)[None] - 2.0 * (alphas[:, 0] * alphas[:, 1])[:, None, None] \
            * ((2.0 - t) * C1 * C2)[None]

    def exact(t):
        u = (2.0 - t) * S1 * S2
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = 0.0
        return u

    # The same source in the separable form f^k = sum_m phi[k, m] sum_q tau_q(t) G[m, q] with
    # phi[k] = (1, alpha_1 alpha_2) and tau = (1, t):
    #   (1 - t) S1 S2 = S1 S2 * 1 - S1 S2 * t,  -2 (2 - t) C1 C2 = -4 C1 C2 * 1 + 2 C1 C2 * t.
    # The oracle evaluates f_fn (the printed form); the library reads G.
    phi = np.stack([np.ones(K), alphas[:, 0] * alphas[:, 1]], axis=1)
    G = np.zeros((2, 2, n, n))
    G[0, 0], G[0, 1] = S1 * S2, -S1 * S2
    G[1, 0], G[1, 1] = -4.0 * C1 * C2, 2.0 * C1 * C2
    return Problem(name=f"problemB{n}", n=n, lo=lo, hi=hi, T=0.5, n_steps=n_steps, sigma=sig,
                   phi=phi, G=G, tau_kind=[TAU_ONE, TAU_LINEAR], tau_rate=[0.0, 0.0],
                   g=exact(0.0), psi_fn=lambda t: np.zeros((n, n)), exact=exact, f_fn=f_fn)
