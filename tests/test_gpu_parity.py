"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle, stage by stage.

Tolerances: 1e-10 relative max-norm for FP64 results, 1e-8 for the mixed path, bit-exact
policies apart from near-ties within 1e-12 relative (lowest index wins on both sides).
Sizes span several 32 x 8 tiles with ragged edges (interior 31, 63, 127, 255 per dimension)
and include the truncation-heavy 33 x 33 case, the degenerate single-control case, the
smallest grid (5 x 5: one level, 9 unknowns), the largest control set (255, the limit of the
one-byte policy), and a case with discount c^k, constant drift b^k and non-zero Dirichlet data.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lisl, multigrid as mg
from tests._gpu_util import TOL_FP64, TOL_MIXED, policies_agree, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_04821_gb300 as slp
    slp.load()   # fails loudly if the library was not built
    return slp


def _solver(prob, **kw):
    import paper_1605_04821_gb300 as slp
    return slp.solver_from_problem(prob, **kw)


CASES = {
    "c33": lambda: W.oracle_scale(False),
    "heavy33": lambda: W.oracle_scale(True),
    "k1_33": lambda: W.manufactured(33, 1, 0.3, 0.3, 0.9, 0.7, T=0.5, n_steps=4),
    "s65": lambda: W.scaled(65, 17, 8, seed=3),
    "s129": lambda: W.scaled(129, 33, 4, s=(0.6, 0.5)),
    "n9": lambda: W.manufactured(9, 3, -0.5, 0.5, 0.8, 0.6, T=0.25, n_steps=2),
    "n5": lambda: W.manufactured(5, 3, -0.5, 0.5, 0.8, 0.6, T=0.25, n_steps=2),
    "k255_33": lambda: W.manufactured(33, 255, -0.95, 0.95, 0.3, 0.2, T=0.25, n_steps=4),
    "cb33": lambda: _discount_drift(W.with_dirichlet(W.manufactured(33, 9, -0.8, 0.8, 1.2, 1.2,
                                                                    T=0.5, n_steps=6))),
}


def _discount_drift(p):
    """Non-zero discount c^k and constant drift b^k (in cells per step) on every control."""
    p.c = np.linspace(-0.5, 0.3, p.K)
    p.drift = np.stack([np.linspace(-2.0, 2.0, p.K), np.linspace(1.5, -1.0, p.K)], axis=1)
    return p


def _perturbed_state(prob, seed=0, amp=0.02):
    rng = np.random.default_rng(seed)
    X = prob.exact(0.3).copy()
    X[1:-1, 1:-1] += amp * rng.standard_normal((prob.n - 2, prob.n - 2))
    return X


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("screen", [0, 1])
def test_argmin_matches_oracle(name, screen):
    prob = CASES[name]()
    s = _solver(prob, argmin_screen=screen)
    t = 0.3
    X = _perturbed_state(prob, seed=1)
    X[0, :] = X[-1, :] = X[:, 0] = X[:, -1] = 0.0
    pol = torch.zeros((prob.n - 2) ** 2, dtype=torch.uint8, device="cuda")
    s.improve(to_dev(X), t, pol)
    V = lisl.control_values(prob, X, t)
    ok, ndiff = policies_agree(pol.cpu().numpy(), lisl.improve(V), V)
    assert ok, f"{ndiff} policy entries differ beyond the tie window"


def _random_policy(prob, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, prob.K, size=(prob.n - 2) ** 2)


@pytest.mark.parametrize("name", ["c33", "heavy33", "s65", "s129", "n9", "n5", "k255_33", "cb33"])
@pytest.mark.parametrize("precision", [0, 1])
def test_operators_on_every_level(name, precision):
    prob = CASES[name]()
    s = _solver(prob, precision=precision)
    dt = prob.dt
    pol = _random_policy(prob, 5)
    # smooth policy blocks too, so that class rows exist on the coarse levels
    if name in ("s65", "s129"):
        n = prob.n - 2
        pol = (np.arange(n)[None, :] // 16 + np.arange(n)[:, None] // 24).ravel() % prob.K
    s.set_policy(to_dev(pol, torch.uint8))
    s.build_hierarchy(dt)
    A, _ = lisl.assemble(prob, pol, prob.g, 0.0, dt)
    H = mg.galerkin_hierarchy(A, prob.n, s.num_levels())
    rng = np.random.default_rng(11)
    dtype = torch.float64 if precision == 0 else torch.float32
    tol = 1e-12 if precision == 0 else 2e-6
    for level in range(s.num_levels()):
        nl = H.n[level]
        x = np.zeros((nl, nl))
        x[1:-1, 1:-1] = rng.standard_normal((nl - 2, nl - 2))
        y = torch.zeros((nl, nl), dtype=dtype, device="cuda")
        s.apply(level, to_dev(x, dtype), y)
        ref = H.A[level] @ x[1:-1, 1:-1].ravel()
        got = y.double().cpu().numpy()[1:-1, 1:-1].ravel()
        assert rel_maxnorm(got, ref) <= tol, f"level {level}"


@pytest.mark.parametrize("name", ["s65", "s129"])
def test_level_stats_describe_the_galerkin_operators(name):
    """sl_hjb_level_stats against the oracle's R A P matrices: every non-zero lies within the
    reported reach of its row, and the class and explicit non-zeros cover the oracle's
    significant entries.  The counts are not compared exactly: an entry that cancels to zero
    in exact arithmetic is a rounding residue of either sign or an exact zero depending on the
    order of the Galerkin sums, which differs between the two sides (about 4 % of the entries
    on the first coarse level of the 65^2 case)."""
    prob = CASES[name]()
    s = _solver(prob, precision=0)
    n = prob.n - 2
    pol = (np.arange(n)[None, :] // 16 + np.arange(n)[:, None] // 24).ravel() % prob.K
    s.set_policy(to_dev(pol, torch.uint8))
    s.build_hierarchy(prob.dt)
    A, _ = lisl.assemble(prob, pol, prob.g, 0.0, prob.dt)
    H = mg.galerkin_hierarchy(A, prob.n, s.num_levels())
    st0 = s.level_stats(0)
    assert st0["n"] == prob.n and st0["class_nnz"] == -1 and st0["explicit_rows"] == 0
    for level in range(1, s.num_levels()):
        st = s.level_stats(level)
        m = H.n[level] - 2
        assert st["n"] == H.n[level]
        assert st["explicit_entries"] == st["explicit_rows"] * (2 * st["reach"] + 1) ** 2
        assert 0 <= st["explicit_nnz"] <= st["explicit_entries"]
        Al = H.A[level].tocoo()
        nz = np.abs(Al.data) > 0
        r, c = Al.row[nz], Al.col[nz]
        assert np.all(np.abs(r % m - c % m) <= st["reach"]), level
        assert np.all(np.abs(r // m - c // m) <= st["reach"]), level
        got = st["class_nnz"] + st["explicit_nnz"]
        big = int((np.abs(Al.data) > 1e-12 * np.abs(Al.data).max()).sum())
        assert big <= got <= 1.1 * nz.sum(), (level, st, big, int(nz.sum()))
        assert s.level_info(level) == (st["n"], st["explicit_rows"], got)


@pytest.mark.parametrize("name", ["c33", "heavy33", "s65", "s129", "cb33"])
def test_vcycle_matches_oracle(name):
    prob = CASES[name]()
    s = _solver(prob, precision=0)
    dt = prob.dt
    n = prob.n - 2
    pol = (np.arange(n)[None, :] // 12 + 2 * (np.arange(n)[:, None] // 20)).ravel() % prob.K
    s.set_policy(to_dev(pol, torch.uint8))
    s.build_hierarchy(dt)
    A, _ = lisl.assemble(prob, pol, prob.g, 0.0, dt)
    H = mg.galerkin_hierarchy(A, prob.n, s.num_levels())
    rng = np.random.default_rng(2)
    b = np.zeros((prob.n, prob.n))
    b[1:-1, 1:-1] = rng.standard_normal((n, n))
    x = torch.zeros((prob.n, prob.n), dtype=torch.float64, device="cuda")
    s.vcycle(to_dev(b), x)
    ref = mg.vcycle(H, b[1:-1, 1:-1].ravel(), 2, 2, 0.8)
    assert rel_maxnorm(x.cpu().numpy()[1:-1, 1:-1].ravel(), ref) <= 1e-11


@pytest.mark.parametrize("name", ["c33", "heavy33", "s65", "s129", "cb33"])
@pytest.mark.parametrize("precision", [0, 1])
def test_linear_solve_matches_direct_solve(name, precision):
    prob = CASES[name]()
    s = _solver(prob, precision=precision)
    dt, t = prob.dt, prob.dt
    pol = _random_policy(prob, 9)
    s.set_policy(to_dev(pol, torch.uint8))
    U = prob.g
    A, F = lisl.assemble(prob, pol, U, t, dt)
    ref = lisl.direct_solve(A, F)
    x = to_dev(U)
    s.linear_solve(to_dev(U), x, t, dt)
    got = x.cpu().numpy()[1:-1, 1:-1].ravel()
    assert rel_maxnorm(got, ref) <= (TOL_FP64 if precision == 0 else TOL_MIXED)


@pytest.mark.parametrize("name", ["c33", "heavy33", "k1_33", "s65", "s129", "n9", "n5", "k255_33",
                                  "cb33"])
@pytest.mark.parametrize("precision", [0, 1])
def test_full_solve_matches_oracle(name, precision):
    prob = CASES[name]()
    s = _solver(prob, precision=precision, argmin_screen=precision)
    ref = lisl.solve(prob)
    u = to_dev(prob.g)
    pol = torch.zeros((prob.n - 2) ** 2, dtype=torch.uint8, device="cuda")
    stats = s.solve(u, 0.0, prob.T, prob.n_steps, pol)
    err = rel_maxnorm(u.cpu().numpy(), ref.U)
    assert err <= (TOL_FP64 if precision == 0 else TOL_MIXED), (err, stats)
    # final policy: equal apart from near-ties of the last improvement
    V = lisl.control_values(prob, ref.U, prob.T)
    ok, nd = policies_agree(pol.cpu().numpy(), ref.policies[-1], V)
    assert ok, nd
    assert stats["steps"] == prob.n_steps


def test_step_by_step_policies_and_iterations():
    prob = CASES["heavy33"]()
    s = _solver(prob, precision=0)
    ref = lisl.solve(prob)
    u = to_dev(prob.g)
    pol = torch.zeros((prob.n - 2) ** 2, dtype=torch.uint8, device="cuda")
    dt = prob.dt
    U = prob.g.copy()
    for step in range(prob.n_steps):
        s.step(u, (step + 1) * dt, dt, pol)
        r = lisl.howard_step(prob, U, (step + 1) * dt, dt,
                             policy0=None if step == 0 else ref.policies[step - 1])
        U = r.X
        assert rel_maxnorm(u.cpu().numpy(), r.X) <= TOL_FP64
        V = lisl.control_values(prob, r.X, (step + 1) * dt)
        ok, nd = policies_agree(pol.cpu().numpy(), r.policy, V)
        assert ok, (step, nd)
