"""Two-colour (red-black) Gauss-Seidel smoothing (sl_opts.smoother = 1) on the GPU against the
oracle: one V-cycle element by element (FP64 at 1e-11; FP32 with the single-block tail on the
coarse levels, within the FP32 rounding of a cycle), and full Howard marches at 1e-10 (FP64)
and 1e-8 (mixed)."""
import numpy as np
import pytest

from oracle import lisl, multigrid as mg
from tests._gpu_util import TOL_FP64, TOL_MIXED, rel_maxnorm, to_dev
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(prob, **kw):
    import paper_1605_04821_gb300 as S
    S.load()
    return S.solver_from_problem(prob, smoother=1, omega=1.0, **kw)


@pytest.mark.parametrize("name", ["c33", "heavy33", "s65", "s129", "cb33"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5)])
def test_vcycle_rbgs_matches_oracle(name, precision, tol):
    prob = CASES[name]()
    s = _solver(prob, precision=precision, coarse_tail_rows=(0 if precision == 0 else 1024))
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
    dtype = torch.float64 if precision == 0 else torch.float32
    x = torch.zeros((prob.n, prob.n), dtype=dtype, device="cuda")
    s.vcycle(to_dev(b, dtype), x)
    ref = mg.vcycle(H, b[1:-1, 1:-1].ravel(), 2, 2, 1.0, smoother="rbgs")
    assert rel_maxnorm(x.double().cpu().numpy()[1:-1, 1:-1].ravel(), ref) <= tol
    s.close()


@pytest.mark.parametrize("name", ["c33", "heavy33", "s65", "cb33"])
@pytest.mark.parametrize("precision", [0, 1])
def test_full_solve_rbgs_matches_oracle(name, precision):
    prob = CASES[name]()
    s = _solver(prob, precision=precision, argmin_screen=precision)
    u = to_dev(prob.g)
    st = s.solve(u, 0.0, prob.T, prob.n_steps)
    ref = lisl.solve(prob)
    assert rel_maxnorm(u.cpu().numpy(), ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)
    assert st["graph_steps"] == prob.n_steps
    s.close()
