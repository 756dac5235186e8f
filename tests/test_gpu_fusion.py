"""The fused coarse-level passes of the V-cycle (sl_opts.coarse_fusion = 1: pre-smoothing,
residual and full-weighting restriction in one launch; prolongation and the first
post-smoothing sweep in another) against one launch per operation (coarse_fusion = 0).

The fused kernels compute every value with the same operations in the same order as the
one-pass kernels, so the results must agree bit for bit: single V-cycles in both precisions,
with V(1,1) and V(2,2), on grids whose coarse levels take every tile height (32, 16 and 8
rows), with class rows, explicit rows and wide stencils (the 2049^2 workload), the x-dependent
diffusion of Problem A (all coarse rows explicit), and whole marches.  The oracle parity of
the fused cycle is covered by the V-cycle and full-solve tests, which run with the default.
"""
import numpy as np
import pytest

import workloads as W
from tests._gpu_util import to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _policy(m, K, seed):
    rng = np.random.default_rng(seed)
    base = (np.arange(m)[None, :] // 13 + 3 * (np.arange(m)[:, None] // 17)).ravel() % K
    noise = rng.integers(0, K, size=m * m)
    return np.where(rng.random(m * m) < 0.05, noise, base).astype(np.uint8)


def _cycles(prob, precision, nu, **kw):
    S = _lib()
    n = prob.n
    pol = to_dev(_policy(n - 2, prob.K, n), torch.uint8)
    rng = np.random.default_rng(n + 3)
    b = np.zeros((n, n))
    b[1:-1, 1:-1] = rng.standard_normal((n - 2, n - 2))
    dtype = torch.float64 if precision == 0 else torch.float32
    out = []
    for fusion in (0, 1):
        s = S.solver_from_problem(prob, precision=precision, nu1=nu, nu2=nu, coarse_fusion=fusion, **kw)
        s.set_policy(pol)
        s.build_hierarchy(prob.dt)
        x = torch.zeros((n, n), dtype=dtype, device="cuda")
        s.vcycle(to_dev(b, dtype), x)
        torch.cuda.synchronize()
        out.append(x)
        s.close()
    return out


@pytest.mark.parametrize("n", [65, 257, 513, 1025])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_fused_equals_unfused(n, precision, nu):
    prob = W.scaled(n, 17, 4, s=(0.35, 0.25), seed=n)
    a, b = _cycles(prob, precision, nu)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b)


def test_vcycle_fused_equals_unfused_2049():
    prob = W.mixed_2049(seed=0)
    a, b = _cycles(prob, 1, 1, argmin_screen=1)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_vcycle_fused_equals_unfused_general_fine_level(precision):
    """Problem A (x-dependent sigma): every coarse row is explicit."""
    a, b = _cycles(W.problem_A(81), precision, 2)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_march_fused_equals_unfused(precision):
    S = _lib()
    prob = W.scaled(257, 33, 4, seed=9)
    prob.T = 4.0 / 64
    outs = []
    for fusion in (0, 1):
        s = S.solver_from_problem(prob, precision=precision, argmin_screen=precision, coarse_fusion=fusion)
        u = to_dev(prob.g)
        st = s.solve(u, 0.0, prob.T, prob.n_steps)
        s.close()
        outs.append((u, st))
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1]["krylov_iters"] == outs[1][1]["krylov_iters"]


@pytest.mark.parametrize("n", [129, 513])
@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycle_tail_matches_level_by_level_cycle(n, smoother):
    """The single-block tail (levels of at most 1024 rows; in shared memory when they fit, as
    here) against the same levels run one launch per operation: equal to FP32 rounding (the
    explicit rows sum their windows in another order)."""
    S = _lib()
    prob = W.scaled(n, 17, 4, seed=n + 1)
    pol = to_dev(_policy(n - 2, prob.K, n), torch.uint8)
    rng = np.random.default_rng(n)
    b = np.zeros((n, n))
    b[1:-1, 1:-1] = rng.standard_normal((n - 2, n - 2))
    out = []
    for tail in (1024, 0):
        kw = dict(omega=1.0) if smoother == 1 else {}
        s = S.solver_from_problem(prob, precision=1, smoother=smoother, coarse_tail_rows=tail, **kw)
        s.set_policy(pol)
        s.build_hierarchy(prob.dt)
        x = torch.zeros((n, n), dtype=torch.float32, device="cuda")
        s.vcycle(to_dev(b, torch.float32), x)
        torch.cuda.synchronize()
        out.append(x.double())
        s.close()
    a, c = out
    assert torch.isfinite(a).all()
    assert float((a - c).abs().max() / c.abs().max()) <= 1e-5
