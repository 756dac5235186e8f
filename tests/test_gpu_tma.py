"""The FP32 fine-level operator with TMA-staged tiles (k_fine_op_tma, sl_opts.fine_tma = 1)
against the same operator with tiles staged by the threads (fine_tma = 0).

Both compute every row with the same device function from the same staged values, so the
outputs must agree bit for bit: the FP32 apply y = A x on random vectors, one V-cycle (its
fine level runs the Jacobi and residual variants), and a whole mixed-precision march, on grids
with interior tiles (bulk copies) and boundary tiles (staged by the threads), including a wide
stencil (a halo of about seven nodes at 257^2 with s = 1.2) and the 2049^2 grid.
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


def _pair(p, **kw):
    S = _lib()
    out = []
    for tma in (0, 1):
        out.append(S.solver_from_problem(p, precision=1, argmin_screen=1, fine_tma=tma, **kw))
    return out


def _policy(p, seed):
    rng = np.random.default_rng(seed)
    m = p.n - 2
    base = (np.arange(m)[None, :] // 7 + 3 * (np.arange(m)[:, None] // 11)).ravel() % p.K
    noise = rng.integers(0, p.K, size=m * m)
    pol = np.where(rng.random(m * m) < 0.1, noise, base).astype(np.uint8)
    return torch.as_tensor(pol, device="cuda")


@pytest.mark.parametrize("n,s", [(129, (0.3, 0.2)), (257, (1.2, 1.2)), (513, (0.3, 0.2)),
                                 (1025, (0.35, 0.25)), (2049, (0.3092, 0.2174))])
def test_apply_and_vcycle_bit_identical(n, s):
    p = W.scaled(n, 33, 4, s=s)
    a, b = _pair(p)
    pol = _policy(p, n)
    rng = np.random.default_rng(n + 1)
    x = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    x[1:-1, 1:-1] = torch.as_tensor(rng.standard_normal((n - 2, n - 2)), dtype=torch.float32, device="cuda")
    ys = []
    for sol in (a, b):
        sol.set_policy(pol)
        sol.build_hierarchy(p.dt)
        y = torch.full_like(x, float("nan"))
        y[0, :] = y[-1, :] = y[:, 0] = y[:, -1] = 0.0
        sol.apply(0, x, y)
        v = torch.zeros_like(x)
        sol.vcycle(x, v)
        torch.cuda.synchronize()
        ys.append((y, v))
    assert torch.isfinite(ys[0][0]).all()
    assert torch.equal(ys[0][0], ys[1][0])
    assert torch.equal(ys[0][1], ys[1][1])
    a.close()
    b.close()


@pytest.mark.parametrize("n", [257, 513])
def test_march_bit_identical(n):
    p = W.scaled(n, 33, 4, seed=7)
    p.T = 4.0 / 64
    outs = []
    for sol in _pair(p):
        u = to_dev(p.g)
        st = sol.solve(u, 0.0, p.T, p.n_steps)
        sol.close()
        outs.append((u, st))
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1]["krylov_iters"] == outs[1][1]["krylov_iters"]
