"""Device-driven steps (use_graphs 2): each implicit step is one CUDA-graph launch whose Howard,
refinement and BiCGSTAB loops are conditional graph nodes with their tests on the device.

The graph runs the kernels of the host-driven step in the same order on the same buffers, so
the two modes must agree bit for bit: the state U after every step, the final policy and the
iteration counts.  Every step of mode 2 must have run as a graph launch (graph_steps), and the
result must also match the oracle.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import lisl
from tests._gpu_util import TOL_FP64, TOL_MIXED, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(name):
    if name == "c33":
        p = W.oracle_scale(False)
    elif name == "heavy33":
        p = W.oracle_scale(True)
    elif name == "cb33":
        p = W.with_dirichlet(W.oracle_scale(True))
        p.c = np.linspace(-0.5, 0.3, p.K)
        p.drift = np.stack([np.linspace(-2.0, 2.0, p.K), np.linspace(1.5, -1.0, p.K)], axis=1)
    else:
        p = W.scaled(129, 33, 6, seed=4)
    p = copy.copy(p)
    p.n_steps = min(p.n_steps, 6)
    p.T = 0.25
    return p


def _march(p, mode, precision, **kw):
    import paper_1605_04821_gb300 as S
    S.load()
    sol = S.solver_from_problem(p, precision=precision, argmin_screen=precision, use_graphs=mode, **kw)
    u = to_dev(p.g)
    m = p.n - 2
    pol = torch.empty(m * m, dtype=torch.uint8, device="cuda")
    dt = p.T / p.n_steps
    us, stats = [], []
    for i in range(1, p.n_steps + 1):
        stats.append(sol.step(u, i * dt, dt, policy_out=pol))
        us.append(u.clone())
    sol.close()
    return us, pol.clone(), stats


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["c33", "heavy33", "cb33", "s129"])
def test_graph_steps_equal_host_steps(name, precision):
    p = _case(name)
    u1, pol1, st1 = _march(p, 1, precision)
    u2, pol2, st2 = _march(p, 2, precision)
    for i, (a, b) in enumerate(zip(u1, u2)):
        assert torch.equal(a, b), f"step {i + 1} differs"
    assert torch.equal(pol1, pol2)
    for a, b in zip(st1, st2):
        for key in ("pi_iters", "krylov_iters", "ir_iters", "rebuilds", "policy_changes"):
            assert a[key] == b[key], (key, a[key], b[key])
        assert a["graph_steps"] == 0 and b["graph_steps"] == 1
    ref = lisl.solve(p)
    assert rel_maxnorm(u2[-1].cpu().numpy(), ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("opts", [dict(howard_init=1), dict(howard_loose_tol=1e-6),
                                  dict(howard_init=1, howard_loose_tol=1e-6),
                                  dict(ir_recursive=0), dict(ir_recursive=1)])
def test_howard_variants_graph_equal_host_and_match_the_oracle(opts, precision):
    """The Howard start (sl_opts.howard_init), the loose first solve (howard_loose_tol) and the
    refinement rounds on the inner solve's own residual (ir_recursive; the default is 3) run the
    same way in both modes and reach the oracle's solution: the last solve of every step stays
    at krylov_tol and its policy is the improvement of its result."""
    p = _case("s129")
    u1, pol1, st1 = _march(p, 1, precision, **opts)
    u2, pol2, st2 = _march(p, 2, precision, **opts)
    for i, (a, b) in enumerate(zip(u1, u2)):
        assert torch.equal(a, b), f"step {i + 1} differs"
    assert torch.equal(pol1, pol2)
    for a, b in zip(st1, st2):
        for key in ("pi_iters", "krylov_iters", "ir_iters", "rebuilds", "policy_changes"):
            assert a[key] == b[key], (key, a[key], b[key])
    ref = lisl.solve(p)
    assert rel_maxnorm(u2[-1].cpu().numpy(), ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)
    if "howard_loose_tol" in opts:  # every step solved at least twice (loose, then tight)
        assert all(st["pi_iters"] >= 2 for st in st2)


def test_graph_solve_counts_every_step():
    import paper_1605_04821_gb300 as S
    S.load()
    p = _case("heavy33")
    sol = S.solver_from_problem(p, precision=1, argmin_screen=1)
    assert sol.opts.use_graphs == 2
    u = to_dev(p.g)
    st = sol.solve(u, 0.0, p.T, p.n_steps)
    assert st["graph_steps"] == p.n_steps == st["steps"]
    sol.close()


def test_step_size_change_recaptures():
    """A new step size is captured again (the graph holds dt); the march stays equal to the
    host-driven one."""
    import paper_1605_04821_gb300 as S
    S.load()
    p = _case("c33")
    outs = []
    for mode in (1, 2):
        sol = S.solver_from_problem(p, use_graphs=mode)
        u = to_dev(p.g)
        t = 0.0
        for dt in (0.05, 0.05, 0.02, 0.05):
            t += dt
            sol.step(u, t, dt)
        outs.append(u)
        sol.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["heavy33", "s129"])
def test_argmin_skip_keeps_every_decision(name, mode):
    """sl_opts.argmin_skip: re-deciding only the nodes whose margin does not cover the move of X
    since the step's last improvement gives the policies, states and counts of re-deciding every
    node, bit for bit."""
    p = _case(name)
    u0, pol0, st0 = _march(p, mode, 1, argmin_skip=0)
    u1, pol1, st1 = _march(p, mode, 1, argmin_skip=1)
    for i, (a, b) in enumerate(zip(u0, u1)):
        assert torch.equal(a, b), f"step {i + 1} differs"
    assert torch.equal(pol0, pol1)
    for a, b in zip(st0, st1):
        for key in ("pi_iters", "krylov_iters", "ir_iters", "rebuilds", "policy_changes"):
            assert a[key] == b[key], (key, a[key], b[key])


def test_argmin_skip_on_the_2049_workload():
    """The same on three steps of the 2049^2, 65-control workload, where most nodes keep their
    control in the improvement that follows each step's tight solve."""
    import paper_1605_04821_gb300 as S
    S.load()
    p = W.mixed_2049(seed=0)
    dt = 1.0 / 128
    outs = []
    for skip in (0, 1):
        sol = S.solver_from_problem(p, precision=1, argmin_screen=1, argmin_skip=skip)
        u = to_dev(p.g)
        m = p.n - 2
        pol = torch.empty(m * m, dtype=torch.uint8, device="cuda")
        sts = [sol.step(u, i * dt, dt, policy_out=pol) for i in range(1, 4)]
        sol.close()
        outs.append((u, pol, sts))
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    for a, b in zip(outs[0][2], outs[1][2]):
        assert a["pi_iters"] == b["pi_iters"] and a["policy_changes"] == b["policy_changes"]
