"""Failure statuses of the library, provoked on the host side (bad arguments, a violated CFL
bound, an iteration cap reached, a NaN in the input), never by a GPU fault: every call
returns its status, and the CUDA context stays usable, so a correct solve right afterwards
still matches the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import lisl
from tests._gpu_util import TOL_FP64, TOL_MIXED, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _check_context_still_works(S):
    p = W.manufactured(17, 3, -0.5, 0.5, 0.8, 0.6, T=0.25, n_steps=2)
    sol = S.solver_from_problem(p)
    u = to_dev(p.g)
    sol.solve(u, 0.0, p.T, p.n_steps)
    assert rel_maxnorm(u.cpu().numpy(), lisl.solve(p).U) <= TOL_FP64
    sol.close()


def test_invalid_arguments_are_refused():
    S = _lib()
    with pytest.raises(S.SLError) as e:   # coarsest level of a 20 x 20 grid is too large
        S.solver_from_problem(W.manufactured(20, 3, -0.5, 0.5, 0.8, 0.6))
    assert e.value.status == S.SL_EINVAL
    p = W.manufactured(17, 3, -0.5, 0.5, 0.8, 0.6)
    with pytest.raises(S.SLError):
        S.solver_from_problem(p, precision=2)
    with pytest.raises(S.SLError):
        S.solver_from_problem(p, precond=3)
    with pytest.raises(S.SLError):
        S.solver_from_problem(p, ir_recursive=-1)
    sol = S.solver_from_problem(p)
    with pytest.raises(S.SLError) as e:
        sol.step(to_dev(p.g), 0.1, -0.1)
    assert e.value.status == S.SL_EINVAL
    with pytest.raises(S.SLError) as e:   # adjoint without a recorded march
        sol.adjoint(to_dev(p.g), to_dev(np.zeros_like(p.g)))
    assert e.value.status == S.SL_EINVAL
    sol.close()
    _check_context_still_works(S)


def test_cfl_violation():
    S = _lib()
    p = W.manufactured(17, 3, -0.5, 0.5, 0.8, 0.6, T=0.25, n_steps=2)
    p.c = np.full(p.K, 100.0)   # dt * c = 12.5 > 1
    sol = S.solver_from_problem(p)
    with pytest.raises(S.SLError) as e:
        sol.solve(to_dev(p.g), 0.0, p.T, p.n_steps)
    assert e.value.status == S.SL_ECFL
    sol.close()
    _check_context_still_works(S)


@pytest.mark.parametrize("precision", [0, 1])
def test_krylov_cap_reached(precision):
    S = _lib()
    p = W.oracle_scale(True)
    kw = dict(kry_max=1, krylov_tol=1e-15) if precision == 0 else dict(ir_max=0, kry_max=1, krylov_tol=1e-15)
    sol = S.solver_from_problem(p, precision=precision, **kw)
    with pytest.raises(S.SLError) as e:
        sol.solve(to_dev(p.g), 0.0, p.T, p.n_steps)
    assert e.value.status == S.SL_ENOCONV_KRYLOV
    sol.close()
    _check_context_still_works(S)


def test_howard_cap_reached():
    S = _lib()
    p = W.oracle_scale(True)
    sol = S.solver_from_problem(p, pi_max=1, pi_tol=0.0)
    with pytest.raises(S.SLError) as e:
        sol.solve(to_dev(p.g), 0.0, p.T, p.n_steps)
    assert e.value.status == S.SL_ENOCONV_PI
    sol.close()
    _check_context_still_works(S)


def test_nan_input_is_reported():
    S = _lib()
    p = W.oracle_scale(False)
    g = p.g.copy()
    g[10, 12] = np.nan
    sol = S.solver_from_problem(p)
    with pytest.raises(S.SLError) as e:
        sol.solve(to_dev(g), 0.0, p.T, p.n_steps)
    assert e.value.status == S.SL_ENAN
    sol.close()
    _check_context_still_works(S)


_BREAKDOWN_REF = {}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("use_graphs", [0, 1, 2])
def test_bicgstab_breakdown_restarts(precision, use_graphs):
    """SL_EBREAKDOWN is handled inside the solves: a breakdown marked on the first BiCGSTAB
    iteration of the march (sl_hjb_inject_breakdown, as if rho had vanished) sends the solve
    back to its true residual.  The march still ends with SL_OK and meets the oracle; it is not
    bit-identical to the unmarked march (the restart changes the iterates), while a mark that
    is cancelled before the march leaves it bit-identical.  The inner tolerance is tightened so
    that no first FP32 iteration can meet its stop test (a mark on a converging iteration has
    no effect)."""
    import torch
    S = _lib()
    p = W.oracle_scale(True)
    if "U" not in _BREAKDOWN_REF:
        _BREAKDOWN_REF["U"] = lisl.solve(p).U
    kw = dict(precision=precision, use_graphs=use_graphs)
    if precision == 1:
        kw["inner_tol"] = 1e-6
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    runs = {}
    for mark in ("none", "first", "cancelled"):
        sol = S.solver_from_problem(p, **kw)
        if mark == "first":
            sol.inject_breakdown(1)
        elif mark == "cancelled":
            sol.inject_breakdown(3)
            sol.inject_breakdown(0)
        u = to_dev(p.g)
        st = sol.solve(u, 0.0, p.T, p.n_steps)
        sol.close()
        assert rel_maxnorm(u.cpu().numpy(), _BREAKDOWN_REF["U"]) <= tol, (mark, st)
        runs[mark] = (u, st)
    assert not torch.equal(runs["first"][0], runs["none"][0])
    assert torch.equal(runs["cancelled"][0], runs["none"][0])
    assert runs["cancelled"][1]["krylov_iters"] == runs["none"][1]["krylov_iters"]
    assert runs["first"][1]["steps"] == runs["none"][1]["steps"] == p.n_steps
