"""Coefficient callbacks (sl_field_cb) through the C ABI.

Eqs. 1.1-1.3 let f and psi be general functions of (t, x).  These tests pass data that the
separable form cannot express, through callbacks that the library calls at each step's t_n:

* Problem A of Section 2.4 with its printed source (the form read in the workloads module),
  evaluated on the device by a torch callback, against the oracle, which evaluates the same
  printed formula (f_fn), element by element: 1e-10 in FP64, 1e-8 in mixed precision.
* The manufactured uncertain-correlation problem with a time-dependent, non-separable
  Dirichlet datum psi(t, x) = 0.2 sin(x1 + 2 t) + 0.1 cos(t x2) from a callback that uploads
  host values, against the oracle with the same psi.
* The callbacks are called once per source table and step, at t_n = t0 + n dt.
"""
import copy
import math

import numpy as np
import pytest

import workloads as W
from oracle import lisl
from tests._gpu_util import TOL_FP64, TOL_MIXED, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _problem_a_source(n, lo, hi, calls):
    """The printed Problem A source, (1/2 - t) S1 S2 + (3/2 - t) [sqrt(C1^2 S2^2 + S1^2 C2^2)
    - 2 sin(x1 + x2) cos(x1 + x2) C1 C2], computed on the device at the callback's t."""
    x = lo + (hi - lo) / (n - 1) * torch.arange(n, dtype=torch.float64, device="cuda")
    X2, X1 = torch.meshgrid(x, x, indexing="ij")
    S1, S2, C1, C2 = torch.sin(X1), torch.sin(X2), torch.cos(X1), torch.cos(X2)
    sp, cp = torch.sin(X1 + X2), torch.cos(X1 + X2)
    Q = torch.sqrt(C1 ** 2 * S2 ** 2 + S1 ** 2 * C2 ** 2) - 2.0 * sp * cp * C1 * C2

    def fn(t, m, out):
        calls.append((t, m))
        out.copy_((0.5 - t) * S1 * S2 + (1.5 - t) * Q)
    return fn


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,steps", [(41, 1), (81, 1), (81, 3)])
def test_problem_a_printed_source_through_a_callback(n, steps, precision):
    S = _lib()
    p = W.problem_A(n, n_alpha=40, n_steps=steps)
    ref = lisl.solve(p)                       # evaluates the printed source (f_fn)
    args, kw = S._problem_args(p, torch.device("cuda"))
    args = list(args)
    args[5] = None                            # no separable tables: the callback gives F_0
    calls = []
    sol = S.Solver(*args, **kw, f_cb=_problem_a_source(p.n, p.lo, p.hi, calls),
                   precision=precision, argmin_screen=precision)
    u = to_dev(p.g)
    sol.solve(u, 0.0, p.T, p.n_steps)
    torch.cuda.synchronize()
    assert rel_maxnorm(u.cpu().numpy(), ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)
    dt = p.T / p.n_steps
    assert [m for _, m in calls] == [0] * steps
    assert np.allclose([t for t, _ in calls], dt * np.arange(1, steps + 1), rtol=0, atol=1e-15)
    sol.close()


def _psi(t, X1, X2):
    return 0.2 * np.sin(X1 + 2.0 * t) + 0.1 * np.cos(t * X2)


@pytest.mark.parametrize("precision", [0, 1])
def test_time_dependent_boundary_through_a_callback(precision):
    S = _lib()
    p = copy.copy(W.oracle_scale(truncation_heavy=True))
    p.n_steps, p.T = 6, 0.5
    X1, X2 = p.coords()
    p.psi_fn = lambda t: _psi(t, X1, X2)
    g = p.g.copy()
    b = _psi(0.0, X1, X2)
    g[0, :], g[-1, :], g[:, 0], g[:, -1] = b[0, :], b[-1, :], b[:, 0], b[:, -1]
    p.g = g
    ref = lisl.solve(p)
    calls = []

    def psi_cb(t, m, out):
        calls.append((t, m))
        out.copy_(torch.as_tensor(_psi(t, X1, X2), device="cuda"))

    args, kw = S._problem_args(p, torch.device("cuda"))
    kw.pop("Psi", None)
    sol = S.Solver(*args, **kw, psi_cb=psi_cb, precision=precision, argmin_screen=precision)
    u = to_dev(p.g)
    sol.solve(u, 0.0, p.T, p.n_steps)
    torch.cuda.synchronize()
    U = u.cpu().numpy()
    assert rel_maxnorm(U, ref.U) <= (TOL_FP64 if precision == 0 else TOL_MIXED)
    # the boundary carries psi(T)
    assert np.array_equal(U[0, :], ref.U[0, :]) and np.array_equal(U[:, -1], ref.U[:, -1])
    dt = p.T / p.n_steps
    assert np.allclose([t for t, _ in calls], dt * np.arange(1, p.n_steps + 1), rtol=0, atol=1e-15)
    sol.close()


def test_callback_error_is_raised_after_the_call():
    S = _lib()
    p = W.problem_A(41, n_alpha=8, n_steps=1)
    args, kw = S._problem_args(p, torch.device("cuda"))
    args = list(args)
    args[5] = None

    def bad(t, m, out):
        raise ValueError("no source here")

    sol = S.Solver(*args, **kw, f_cb=bad)
    u = to_dev(p.g)
    with pytest.raises(RuntimeError, match="callback"):
        sol.solve(u, 0.0, p.T, 1)
    sol.close()
