"""Full-size checks: the 2049^2, 65-control workload in the launch configuration of the
benchmark (V(1,1) cycles, FP32 argmin screen in mixed precision), node by node against the
oracle at sampled nodes.

After each of the first two implicit steps the discrete HJB equation
max_k (A^k X - F^k)_j = X_j - U^{n-1}_j - dt min_k v_k(j) = 0 (Eq. 1.10) must hold at
every sampled node j, with v_k(j) evaluated by the oracle from the GPU's U^{n-1} and X = U^n,
and the GPU's final policy must be the oracle's argmin there (apart from near-ties).  The
samples are random interior nodes, the corners, nodes of the truncation band and nodes on the
policy's switching curves.  The mixed path must stay within 1e-8 of the FP64 path everywhere.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lisl
from tests._gpu_util import policies_agree, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu

HJB_RES_TOL = 1e-10   # |residual_j| / max(1, ||U^n||_inf)


def _samples(n, pol, B, seed):
    m = n - 2
    rng = np.random.default_rng(seed)
    i1 = list(rng.integers(1, n - 1, 2000))
    i2 = list(rng.integers(1, n - 1, 2000))
    for c1 in (1, m):
        for c2 in (1, m):
            i1.append(c1)
            i2.append(c2)
    band = rng.integers(1, B + 1, 200)
    along = rng.integers(1, n - 1, 200)
    i1 += list(band) + list(along)
    i2 += list(along) + list(n - 1 - band)
    P = pol.reshape(m, m)
    sw = np.argwhere(P[:, 1:] != P[:, :-1])
    pick = sw[rng.permutation(len(sw))[:500]]
    i2 += list(pick[:, 0] + 1)
    i1 += list(pick[:, 1] + 1)
    return np.array(i1, dtype=np.int64), np.array(i2, dtype=np.int64)


@pytest.fixture(scope="module")
def runs():
    import torch

    import paper_1605_04821_gb300 as slp
    slp.load()
    prob = W.mixed_2049(seed=0)
    dt = 1.0 / 128
    out = {}
    for prec in (1, 0):
        s = slp.solver_from_problem(prob, precision=prec, argmin_screen=prec, nu1=1, nu2=1)
        u = to_dev(prob.g)
        pol = torch.zeros((prob.n - 2) ** 2, dtype=torch.uint8, device="cuda")
        states, pols = [prob.g.copy()], []
        for step in (1, 2):
            s.step(u, step * dt, dt, pol)
            states.append(u.cpu().numpy())
            pols.append(pol.cpu().numpy().astype(np.int64))
        out[prec] = (states, pols)
        s.close()
        del u
        torch.cuda.empty_cache()
    return prob, dt, out


@pytest.mark.parametrize("precision", [1, 0])
def test_full_size_steps_solve_the_discrete_hjb_at_sampled_nodes(runs, precision):
    prob, dt, out = runs
    states, pols = out[precision]
    B = int(np.ceil(max(prob.s1, prob.s2) / np.sqrt(prob.h))) + 1
    for step in (1, 2):
        U_prev, X, pol = states[step - 1], states[step], pols[step - 1]
        i1, i2 = _samples(prob.n, pol, B, seed=step)
        V = lisl.control_values_at(prob, X, step * dt, i1, i2)
        flat = i2 * prob.n + i1
        res = X.ravel()[flat] - U_prev.ravel()[flat] - dt * V.min(axis=0)
        scale = max(1.0, np.abs(X).max())
        assert np.abs(res).max() <= HJB_RES_TOL * scale, (step, np.abs(res).max())
        J = (i2 - 1) * (prob.n - 2) + (i1 - 1)
        ok, nd = policies_agree(pol[J], lisl.improve(V), V)
        assert ok, (step, nd)


def test_full_size_mixed_path_within_1e8_of_fp64(runs):
    _, _, out = runs
    for step in (1, 2):
        assert rel_maxnorm(out[1][0][step], out[0][0][step]) <= 1e-8
