"""GPU checks of the batched solve (sl_batch_*): every instance of a batch solved by several
worker threads on their own streams equals, bit for bit, the same instance solved alone on a
new handle; one instance also matches the oracle; a failing instance leaves the others
untouched; a second run repeats the first exactly."""
import numpy as np
import pytest

import workloads as W
from tests._gpu_util import TOL_FP64, rel_maxnorm, to_dev

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _instances():
    return W.batched(n_inst=12, seed=3, sizes=(33, 65, 129), k_range=(5, 33), n_steps=4, T=0.25)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_solves_bit_for_bit(precision):
    import torch
    S = _lib()
    probs = _instances()
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=4, precision=precision, argmin_screen=precision, nu1=1, nu2=1)
    assert sorted(set(b.worker_of(i) for i in range(len(probs)))) == [0, 1, 2, 3]
    b.run()   # first run: every handle captures its CUDA graphs
    for p, u in zip(probs, us):
        u.copy_(to_dev(p.g))
    l0 = S.launch_count()
    st, stats = b.run()
    torch.cuda.synchronize()
    batch_launches = S.launch_count() - l0
    assert st == [0] * len(probs), b.last_error()
    seq_launches = 0
    for p, u, s_ in zip(probs, us, stats):
        sol = S.solver_from_problem(p, precision=precision, argmin_screen=precision, nu1=1, nu2=1)
        v = to_dev(p.g)
        sol.solve(to_dev(p.g), 0.0, p.T, p.n_steps)   # capture the graphs, as the first batch run did
        sol.reset()
        l1 = S.launch_count()
        ref = sol.solve(v, 0.0, p.T, p.n_steps)
        seq_launches += S.launch_count() - l1
        sol.close()
        assert torch.equal(u, v)
        assert s_["steps"] == p.n_steps and s_["krylov_iters"] == ref["krylov_iters"]
    # the launch counter stays exact while several threads launch and capture at once
    assert batch_launches == seq_launches
    b.close()


def test_batch_instance_matches_oracle():
    from oracle import lisl
    S = _lib()
    probs = [p for p in _instances() if p.n == 33][:2]
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=2, precision=0)
    st, _ = b.run()
    assert st == [0, 0]
    for p, u in zip(probs, us):
        assert rel_maxnorm(u.cpu().numpy(), lisl.solve(p).U) <= TOL_FP64
    b.close()


def test_failing_instance_does_not_stop_the_others():
    import torch
    S = _lib()
    probs = _instances()[:5]
    bad = 2
    probs[bad].c = np.full(probs[bad].K, 100.0)   # dt * c = 6.25 > 1: SL_ECFL
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=3, precision=1, argmin_screen=1)
    st, _ = b.run()
    assert st[bad] == S.SL_ECFL and all(s == 0 for i, s in enumerate(st) if i != bad)
    assert "instance 2" in b.last_error()
    for i, (p, u) in enumerate(zip(probs, us)):
        if i == bad:
            continue
        sol = S.solver_from_problem(p, precision=1, argmin_screen=1)
        v = to_dev(p.g)
        sol.solve(v, 0.0, p.T, p.n_steps)
        sol.close()
        assert torch.equal(u, v)
    b.close()


def test_second_run_repeats_the_first():
    import torch
    S = _lib()
    probs = _instances()[:6]
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=3, precision=1, argmin_screen=1)
    b.run()
    first = [u.clone() for u in us]
    for p, u in zip(probs, us):
        u.copy_(to_dev(p.g))
    b.run()
    assert all(torch.equal(a, u) for a, u in zip(first, us))
    b.close()


def test_many_workers_on_uneven_instances_never_fail():
    """Instances whose kernels need different amounts of shared memory, launched from 16
    threads at once, three runs in a row: every run succeeds and repeats the first."""
    import torch
    S = _lib()
    probs = W.batched(n_inst=40, seed=7, sizes=(65, 129, 257), k_range=(17, 65), n_steps=3, T=3 / 32)
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=16, precision=1, argmin_screen=1, nu1=1, nu2=1)
    first = None
    for _ in range(3):
        for p, u in zip(probs, us):
            u.copy_(to_dev(p.g))
        st, _ = b.run()
        torch.cuda.synchronize()
        assert st == [0] * len(probs), b.last_error()
        if first is None:
            first = [u.clone() for u in us]
        else:
            assert all(torch.equal(a, u) for a, u in zip(first, us))
    b.close()


def test_autotuned_batch_equals_single_solves_with_the_chosen_launch():
    """sl_batch_autotune picks a V-cycle tail per grid size from probe runs of the whole batch,
    restores the state vectors, and every instance then equals, bit for bit, a single solve with
    the chosen configuration (and the oracle within the mixed tolerance)."""
    import torch
    from oracle import lisl
    from tests._gpu_util import TOL_MIXED
    S = _lib()
    probs = W.batched(n_inst=10, seed=5, sizes=(65, 129), k_range=(5, 17), n_steps=4, T=0.25)
    us = [to_dev(p.g) for p in probs]
    b = S.Batch(probs, us, workers=4, precision=1, argmin_screen=1, nu1=1, nu2=1, use_graphs=1)
    choices = b.autotune(probe_steps=1, max_tail_rows=4096)
    assert sorted(c["n"] for c in choices) == sorted(set(p.n for p in probs))
    level_rows = {65: {0, 31 * 31, 15 * 15, 7 * 7}, 129: {0, 63 * 63, 31 * 31, 15 * 15, 7 * 7}}
    for c in choices:
        assert c["coarse_tail_rows"] in level_rows[c["n"]], c
        assert c["probe_seconds"] > 0
    for p, u in zip(probs, us):
        assert torch.equal(u, to_dev(p.g))
    st, _ = b.run()
    torch.cuda.synchronize()
    assert st == [0] * len(probs), b.last_error()
    tail = {c["n"]: c["coarse_tail_rows"] for c in choices}
    for p, u in zip(probs, us):
        sol = S.solver_from_problem(p, precision=1, argmin_screen=1, nu1=1, nu2=1, use_graphs=1,
                                    coarse_tail_rows=tail[p.n])
        v = to_dev(p.g)
        sol.solve(v, 0.0, p.T, p.n_steps)
        sol.close()
        assert torch.equal(u, v)
    p, u = probs[0], us[0]
    assert rel_maxnorm(u.cpu().numpy(), lisl.solve(p).U) <= TOL_MIXED
    b.close()
