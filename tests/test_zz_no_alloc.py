"""sl_hjb_vcycle_noalloc, the V-cycle entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc while they run, for example a host application
whose own pool allocator has reserved the device memory, or a latency-bound loop that cannot
take the device-wide synchronisation of cudaMalloc/cudaFree: its work vectors live in a 2 MiB
static device array of the library.  The checks call it through the C ABI twice in a row and
compare each result with sl_hjb_vcycle on the same input, within the V-cycle parity tolerance
of the other GPU tests.  This file is collected last so that a failure here never hides the
others.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_04821_gb300 as slp
    slp.load()
    return slp


def _solver_with_hierarchy(prob, precision):
    import paper_1605_04821_gb300 as slp
    s = slp.solver_from_problem(prob, precision=precision)
    n = prob.n - 2
    pol = (np.arange(n)[None, :] // 12 + 2 * (np.arange(n)[:, None] // 20)).ravel() % prob.K
    s.set_policy(torch.as_tensor(pol, dtype=torch.uint8, device="cuda"))
    s.build_hierarchy(prob.dt)
    return s


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
@pytest.mark.parametrize("n", [129, 257])
def test_noalloc_vcycle_matches_vcycle_twice(precision, tol, n):
    prob = W.scaled(n, 17, 8, seed=4)
    s = _solver_with_hierarchy(prob, precision)
    dtype = torch.float64 if precision == 0 else torch.float32
    rng = np.random.default_rng(n + precision)
    for call in range(2):
        b = torch.zeros((n, n), dtype=dtype, device="cuda")
        b[1:-1, 1:-1] = torch.as_tensor(rng.standard_normal((n - 2, n - 2)), dtype=dtype, device="cuda")
        ref = torch.zeros_like(b)
        got = torch.zeros_like(b)
        got[1:-1, 1:-1] = float("nan")   # every interior entry must be written; boundary stays 0
        s.vcycle(b, ref)
        s.vcycle_noalloc(b, got)
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err <= tol, (call, err)
        assert torch.all(got[0, :] == 0) and torch.all(got[:, 0] == 0)   # boundary untouched
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import paper_1605_04821_gb300 as slp
    prob = W.scaled(513, 5, 4, seed=1)
    s = _solver_with_hierarchy(prob, 0)
    b = torch.zeros((513, 513), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(slp.SLError) as e:
        s.vcycle_noalloc(b, x)
    assert e.value.status == slp.SL_EINVAL and "bytes" in str(e.value)
    s.close()
