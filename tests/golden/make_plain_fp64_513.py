"""Writes tests/golden/plain_fp64_513.npz: the oracle's march on the 513 x 513 FP64 workload.

Workload: uncertain-correlation HJB on [-2, 2]^2, 513 x 513 nodes, 33 controls rho in
[-0.9, 0.9], s1 = 0.3, s2 = 0.2, T = 1, 64 implicit Euler steps (theta = 1), Howard policy
iteration with a sparse direct solve per iteration (Section 1 and Eq. 2.11 of the paper;
the oracle's readings of the stop rule and tie-breaking).

The file is produced by the CPU oracle alone (this script imports nothing but `oracle` and
`workloads`); the GPU parity test reads it because the direct-solve march takes hours on one
core (about 60 s per sparse LU factorisation at this size).

Stored arrays:
  U_T        (513, 513) float64  U at t = T (boundary = psi = 0)
  policy_T   (511 * 511,) uint8  final policy of the last step
  U_1        (513, 513) float64  U after the first step
  policy_1   (511 * 511,) uint8  final policy of the first step
  pi_iters   (64,) int32         Howard iterations per step
  seconds    ()  float64         wall time of the march

    python tests/golden/make_plain_fp64_513.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import lisl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plain_fp64_513.npz")


def main():
    p = W.plain_fp64()
    dt = p.T / p.n_steps
    U = p.g.copy()
    policy = None
    pis = []
    t0 = time.perf_counter()
    U_1 = pol_1 = None
    for s in range(1, p.n_steps + 1):
        r = lisl.howard_step(p, U, s * dt, dt, policy0=policy)
        if not r.converged:
            raise RuntimeError(f"oracle Howard iteration did not converge at step {s}")
        U, policy = r.X, r.policy
        pis.append(r.pi_iters)
        if s == 1:
            U_1, pol_1 = U.copy(), policy.copy()
        print(f"step {s}: {r.pi_iters} Howard iterations, {time.perf_counter() - t0:.0f} s", flush=True)
    np.savez_compressed(OUT, U_T=U, policy_T=policy.astype(np.uint8), U_1=U_1,
                        policy_1=pol_1.astype(np.uint8), pi_iters=np.asarray(pis, dtype=np.int32),
                        seconds=np.float64(time.perf_counter() - t0))
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
