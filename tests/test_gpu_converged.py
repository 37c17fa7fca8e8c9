"""Converged runs of every storage format against the converged FP64 oracle
(128x128 two-phase media: the benchmark recipe and the same medium with K
widened to log-uniform [1e-6, 1e-2]; oracle values in
tests/golden/converged_128.json, written by make_converged_128.py from
oracle/ alone).

16-bit storage rounds stochastically, so its mean velocity carries a noise
floor that falls as the lattice grows.  The convergence floor of a format is
the smallest tol (relative change of U_x per 1000 steps, on 3 consecutive
checks) at which the solver's own test still fires within 1e6 steps on these
128^2 media: FP32 1e-7, FP16 1e-5, BF16 1e-4 (at 2048^2 BF16 reaches 1e-6).
Each run stops at its floor; the K_app at that stop and the time average of
K_app over the next 100 checks are compared with the oracle.  The average is
the converged permeability of the statistically steady state: within the
spec bounds (1e-4 FP32, 1e-3 16-bit).  A single 16-bit sample at the
stop also carries that state's fluctuation (BF16: about 2.5e-4 rms here).
"""

import json
import os

import numpy as np
import pytest

import media

pytestmark = pytest.mark.gpu

GOLD_PATH = os.path.join(os.path.dirname(__file__), "golden", "converged_128.json")
FLOOR = {"f32": 1e-7, "f16": 1e-5, "bf16": 1e-4}
BOUND_AVG = {"f32": 1e-4, "f16": 1e-3, "bf16": 1e-3}
BOUND_STOP = {"f32": 1e-4, "f16": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module")
def pkg():
    from paper_1601_00704_gb300 import build
    build.build()
    import paper_1601_00704_gb300 as p
    return p


@pytest.fixture(scope="module")
def gold():
    return json.load(open(GOLD_PATH))


@pytest.mark.parametrize("case", ["two_phase", "two_phase_wide_k"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_converged_kapp_matches_converged_oracle(pkg, gold, case, storage):
    import torch
    g = gold[case]
    kw = {k: tuple(v) for k, v in g["kw"].items()}
    eps, K, _ = media.two_phase_medium(128, 128, seed=0, **kw)
    s = pkg.Solver(128, 128, storage=storage, stream=torch.cuda.Stream())
    s.set_medium(eps, K)
    s.set_force(1e-6)
    s.set_convergence(3)
    steps, conv = s.step(1_000_000, tol=FLOOR[storage], check_every=1000)
    assert conv, f"{storage} did not converge at tol {FLOOR[storage]:g}"
    k_stop = s.permeability()
    ks = []
    for _ in range(100):
        s.step(1000)
        ks.append(s.permeability())
    k_avg = float(np.mean(ks))
    k_ref = g["k_app"]
    e_stop, e_avg = k_stop / k_ref - 1, k_avg / k_ref - 1
    print(f"{case} {storage}: stop at {steps} steps, K_app rel {e_stop:+.2e}; "
          f"mean over 1e5 further steps {e_avg:+.2e} (rms {np.std(ks) / k_avg:.1e})")
    assert abs(e_avg) <= BOUND_AVG[storage]
    assert abs(e_stop) <= BOUND_STOP[storage]
