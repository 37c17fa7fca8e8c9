"""What the trained surrogate gains over the plain GLBM: on unseen media of
its training recipe (256^2, new seeds), starting from f_eq(rho_pred, u_pred)
reaches |K_app/K_ref - 1| <= 1e-3 in fewer steps than starting from rest,
and both runs converge to the same K_app (the solver, not the network,
decides the answer)."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1601_00704_gb300 import build
    build.build()
    import json

    import paper_1601_00704_gb300 as pkg
    from paper_1601_00704_gb300 import surrogate
    from paper_1601_00704_gb300 import train_surrogate as T
    if not os.path.exists(T.DEFAULT_WEIGHTS):
        pytest.fail(f"trained weights missing: {T.DEFAULT_WEIGHTS}")
    meta = json.load(open(os.path.splitext(T.DEFAULT_WEIGHTS)[0] + ".json"))
    net = surrogate.UNet(base=meta["base"], levels=meta["levels"], max_ch=meta.get("max_ch"))
    net.load(T.DEFAULT_WEIGHTS)
    return pkg, T, net


def test_warm_start_saves_steps(setup):
    import media
    pkg, T, net = setup
    cold_total = warm_total = 0
    for seed in (9001, 9002, 9003, 9004):
        m = media.shale_batch(1, seed=seed, sides=(256,))[0]
        K = T.medium_k(pkg, m)
        ref = pkg.Solver(256, 256)
        ref.set_medium(m["eps"], K)
        ref.set_force(T.G)
        ref.step(2_000_000, tol=1e-7, check_every=10000)
        k_ref = ref.permeability()
        pred = T.predict(net, m["eps"], K)
        cold = T.time_to_k(pkg, m["eps"], K, k_ref)
        warm = T.time_to_k(pkg, m["eps"], K, k_ref, init=pred)
        assert cold["met"] and warm["met"]
        cold_total += cold["steps"]
        warm_total += warm["steps"]
        print(f"seed {seed}: cold {cold['steps']} steps, warm {warm['steps']} steps")
        # converged answers agree: the warm run continued to the same limit
        a = pkg.Solver(256, 256)
        a.set_medium(m["eps"], K)
        a.set_force(T.G)
        a.init_equilibrium(*pred)
        a.step(2_000_000, tol=1e-7, check_every=10000)
        assert a.permeability() == pytest.approx(k_ref, rel=2e-4)
    print(f"total: cold {cold_total}, warm {warm_total}")
    assert warm_total <= 0.5 * cold_total
