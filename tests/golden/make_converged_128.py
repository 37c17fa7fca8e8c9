"""Write converged_128.json: the FP64 oracle's converged Darcy permeability
of the two 128x128 parity media (the two-phase medium of the benchmark
recipe, and the same medium with K widened to log-uniform [1e-6, 1e-2]),
used by the reduced-precision convergence tests.  Calls only oracle/ (and
the seeded input generator):

    python tests/golden/make_converged_128.py

The oracle runs until the mean velocity changes by at most 1e-12 relative
per 1000 steps, or 1.5e6 steps."""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import media  # noqa: E402
import oracle  # noqa: E402

CASES = {
    "two_phase": {},
    "two_phase_wide_k": {"k_iom": (1e-6, 1e-2), "k_om": (1e-6, 1e-2)},
}


def main():
    oracle.build()
    out = {"recipe": "media.two_phase_medium(128, 128, seed=0, **kw), G = (1e-6, 0), tau = 1, walls in y",
           "stop": "relative change of U_x <= 1e-12 per 1000 steps, or 1.5e6 steps"}
    for name, kw in CASES.items():
        eps, K, _ = media.two_phase_medium(128, 128, seed=0, **kw)
        o = oracle.Oracle(128, 128, tau=1.0, threads=os.cpu_count())
        o.set_medium(eps, K)
        o.set_force(1e-6)
        t0 = time.time()
        steps, conv = o.step(1_500_000, tol=1e-12, check_every=1000)
        out[name] = {"kw": {k: list(v) for k, v in kw.items()}, "k_app": o.permeability(),
                     "mean_u": list(o.mean_u), "steps": steps, "converged": conv}
        print(name, out[name], f"{time.time() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, "converged_128.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
