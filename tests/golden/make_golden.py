"""Writes the stored oracle fits used by the parity tests.

Calls only the FP64 CPU oracle (``oracle/``) and the seeded input generator.
Each output file holds a fingerprint of the generated inputs (so a test can
check that it regenerated the same data), the oracle's converged
coefficients and its fit statistics.

    python tests/golden/make_golden.py c1 c2
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1404_3177_gb300 import datagen  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def fingerprint(prob) -> str:
    h = hashlib.sha256()
    for a in (prob.X, prob.Y, prob.Z, prob.choice):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def write(name, prob, theta, stats, seconds):
    path = os.path.join(HERE, f"oracle_fit_{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# Oracle Newton-Raphson fit of workload {prob.name} from theta = 0\n")
        fh.write("# written by tests/golden/make_golden.py (FP64 CPU oracle only)\n")
        fh.write(f"name {prob.name}\nN {prob.N}\nK {prob.K}\np {prob.p}\nd {prob.d}\nf {prob.f}\n")
        fh.write(f"gamma_base {prob.gamma_base}\nfingerprint {fingerprint(prob)}\n")
        for k in ("iters", "ls_evals", "stop", "loglik", "grad_inf"):
            v = stats[k]
            fh.write(f"{k} {v!r}\n" if isinstance(v, float) else f"{k} {v}\n")
        fh.write(f"oracle_seconds {seconds:.1f}\n")
        fh.write(f"n_theta {theta.size}\ntheta\n")
        for v in theta:
            fh.write(f"{float(v)!r}\n")
    print("wrote", path, stats, f"{seconds:.1f}s", flush=True)


def main(names):
    makers = {"c1": datagen.config1, "c2": datagen.config2}
    for name in names:
        prob = makers[name]()
        t0 = time.time()
        theta, stats = oracle.fit(prob, gtol=1e-8, steptol=1e-12, maxiter=100)
        write(name, prob, theta, stats, time.time() - t0)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1"])
