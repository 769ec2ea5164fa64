"""Writes the stored oracle values in this folder. Calls only the oracle.

Usage: python tests/golden/make_golden.py
Output: oracle_2d_coulomb_128.json -- observables of the FP64 oracle on the
2D 128^2 Coulomb workload (s=0.8, Omega=0.6, beta=100, lambda=10, dt=1e-3)
at steps 0, 10, 50 and 100.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fse_inputs as I  # noqa: E402
import oracle as O  # noqa: E402


def main():
    name = "2d_coulomb_128"
    d = I.workload(name)
    p = O.params(d)
    psi = I.psi0(name)
    C = O.gausum_multiplier(p)
    out = {"workload": name, "steps": {}}
    done = 0
    for n in (0, 10, 50, 100):
        psi = O.evolve(psi, p, done * p.dt, n - done, None, C)
        done = n
        ob = O.observables(psi, p, n * p.dt, None, C)
        out["steps"][str(n)] = {k: (list(map(float, v)) if hasattr(v, "__len__") else float(v)) for k, v in ob.items()}
    with open(os.path.join(HERE, "oracle_2d_coulomb_128.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
