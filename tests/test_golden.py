"""The oracle still reproduces its stored observables (regression pin of the stored file)."""
import json
import os

import numpy as np

import fse_inputs as I
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_stored_observables():
    ref = json.load(open(os.path.join(HERE, "golden", "oracle_2d_coulomb_128.json")))
    d = I.workload(ref["workload"])
    p = O.params(d)
    psi = I.psi0(ref["workload"])
    C = O.gausum_multiplier(p)
    psi = O.evolve(psi, p, 0.0, 10, None, C)
    ob = O.observables(psi, p, 10 * p.dt, None, C)
    st = ref["steps"]["10"]
    for k in ("mass", "energy", "e_kin", "e_pot", "e_int", "e_non", "lz"):
        assert abs(ob[k] - st[k]) <= 1e-12 * max(1.0, abs(st[k])), k
    assert np.allclose(ob["xc"], st["xc"], rtol=0, atol=1e-12)
    # the stored run conserves mass and keeps the energy within its O(dt^2) splitting error
    e0 = ref["steps"]["0"]["energy"]
    assert abs(ref["steps"]["100"]["mass"] - ref["steps"]["0"]["mass"]) < 1e-12
    assert abs(ref["steps"]["100"]["energy"] - e0) < 1e-4 * abs(e0)
