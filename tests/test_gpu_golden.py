"""The float64 GPU path reproduces the stored oracle observables of the 2D 128^2 workload."""
import json
import os

import numpy as np
import pytest

import fse_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


def test_gpu_observables_match_stored_oracle_values(lib):
    ref = json.load(open(os.path.join(HERE, "golden", "oracle_2d_coulomb_128.json")))
    d = I.workload(ref["workload"])
    plan = lib.Plan(d)
    x = plan.to_device(I.psi0(ref["workload"]))
    done = 0
    for n in (0, 10, 50, 100):
        plan.step(x, done * d["dt"], n - done)
        done = n
        ob = plan.observables(x, n * d["dt"])
        st = ref["steps"][str(n)]
        for k in ("mass", "energy", "e_kin", "e_pot", "e_int", "e_non", "e_rot", "lz"):
            assert abs(ob[k] - st[k]) <= 1e-10 * max(1.0, abs(st[k])), (n, k, ob[k], st[k])
        assert np.allclose(ob["xc"], st["xc"], rtol=0, atol=1e-10)
        assert np.allclose(ob["width"], st["width"], rtol=1e-10, atol=1e-12)
