"""GPU observables (fse_observables) against the FP64 oracle's observables, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(p, seed=0):
    X = O.coords(p)
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.5, 0.5, p.dim)
    k = rng.uniform(-0.8, 0.8, p.dim)
    e = sum(-0.5 * (1.0 + 0.2 * j) * (X[j] - c[j]) ** 2 + 1j * k[j] * X[j] for j in range(p.dim))
    psi = np.exp(e)
    return psi / math.sqrt(O.mass(psi, p))


CASES = {
    "2d_coulomb_f64": dict(dim=2, n=(64, 48), lo=(-7.0, -6.0), hi=(7.0, 6.0), s=0.7, omega=0.6, beta=40.0,
                           lam=8.0, dt=1e-3, kernel="coulomb", gamma=(1.0, 1.4), prec="f64"),
    "3d_ddi_f64": dict(dim=3, n=(32, 24, 16), lo=(-5.0, -5.0, -4.0), hi=(5.0, 5.0, 4.0), s=0.6, omega=0.9,
                       beta=50.0, lam=20.0, dt=1e-3, kernel="ddi3d",
                       dip_n=(1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)), gamma=(1.0, 1.2, 2.0), prec="f64"),
    "3d_coulomb_f32": dict(dim=3, n=(32, 32, 32), lo=(-5.0,) * 3, hi=(5.0,) * 3, s=0.8, omega=0.4,
                           beta=30.0, lam=10.0, dt=1e-3, kernel="coulomb", gamma=(1.0, 1.1, 1.3), prec="f32"),
    "2d_ddi_f64": dict(dim=2, n=(48, 48), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.8, omega=0.7, beta=20.0,
                       lam=15.0, dt=1e-3, kernel="ddi2d", dip_n=(0.48, -0.36, 0.8), gamma=(1.0, 1.3), prec="f64"),
    "2d_lattice_f64": dict(dim=2, n=(64, 64), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.9, omega=0.5, beta=20.0,
                           lam=5.0, dt=1e-3, kernel="coulomb", gamma=(1.0, 1.0), lat_amp=10.0,
                           lat_k=(math.pi, math.pi), prec="f64"),
    "2d_none_f64": dict(dim=2, n=(32, 32), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=1.0, omega=0.3, beta=10.0,
                        lam=0.0, dt=1e-3, kernel="none", gamma=(1.0, 1.0), prec="f64"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_observables_match_oracle(lib, name):
    d = CASES[name]
    p = O.params(d)
    psi = _state(p, seed=len(name))
    t = 0.37
    gam = (1.1, 0.9, 1.3)[: p.dim]
    ref = O.observables(psi, p, t, gam)
    plan = lib.Plan(d)
    x = plan.to_device(psi)
    got = plan.observables(x, t, gam)
    tol = 1e-12 if d["prec"] == "f64" else 2e-6
    scale = max(abs(ref["energy"]), abs(ref["e_kin"]), 1.0)
    for k in ("mass", "e_kin", "e_pot", "e_int", "e_non", "e_rot", "energy", "lz"):
        assert abs(got[k] - ref[k]) <= tol * max(scale, abs(ref[k])), (k, got[k], ref[k])
    assert np.max(np.abs(got["xc"] - ref["xc"])) <= tol * 10
    assert np.max(np.abs(got["width"] - ref["width"])) <= tol * 10 * max(1.0, np.max(ref["width"]))


def test_observables_leave_psi_unchanged(lib):
    d = CASES["3d_ddi_f64"]
    p = O.params(d)
    psi = _state(p)
    plan = lib.Plan(d)
    x = plan.to_device(psi)
    before = x.clone()
    plan.observables(x, 0.0)
    assert torch.equal(before, x)
