"""GPU adjoint step (fse_step_adjoint) and the autograd wrapper against the oracle adjoint
and against central finite differences of the GPU forward map."""
import math

import numpy as np
import pytest

import fse_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _state(p, seed):
    X = O.coords(p)
    rng = np.random.default_rng(seed)
    e = sum(-0.5 * (X[j] - rng.uniform(-0.5, 0.5)) ** 2 + 1j * rng.uniform(-0.5, 0.5) * X[j] for j in range(p.dim))
    psi = np.exp(e)
    return psi / math.sqrt(O.mass(psi, p))


CASES = {
    "2d_coulomb": dict(dim=2, n=(32, 48), lo=(-6.0, -7.0), hi=(6.0, 7.0), s=0.6, omega=0.7, beta=60.0, lam=15.0,
                       dt=1e-2, kernel="coulomb", gamma=(1.0, 1.2), prec="f64"),
    "3d_ddi": dict(dim=3, n=(16, 24, 16), lo=(-5.0,) * 3, hi=(5.0,) * 3, s=0.7, omega=0.8, beta=50.0, lam=20.0,
                   dt=5e-3, kernel="ddi3d", dip_n=(0.6, 0.0, 0.8), gamma=(1.0, 1.2, 2.0), prec="f64"),
    "2d_none": dict(dim=2, n=(32, 32), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.9, omega=0.5, beta=30.0, lam=0.0,
                    dt=1e-2, kernel="none", gamma=(1.0, 1.1), prec="f64"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_step_matches_oracle(lib, name):
    d = CASES[name]
    p = O.params(d)
    psi = _state(p, 1)
    g = _state(p, 2) * (1.0 + 0.5j)
    gam = tuple(1.0 + 0.1 * v for v in range(p.dim))
    ref_g, ref_dg = O.adjoint_split_step(psi, g, p, 0.3, gam)
    plan = lib.Plan(d)
    x = plan.to_device(psi)
    gd = plan.to_device(g)
    dg = plan.adjoint(x, gd, 0.3, np.array(gam), want_dgamma=True)
    assert _rel(gd.cpu().numpy(), ref_g) < 1e-12
    assert np.max(np.abs(dg[:p.dim] - ref_dg)) < 1e-11 * max(1.0, np.max(np.abs(ref_dg)))
    assert torch.equal(x, plan.to_device(psi))  # psi_n unchanged


def test_autograd_matches_oracle_gradient(lib):
    from paper_1512_03210_gb300.autograd import evolve, overlap_objective
    d = CASES["2d_coulomb"]
    p = O.params(d)
    psi0 = _state(p, 3)
    tgt = _state(p, 4)
    nst = 12
    rng = np.random.default_rng(5)
    gam = 1.0 + 0.1 * rng.standard_normal((nst, 2))
    ref_g, ref_dg = O.gradient_adjoint(psi0, tgt, p, 0.0, nst, gam)
    plan = lib.Plan(d)
    x0 = plan.to_device(psi0).requires_grad_(True)
    gt = torch.tensor(gam, dtype=torch.float64, requires_grad=True)
    out = evolve(plan, x0, gt, 0.0)
    J = overlap_objective(out, plan.to_device(tgt), float(np.prod(O.mesh_size(p))))
    J.backward()
    assert _rel(x0.grad.cpu().numpy(), ref_g) < 1e-10
    assert _rel(gt.grad.numpy(), ref_dg) < 1e-10


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_workload_against_finite_differences(lib, prec):
    """256^2, 200 steps, per-step trap frequencies, sqrt(T) checkpoints: gradients within
    1e-4 (relative) of central finite differences of the float64 GPU forward map."""
    from paper_1512_03210_gb300.autograd import evolve, overlap_objective
    d = I.workload("adjoint_2d_256")
    nst = d["steps"]
    gam = I.adjoint_gammas(nst)
    p = O.params(d)
    psi0 = I.psi0("adjoint_2d_256")
    tgt = I.adjoint_target(d)
    cell = float(np.prod(O.mesh_size(p)))
    plan = lib.Plan(dict(d, prec=prec))
    x0 = plan.to_device(psi0).requires_grad_(True)
    gt = torch.tensor(gam, dtype=torch.float64, requires_grad=True)
    J = overlap_objective(evolve(plan, x0, gt, 0.0), plan.to_device(tgt), cell)
    J.backward()
    g_psi = x0.grad.to(torch.complex128).cpu().numpy()
    g_gam = gt.grad.numpy()
    ref = lib.Plan(dict(d, prec="f64"))
    tg = ref.to_device(tgt)

    def Jf(psi, gm):
        x = ref.to_device(psi)
        ref.step(x, 0.0, nst, gm)
        c = cell * torch.sum(x * torch.conj(tg))
        return float(abs(complex(c.item())) ** 2)

    rng = np.random.default_rng(11)
    for (n, v) in [(0, 0), (57, 1), (120, 0), (199, 1), (150, 1)]:
        e = np.zeros_like(gam)
        h = 1e-4
        e[n, v] = h
        fd = (Jf(psi0, gam + e) - Jf(psi0, gam - e)) / (2 * h)
        # relative to the component itself, with a floor for components far
        # below the largest one: the float32 adjoint rounds at about 1e-6 of
        # max|dJ/dgamma| (floor 1e-2 * 1e-4 of it), the float64 one at ~1e-14
        # (floor 1e-5 * 1e-4 of it)
        floor = (1e-2 if prec == "f32" else 1e-5) * np.max(np.abs(g_gam))
        print(f"dJ/dgamma[{n},{v}] = {g_gam[n, v]:.6e}, fd {fd:.6e}, |g|/max|g| {abs(g_gam[n, v]) / np.max(np.abs(g_gam)):.2e}")
        assert abs(g_gam[n, v] - fd) <= 1e-4 * max(abs(fd), floor), (n, v, g_gam[n, v], fd)
    for _ in range(2):
        dirn = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
        dirn *= np.exp(-0.05 * (O.coords(p)[0] ** 2 + O.coords(p)[1] ** 2))
        h = 1e-4
        fd = (Jf(psi0 + h * dirn, gam) - Jf(psi0 - h * dirn, gam)) / (2 * h)
        an = float(np.sum((np.conj(g_psi) * dirn).real))
        assert abs(an - fd) <= 1e-4 * abs(fd), (an, fd)
