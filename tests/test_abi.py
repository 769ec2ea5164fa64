"""The C-ABI library loads on a machine without a GPU, exports every function
declared in include/fse.h, and validates plan parameters on the host."""
import ctypes as ct
import os

import pytest

import fse_inputs as I
import paper_1512_03210_gb300 as fse


def test_header_declares_the_boundary():
    names = fse.header_functions()
    for required in ("fse_plan_create", "fse_plan_set_workspace", "fse_kernel_precompute", "fse_step",
                     "fse_step_adjoint", "fse_observables", "fse_plan_destroy", "fse_status_string"):
        assert required in names


def test_library_exports_every_header_function():
    lib = fse.load()
    for name in fse.header_functions():
        assert hasattr(lib, name), name


def test_status_strings():
    assert fse.fse_status_string(0) == "ok"
    assert "workspace" in fse.fse_status_string(3)


def _create(p):
    lib = fse.load()
    fp = fse.to_params(p)
    h = ct.c_void_p()
    nb = ct.c_size_t()
    st = lib.fse_plan_create(ct.byref(fp), None, ct.byref(h), ct.byref(nb))
    if h.value:
        lib.fse_plan_destroy(h)
    return st, nb.value


def test_plan_validation_on_host():
    good = I.workload("2d_coulomb_128")
    st, nb = _create(good)
    assert st == 0 and nb > 0
    # workspace grows with the padded spectrum: 3D 256^3 float32 needs S = 256*512*272 c64
    st, nb3 = _create(I.workload("3d_dipolar_256"))
    assert st == 0 and nb3 > 256 * 512 * 272 * 8
    assert _create(dict(good, dim=4))[0] == 1
    assert _create(dict(good, s=0.0))[0] == 1
    assert _create(dict(good, dt=0.0))[0] == 1
    assert _create(dict(good, hi=(-9.0, 8.0)))[0] == 1
    assert _create(dict(good, kernel="ddi3d"))[0] == 1           # the DDI kernel needs dim 3
    assert _create(dict(good, n=(100, 128)))[0] == 2             # 100 is not 2^a or 3*2^a
    assert _create(dict(good, n=(1024, 1024)))[0] == 2           # above the largest size
    # Coulomb-type exponent: 0 < mu <= dim - 1 (Eq. Kernel); the DDI kernel uses mu = 1
    assert _create(dict(good, mu=0.5))[0] == 0
    assert _create(dict(good, mu=0.0))[0] == 1
    assert _create(dict(good, mu=1.5))[0] == 1
    d3 = I.workload("3d_dipolar_128")
    assert _create(dict(d3, kernel="coulomb", mu=2.0))[0] == 0
    assert _create(dict(d3, kernel="coulomb", mu=2.5))[0] == 1
    assert _create(dict(d3, mu=0.5))[0] == 1
    # the 2D DDI kernel needs dim 2 and mu = 1
    assert _create(dict(good, kernel="ddi2d"))[0] == 0
    assert _create(dict(good, kernel="ddi2d", mu=0.5))[0] == 1
    assert _create(dict(d3, kernel="ddi2d"))[0] == 1
    # optical lattice: finite parameters, 0..16 quadrature nodes
    assert _create(dict(good, lat_amp=10.0, lat_k=(3.14, 3.14), quad_nodes=12))[0] == 0
    assert _create(dict(good, lat_amp=10.0, quad_nodes=17))[0] == 1
    assert _create(dict(good, lat_amp=float("nan")))[0] == 1
    # splitting order: 2 (TS2-GauSum) or 4 (triple jump)
    assert _create(dict(good, order=4))[0] == 0
    assert _create(dict(good, order=3))[0] == 1


def test_null_arguments_rejected():
    lib = fse.load()
    assert lib.fse_plan_create(None, None, None, None) == 1
    assert lib.fse_step(None, None, ct.c_double(0.0), 1, None) == 1
    assert lib.fse_kernel_precompute(None) == 1
    assert lib.fse_plan_destroy(None) == 0


def test_set_workspace_checks_size_and_alignment():
    lib = fse.load()
    fp = fse.to_params(I.workload("2d_coulomb_128"))
    h = ct.c_void_p()
    nb = ct.c_size_t()
    assert lib.fse_plan_create(ct.byref(fp), None, ct.byref(h), ct.byref(nb)) == 0
    try:
        # host-side checks only: no device memory is touched
        assert lib.fse_plan_set_workspace(h, ct.c_void_p(4096 * 1024), nb.value - 1) == 3
        assert lib.fse_plan_set_workspace(h, ct.c_void_p(4096 * 1024 + 8), nb.value) == 1
        assert lib.fse_step(h, ct.c_void_p(4096 * 1024), ct.c_double(0.0), 1, None) == 1  # no precompute
        assert "precompute" in fse.fse_plan_error(h)
    finally:
        lib.fse_plan_destroy(h)


def test_plan_rejects_non_finite_scalars():
    good = I.workload("2d_coulomb_128")
    nan = float("nan")
    for key, val in (("beta", nan), ("omega", float("inf")), ("lam", nan), ("gamma", (1.0, nan)),
                     ("s", float("inf")), ("lo", (-8.0, nan))):
        assert _create(dict(good, **{key: val}))[0] == 1, key


def _batch_create(runs):
    lib = fse.load()
    arr = (fse.FseParams * len(runs))(*[fse.to_params(r) for r in runs])
    h = ct.c_void_p()
    nb = ct.c_size_t()
    st = lib.fse_batch_create(arr, len(runs), None, ct.byref(h), ct.byref(nb))
    if h.value:
        lib.fse_batch_destroy(h)
    return st


def test_batch_validates_every_run():
    """Every run of a batch gets fse_plan_create's checks, not only the first of
    each size group, and runs that would need another kernel transform (mu,
    Gaussian-sum fit) than the group's first run are refused."""
    runs = I.batched_runs(6)
    assert _batch_create(runs) == 0
    bad = [dict(r) for r in runs]
    bad[3]["s"] = -0.5
    assert _batch_create(bad) == 1
    bad = [dict(r) for r in runs]
    bad[4]["beta"] = float("nan")
    assert _batch_create(bad) == 1
    bad = [dict(r) for r in runs]
    bad[5]["dt"] = float("inf")
    assert _batch_create(bad) == 1
    mixed = [dict(r) for r in runs]
    mixed[2]["mu"] = 0.5
    assert _batch_create(mixed) == 2
    mixed = [dict(r) for r in runs]
    mixed[1]["gs_h"] = 0.1
    assert _batch_create(mixed) == 2
    # explicit defaults are the same fit as the zero defaults
    same = [dict(r) for r in runs]
    same[1]["gs_h"] = 0.125
    same[2]["gs_delta"] = 1e-3
    assert _batch_create(same) == 0
