"""Python binding of the GB300 TS2-GauSum split-step library (include/fse.h).

Argument marshalling only: every grid operation runs in the CUDA library
``_build/libfse.so`` (built in-tree for sm_103a by ``build.py``). PyTorch
provides device memory (the wave function and the caller-owned workspace)
and streams. If the library is missing and cannot be built, ``load()``
raises: there is no CPU fallback.

The functions ``fse_plan_create`` ... ``fse_plan_destroy`` carry the names of
the C entry points; ``Plan`` bundles a plan with its workspace.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

import numpy as np

__all__ = [
    "load", "lib_path", "Plan", "FseParams", "FseObs", "FSE_OK", "FseError",
    "fse_plan_create", "fse_plan_set_workspace", "fse_kernel_precompute", "fse_step",
    "fse_step_host", "fse_step_adjoint", "fse_observables", "fse_plan_set_stream",
    "fse_plan_destroy", "fse_status_string", "fse_plan_error", "fse_plan_launch_count",
    "header_functions", "to_params", "fse_plan_profile", "fse_plan_profile_read", "PASS_KINDS",
    "fse_mass_noalloc", "Batch", "fse_batch_create", "fse_batch_set_workspace", "fse_batch_precompute",
    "fse_batch_step", "fse_batch_destroy", "fse_batch_error", "fse_batch_launch_count",
    "FseGsOpts", "FseGsInfo", "fse_ground_state_workspace", "fse_ground_state", "fse_shift_kick",
]

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "fse.h")

FSE_OK = 0
KERNELS = {"none": 0, "coulomb": 1, "ddi3d": 2, "ddi2d": 3}
PRECS = {"f32": 0, "f64": 1}
PASS_KINDS = ["xfwd", "xinv", "E", "A", "col", "kin", "pad", "khat", "pre", "other"]


class FseParams(ct.Structure):
    _fields_ = [
        ("dim", ct.c_int), ("n", ct.c_int * 3), ("lo", ct.c_double * 3), ("hi", ct.c_double * 3),
        ("s", ct.c_double), ("m", ct.c_double), ("omega", ct.c_double), ("beta", ct.c_double),
        ("lambda_", ct.c_double), ("dt", ct.c_double), ("kernel", ct.c_int), ("mu", ct.c_double),
        ("dip_n", ct.c_double * 3), ("gamma", ct.c_double * 3), ("gs_delta", ct.c_double),
        ("gs_h", ct.c_double), ("gs_tmin", ct.c_double), ("prec", ct.c_int), ("renormalize", ct.c_int),
        ("order", ct.c_int), ("lat_amp", ct.c_double), ("lat_k", ct.c_double * 3), ("quad_nodes", ct.c_int),
    ]


class FseGsOpts(ct.Structure):
    _fields_ = [("dt", ct.c_double), ("max_outer", ct.c_int), ("tol", ct.c_double), ("max_inner", ct.c_int),
                ("inner_tol", ct.c_double)]


class FseGsInfo(ct.Structure):
    _fields_ = [("outer", ct.c_int), ("inner", ct.c_int), ("change", ct.c_double), ("residual", ct.c_double)]


class FseObs(ct.Structure):
    _fields_ = [
        ("mass", ct.c_double), ("e_kin", ct.c_double), ("e_pot", ct.c_double), ("e_int", ct.c_double),
        ("e_non", ct.c_double), ("e_rot", ct.c_double), ("energy", ct.c_double), ("lz", ct.c_double),
        ("xc", ct.c_double * 3), ("width", ct.c_double * 3),
    ]

    def as_dict(self, dim: int) -> dict:
        d = {k: getattr(self, k) for k in ("mass", "e_kin", "e_pot", "e_int", "e_non", "e_rot", "energy", "lz")}
        d["xc"] = np.array(self.xc[:dim])
        d["width"] = np.array(self.width[:dim])
        return d


class FseError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_status_name(status)}" + (f" ({detail})" if detail else ""))


_lib = None


def lib_path() -> str:
    return os.path.join(HERE, "_build", "libfse.so")


def header_functions() -> list:
    """Names of the functions declared in include/fse.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(fse_[a-z_]+)\s*\(", txt)))


def load(build_if_missing: bool = True):
    """Load libfse.so (building it with nvcc if absent); raises if neither works."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        from . import build as _b
        _b.build()
    lib = ct.CDLL(path)
    P = ct.c_void_p
    sig = {
        "fse_plan_create": (ct.c_int, [ct.POINTER(FseParams), P, ct.POINTER(P), ct.POINTER(ct.c_size_t)]),
        "fse_plan_set_workspace": (ct.c_int, [P, P, ct.c_size_t]),
        "fse_kernel_precompute": (ct.c_int, [P]),
        "fse_step": (ct.c_int, [P, P, ct.c_double, ct.c_int, P]),
        "fse_step_host": (ct.c_int, [P, P, ct.c_double, ct.c_int, P]),
        "fse_step_adjoint": (ct.c_int, [P, P, P, ct.c_double, P, P]),
        "fse_observables": (ct.c_int, [P, P, ct.c_double, P, ct.POINTER(FseObs)]),
        "fse_plan_set_stream": (ct.c_int, [P, P]),
        "fse_plan_destroy": (ct.c_int, [P]),
        "fse_status_string": (ct.c_char_p, [ct.c_int]),
        "fse_plan_error": (ct.c_char_p, [P]),
        "fse_plan_launch_count": (ct.c_longlong, [P]),
        "fse_plan_profile": (ct.c_int, [P, ct.c_int]),
        "fse_plan_profile_read": (ct.c_int, [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong)]),
        "fse_mass_noalloc": (ct.c_int, [P, ct.c_int, ct.c_longlong, ct.c_double, P, P]),
        "fse_batch_create": (ct.c_int, [ct.POINTER(FseParams), ct.c_int, P, ct.POINTER(P), ct.POINTER(ct.c_size_t)]),
        "fse_batch_set_workspace": (ct.c_int, [P, P, ct.c_size_t]),
        "fse_batch_precompute": (ct.c_int, [P]),
        "fse_batch_step": (ct.c_int, [P, ct.POINTER(P), ct.c_double, ct.c_int]),
        "fse_batch_destroy": (ct.c_int, [P]),
        "fse_batch_error": (ct.c_char_p, [P]),
        "fse_batch_launch_count": (ct.c_longlong, [P]),
        "fse_ground_state_workspace": (ct.c_int, [P, ct.POINTER(ct.c_size_t)]),
        "fse_ground_state": (ct.c_int, [P, P, P, ct.c_size_t, ct.POINTER(FseGsOpts), ct.POINTER(FseGsInfo)]),
        "fse_shift_kick": (ct.c_int, [P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_name(st: int) -> str:
    try:
        return load().fse_status_string(st).decode()
    except Exception:  # noqa: BLE001 - used while formatting an error
        return f"status {st}"


def _check(st: int, where: str, plan=None):
    if st != FSE_OK:
        detail = load().fse_plan_error(plan).decode() if plan else ""
        raise FseError(st, where, detail)


def to_params(p: dict) -> FseParams:
    """fse_params from a parameter dict (keys of fse_inputs workloads)."""
    fp = FseParams()
    fp.dim = int(p["dim"])
    for j in range(3):
        have = j < min(fp.dim, len(p["n"]))
        fp.n[j] = int(p["n"][j]) if have else 1
        fp.lo[j] = float(p["lo"][j]) if have else 0.0
        fp.hi[j] = float(p["hi"][j]) if have else 1.0
    fp.s = float(p.get("s", 1.0))
    fp.m = float(p.get("m", 0.0))
    fp.omega = float(p.get("omega", 0.0))
    fp.beta = float(p.get("beta", 0.0))
    fp.lambda_ = float(p.get("lam", 0.0))
    fp.dt = float(p.get("dt", 1e-3))
    fp.kernel = KERNELS[p.get("kernel", "coulomb")]
    fp.mu = float(p.get("mu", 1.0))
    dn = tuple(p.get("dip_n", (0.0, 0.0, 1.0)))
    g = tuple(p.get("gamma", (1.0, 1.0, 1.0)))
    for j in range(3):
        fp.dip_n[j] = float(dn[j])
        fp.gamma[j] = float(g[j]) if j < len(g) else 1.0
    fp.gs_delta = float(p.get("gs_delta", 0.0))
    fp.gs_h = float(p.get("gs_h", 0.0))
    fp.gs_tmin = float(p.get("gs_tmin", 0.0))
    fp.prec = PRECS[p.get("prec", "f32")]
    fp.renormalize = int(p.get("renormalize", 0))
    fp.order = int(p.get("order", 2))
    fp.lat_amp = float(p.get("lat_amp", 0.0))
    lk = tuple(p.get("lat_k", (0.0, 0.0, 0.0)))
    for j in range(3):
        fp.lat_k[j] = float(lk[j]) if j < len(lk) else 0.0
    fp.quad_nodes = int(p.get("quad_nodes", 0))
    return fp


def _ptr(x) -> int:
    return ct.c_void_p(x.data_ptr()) if x is not None else None


# ----- functions named after the C entry points (marshalling only) -----

def fse_plan_create(params: dict, stream=None):
    """Returns (plan handle, workspace bytes)."""
    lib = load()
    fp = to_params(params)
    h = ct.c_void_p()
    nb = ct.c_size_t()
    st = lib.fse_plan_create(ct.byref(fp), ct.c_void_p(stream or 0), ct.byref(h), ct.byref(nb))
    _check(st, "fse_plan_create")
    return h, nb.value


def fse_plan_set_workspace(plan, ws, nbytes: int):
    _check(load().fse_plan_set_workspace(plan, _ptr(ws), nbytes), "fse_plan_set_workspace", plan)


def fse_kernel_precompute(plan):
    _check(load().fse_kernel_precompute(plan), "fse_kernel_precompute", plan)


def _gammas(g):
    if g is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
    return a, a.ctypes.data_as(ct.c_void_p)


def fse_step(plan, psi, t0: float, nsteps: int, gammas=None):
    keep, gp = _gammas(gammas)
    _check(load().fse_step(plan, _ptr(psi), float(t0), int(nsteps), gp), "fse_step", plan)
    del keep


def fse_step_host(plan, psi_host: np.ndarray, t0: float, nsteps: int, gammas=None):
    keep, gp = _gammas(gammas)
    buf = psi_host if isinstance(psi_host, np.ndarray) else psi_host.numpy()
    assert buf.flags.c_contiguous
    _check(load().fse_step_host(plan, buf.ctypes.data_as(ct.c_void_p), float(t0), int(nsteps), gp),
           "fse_step_host", plan)
    del keep


def fse_step_adjoint(plan, psi_n, g, t_n: float, gamma_n=None, want_dgamma: bool = False, dim: int = 3):
    keep, gp = _gammas(gamma_n)
    dg = np.zeros(dim, dtype=np.float64)
    dgp = dg.ctypes.data_as(ct.c_void_p) if want_dgamma else None
    _check(load().fse_step_adjoint(plan, _ptr(psi_n), _ptr(g), float(t_n), gp, dgp), "fse_step_adjoint", plan)
    del keep
    return dg if want_dgamma else None


def fse_observables(plan, psi, t: float, gamma=None) -> FseObs:
    keep, gp = _gammas(gamma)
    o = FseObs()
    _check(load().fse_observables(plan, _ptr(psi), float(t), gp, ct.byref(o)), "fse_observables", plan)
    del keep
    return o


def fse_ground_state_workspace(plan) -> int:
    n = ct.c_size_t(0)
    _check(load().fse_ground_state_workspace(plan, ct.byref(n)), "fse_ground_state_workspace", plan)
    return n.value


def fse_ground_state(plan, psi, workspace, nbytes: int, dt: float, max_outer: int, tol: float,
                     max_inner: int, inner_tol: float) -> dict:
    o = FseGsOpts(float(dt), int(max_outer), float(tol), int(max_inner), float(inner_tol))
    info = FseGsInfo()
    _check(load().fse_ground_state(plan, _ptr(psi), _ptr(workspace), int(nbytes), ct.byref(o), ct.byref(info)),
           "fse_ground_state", plan)
    return {"outer": info.outer, "inner": info.inner, "change": info.change, "residual": info.residual}


def fse_shift_kick(plan, psi, x0=None, k=None):
    a = (ct.c_double * 3)(*((tuple(x0) + (0.0,) * 3)[:3])) if x0 is not None else None
    b = (ct.c_double * 3)(*((tuple(k) + (0.0,) * 3)[:3])) if k is not None else None
    _check(load().fse_shift_kick(plan, _ptr(psi), a, b), "fse_shift_kick", plan)


def fse_plan_set_stream(plan, stream):
    _check(load().fse_plan_set_stream(plan, ct.c_void_p(stream or 0)), "fse_plan_set_stream", plan)


def fse_plan_profile(plan, enable: bool):
    _check(load().fse_plan_profile(plan, 1 if enable else 0), "fse_plan_profile", plan)


def fse_plan_profile_read(plan) -> dict:
    """{pass kind: (total ms, launches)} since the last read."""
    ms = (ct.c_double * len(PASS_KINDS))()
    cnt = (ct.c_longlong * len(PASS_KINDS))()
    _check(load().fse_plan_profile_read(plan, ms, cnt), "fse_plan_profile_read", plan)
    return {k: (ms[i], int(cnt[i])) for i, k in enumerate(PASS_KINDS)}


def fse_mass_noalloc(psi, prec: str, npoints: int, cell_volume: float, mass_out, stream=None):
    """Mass of psi into mass_out (a one-element float64 device tensor) with no device
    allocation; for callers that cannot allocate (see include/fse.h).

    The C entry point sees only a pointer and a count, so the tensors are
    checked here: psi a contiguous CUDA tensor of the dtype that prec names
    (complex64 for "f32", complex128 for "f64") holding at least npoints
    values, mass_out a CUDA float64 tensor on the same device."""
    import torch
    want = {"f32": torch.complex64, "f64": torch.complex128}
    if prec not in want:
        raise ValueError(f"fse_mass_noalloc: prec must be 'f32' or 'f64', not {prec!r}")
    if not (isinstance(psi, torch.Tensor) and psi.is_cuda and psi.is_contiguous() and psi.dtype == want[prec]):
        raise ValueError(f"fse_mass_noalloc: psi must be a contiguous CUDA {want[prec]} tensor")
    if not (isinstance(mass_out, torch.Tensor) and mass_out.is_cuda and mass_out.dtype == torch.float64
            and mass_out.numel() >= 1 and mass_out.device == psi.device):
        raise ValueError("fse_mass_noalloc: mass_out must be a float64 CUDA tensor on psi's device")
    npoints = int(npoints)
    if not 0 <= npoints <= psi.numel():
        raise ValueError(f"fse_mass_noalloc: npoints {npoints} outside [0, {psi.numel()}]")
    st = load().fse_mass_noalloc(_ptr(psi), PRECS[prec], npoints, float(cell_volume), _ptr(mass_out),
                                 ct.c_void_p(stream or 0))
    _check(st, "fse_mass_noalloc")


def fse_plan_destroy(plan):
    load().fse_plan_destroy(plan)


def fse_status_string(st: int) -> str:
    return load().fse_status_string(st).decode()


def fse_plan_error(plan) -> str:
    return load().fse_plan_error(plan).decode()


def fse_plan_launch_count(plan) -> int:
    return int(load().fse_plan_launch_count(plan))


def _bcheck(st: int, where: str, batch=None):
    if st != FSE_OK:
        detail = load().fse_batch_error(batch).decode() if batch else ""
        raise FseError(st, where, detail)


def fse_batch_create(runs: list, stream=None):
    """Returns (batch handle, workspace bytes) for a list of 2D parameter dicts."""
    arr = (FseParams * len(runs))(*[to_params(r) for r in runs])
    h = ct.c_void_p()
    nb = ct.c_size_t()
    _bcheck(load().fse_batch_create(arr, len(runs), ct.c_void_p(stream or 0), ct.byref(h), ct.byref(nb)),
            "fse_batch_create")
    return h, nb.value


def fse_batch_set_workspace(batch, ws, nbytes: int):
    _bcheck(load().fse_batch_set_workspace(batch, _ptr(ws), nbytes), "fse_batch_set_workspace", batch)


def fse_batch_precompute(batch):
    _bcheck(load().fse_batch_precompute(batch), "fse_batch_precompute", batch)


def fse_batch_step(batch, psis: list, t0: float, nsteps: int):
    arr = (ct.c_void_p * len(psis))(*[x.data_ptr() for x in psis])
    _bcheck(load().fse_batch_step(batch, arr, float(t0), int(nsteps)), "fse_batch_step", batch)


def fse_batch_destroy(batch):
    load().fse_batch_destroy(batch)


def fse_batch_error(batch) -> str:
    return load().fse_batch_error(batch).decode()


def fse_batch_launch_count(batch) -> int:
    return int(load().fse_batch_launch_count(batch))


class Batch:
    """Independent 2D runs advanced together, with a torch-allocated workspace."""

    def __init__(self, runs: list, stream=None, device=None):
        import torch
        self.runs = [dict(r) for r in runs]
        self.device = torch.device(device or "cuda")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        with torch.cuda.device(self.device):
            self.handle, self.ws_bytes = fse_batch_create(self.runs, stream.cuda_stream)
            self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)
            fse_batch_set_workspace(self.handle, self.ws, self.ws_bytes)
            fse_batch_precompute(self.handle)

    def to_device(self, psis: list) -> list:
        import torch
        return [torch.as_tensor(np.ascontiguousarray(p)).to(self.device, torch.complex64).contiguous() for p in psis]

    def step(self, psis: list, t0: float, nsteps: int):
        fse_batch_step(self.handle, psis, t0, nsteps)
        return psis

    @property
    def launches(self) -> int:
        return fse_batch_launch_count(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fse_batch_destroy(h)
            self.handle = None


class Plan:
    """A plan with its torch-allocated workspace on the current CUDA device."""

    def __init__(self, params: dict, stream=None, device=None):
        import torch
        self.params = dict(params)
        self.dim = int(params["dim"])
        self.device = torch.device(device or "cuda")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        with torch.cuda.device(self.device):
            self.handle, self.ws_bytes = fse_plan_create(params, stream.cuda_stream)
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            fse_plan_set_workspace(self.handle, self.ws, self.ws_bytes)
            fse_kernel_precompute(self.handle)
        self.cdtype = torch.complex64 if params.get("prec", "f32") == "f32" else torch.complex128

    @property
    def shape(self):
        return tuple(reversed(tuple(self.params["n"][: self.dim])))

    def to_device(self, psi):
        import torch
        return torch.as_tensor(np.ascontiguousarray(psi)).to(self.device, self.cdtype).contiguous()

    def step(self, psi, t0: float, nsteps: int, gammas=None):
        assert psi.dtype == self.cdtype and psi.is_contiguous() and tuple(psi.shape) == self.shape
        fse_step(self.handle, psi, t0, nsteps, gammas)
        return psi

    def step_host(self, psi_host: np.ndarray, t0: float, nsteps: int, gammas=None):
        fse_step_host(self.handle, psi_host, t0, nsteps, gammas)
        return psi_host

    def adjoint(self, psi_n, g, t_n: float, gamma_n=None, want_dgamma=False):
        return fse_step_adjoint(self.handle, psi_n, g, t_n, gamma_n, want_dgamma, self.dim)

    def observables(self, psi, t: float, gamma=None) -> dict:
        return fse_observables(self.handle, psi, t, gamma).as_dict(self.dim)

    def ground_state(self, psi, dt: float, max_outer: int, tol: float = 0.0, max_inner: int = 500,
                     inner_tol: float = 1e-12) -> dict:
        """GF-GauSum ground state (Section 3.2) from the initial guess psi, in place."""
        import torch
        assert psi.dtype == self.cdtype and psi.is_contiguous() and tuple(psi.shape) == self.shape
        nb = fse_ground_state_workspace(self.handle)
        ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        return fse_ground_state(self.handle, psi, ws, nb, dt, max_outer, tol, max_inner, inner_tol)

    def shift_kick(self, psi, x0=None, k=None):
        """psi <- psi(x - x0) exp(i k.x) in place (Eq. ini_dyn)."""
        fse_shift_kick(self.handle, psi, x0, k)
        return psi

    @property
    def launches(self) -> int:
        return fse_plan_launch_count(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.fse_plan_destroy(h)
            self.handle = None
