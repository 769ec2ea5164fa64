"""Parity bounds shared by the GPU tests, and the check that applies them.

A float32 split step rounds about 6e-8 per FFT pass and per pointwise
operation, 20-30 such operations per element and step; summed in quadrature
along the chain that is a few 1e-7, and <= 2e-6 relative L2 per step even if
they add up coherently: F32_STEP_REL per step (measured on GB300: 3e-7 to
4e-7 per step at every tested size, up to 256^3). The same rounding bounds
every element: an element's error is a few times the RMS error of the field,
so the largest one stays within F32_STEP_ELEM * max|ref| per step (measured:
2e-7 to 5e-7 per step), and a single element wrong by 1e-5 of the field's
scale fails that bound even where it moves the relative L2 by much less. The float64 path differs from the oracle only in
rounding order (radix-8 Stockham passes against numpy's FFT, closed-form
against quadrature step integrals, merged kinetic half steps): F64_STEP_REL
per step, and F64_STEP_ELEM per step for single elements.
"""
import numpy as np

F32_STEP_REL = 2e-6
F32_STEP_ELEM = 3e-6
F64_STEP_REL = 1e-12
F64_STEP_ELEM = 2e-12


def errors(got, ref):
    """(relative L2 error, largest element error relative to max|ref|)."""
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    d = np.abs(got - ref)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max())


def assert_parity(got, ref, rel, elem, what=""):
    """rel L2 <= rel and max|got - ref| <= elem * max|ref|."""
    r, e = errors(got, ref)
    print(f"{what}: rel L2 {r:.3e} (bound {rel:.1e}), max element {e:.3e} (bound {elem:.1e})")
    assert r <= rel, (what, "relative L2", r, rel)
    assert e <= elem, (what, "max element", e, elem)


def bounds(prec, nsteps, factor=1.0):
    """(rel, elem) bounds of an nsteps run in precision prec."""
    if prec == "f32":
        return factor * F32_STEP_REL * nsteps, factor * F32_STEP_ELEM * nsteps
    return factor * F64_STEP_REL * nsteps, factor * F64_STEP_ELEM * nsteps
