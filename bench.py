#!/usr/bin/env python
"""Throughput of the TS2-GauSum split step on GB300 (one JSON line on rank 0).

A bench "step" is one TS2-GauSum split step (Section 4.2, Eqs. tssp1-tssp3)
of the 3D dipolar workload: 256^3 grid on [-12,12]^3 (512^3 padded density
spectrum), s=0.6, Omega=0.9, beta=500, lambda=100, tilted dipole axis,
dt=2.5e-4, synthetic 16-vortex Thomas-Fermi-like initial state. The timed
region is one fse_step call advancing K steps (kinetic half steps of
consecutive steps merged, as a user's long run does); psi (134 MB) and the
padded spectrum (279 MB) exceed the 129 MB L2, so no flush is needed.

Also reported: the float64 GPU path on the same workload, per-kernel event
timing of the dominant kernel against the measured HBM copy bandwidth, an
end-to-end figure through fse_step_host (host buffers, copies inside the
timed region), and the FP64 oracle timed on a bounded sample on host cores.

--impl reference times that oracle alone (rank 0) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "split steps/s, 256³ dipolar FSE: FP32 vs FP64 path, same accuracy; % HBM roofline"
UNIT = "split steps/s"
WORKLOAD = "3d_dipolar_256"
GS_WORKLOAD = "gs_2d_512"   # GF-GauSum ground state, 512^2 on [-32,32]^2, dt = 1e-3
GS_INNER_TOL = 1e-12
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle on a bounded sample (a spawned process, after the GPU legs)
# ---------------------------------------------------------------------------

def _oracle_sample(nsteps: int, gs_steps: int, q) -> None:
    try:
        import numpy as np  # noqa: F401
        import fse_inputs as I
        import oracle as O
        d = I.workload(WORKLOAD)
        p = O.params(d)
        psi = I.psi0(WORKLOAD)
        t0 = time.perf_counter()
        C = O.gausum_multiplier(p)
        t_pre = time.perf_counter() - t0
        t0 = time.perf_counter()
        for n in range(nsteps):
            psi = O.split_step(psi, p, n * p.dt, None, C)
        dt = time.perf_counter() - t0
        r = {"ok": True, "seconds": dt, "steps": nsteps, "precompute_s": t_pre}
        if gs_steps > 0:
            # the ground-state workload: GF-GauSum steps of the oracle
            pg = O.params(I.workload(GS_WORKLOAD))
            phi = I.psi0(GS_WORKLOAD)
            Cg = O.gausum_multiplier(pg)
            t0 = time.perf_counter()
            inner = 0
            for _ in range(gs_steps):
                phi, it = O.gf_step(phi, pg, pg.dt, Cg, GS_INNER_TOL, 500)
                inner += it
            r["gs"] = {"seconds": time.perf_counter() - t0, "steps": gs_steps, "inner": inner}
        q.put(r)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        q.put({"ok": False, "error": repr(e)})


def start_oracle(nsteps: int, gs_steps: int = 0):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_oracle_sample, args=(nsteps, gs_steps, q), daemon=True)
    proc.start()
    return proc, q


def finish_oracle(proc, q, timeout=900.0):
    try:
        r = q.get(timeout=timeout)
    except Exception as e:  # noqa: BLE001
        r = {"ok": False, "error": f"oracle sample did not finish: {e!r}"}
    proc.join(timeout=5)
    return r


def oracle_baseline_dict(r: dict) -> dict:
    if not r.get("ok"):
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r.get("error")}
    return {"value": r["steps"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{r['steps']} split step(s) of the {WORKLOAD} workload in the FP64 numpy oracle "
                      f"(single-threaded numpy FFT; kernel transform precomputed outside the timed "
                      f"region in {r['precompute_s']:.1f} s)"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("gpu_uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def _once(self):
        try:
            out = subprocess.run(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=5).stdout
        except Exception:  # noqa: BLE001
            return
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            if self.uuid and self.uuid not in f[0]:
                continue
            self.samples.append(f)
            break

    def _run(self):
        while not self._stop.is_set():
            self._once()
            self._stop.wait(0.2)

    def __enter__(self):
        self._once()
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._thr.join(timeout=10)
        self._once()

    def summary(self):
        if not self.samples:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(s[1]) for s in self.samples) if v is not None)
        mx = max((v for v in (num(s[2]) for s in self.samples) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of each pass kind (minimum-pass model)
# ---------------------------------------------------------------------------

def pass_bytes(d: dict) -> dict:
    c = 8 if d.get("prec", "f32") == "f32" else 16
    r = c // 2
    if d["dim"] == 3:
        nx, ny, nz = d["n"]
        npsi = nx * ny * nz
        nhalf = nz * ny * (nx + 1)
        nspec = nz * 2 * ny * (nx + 1)
        nchat = (nx + 1) * (ny + 1) * (nz + 1)
        return {"xfwd": 2 * npsi * c, "xinv": 2 * npsi * c, "E": (2 * npsi + nhalf) * c,
                "A": (2 * npsi + nhalf) * c, "col": 2 * npsi * c, "kin": 2 * npsi * c,
                "pad": (nhalf + nspec) * c, "khat": 2 * nspec * c + nchat * r}
    nx, ny = d["n"]
    npsi = nx * ny
    nhalf = ny * (nx + 1)
    return {"xfwd": 2 * npsi * c, "xinv": 2 * npsi * c, "E": (2 * npsi + nhalf) * c,
            "A": (2 * npsi + nhalf) * c, "kin": 2 * npsi * c,
            "khat": 2 * nhalf * c + (nx + 1) * (ny + 1) * r}


def step_model_bytes(d: dict) -> int:
    b = pass_bytes(d)
    if d["dim"] == 3:
        return b["A"] + 2 * b["col"] + b["kin"] + b["E"] + 2 * b["pad"] + b["khat"]
    return b["A"] + b["kin"] + b["E"] + b["khat"]


# sources that define the split step's kernels and their launch arguments; the
# DRAM counters in profiles/traffic.json stand only while these are unchanged
STEP_SOURCES = ("fse_api.cu", "fse_col_f32.cu", "fse_col_f64.cu", "fse_fft.cuh", "fse_fft_x2.cuh", "fse_internal.h",
                "fse_launch.cuh", "fse_passes.cuh", "fse_precompute.cu", "fse_x_f32.cu", "fse_x_f64.cu",
                "fse_xpass_x2.cuh")


def source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1512_03210_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        mp_ = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp_["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def traffic_for(kind: str, workload: str):
    try:
        t = json.load(open(TRAFFIC_FILE))
    except Exception:  # noqa: BLE001
        return None
    e = t.get(workload, {}).get(kind)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("bytes_per_launch")


# ---------------------------------------------------------------------------
# arithmetic ceilings measured on the device (libfse_peaks.so)
# ---------------------------------------------------------------------------

def measure_peaks(torch, dev, stream):
    """DFMA, FFMA and packed FFMA2 throughput (TFLOP/s) of this GPU, with the
    SM clock sampled while each probe runs: the FP64 path of the split step is
    bounded by the first, the float passes by instruction issue."""
    import ctypes as ct
    from paper_1512_03210_gb300 import build as B
    lib = ct.CDLL(B.PEAKS_LIB)
    lib.fse_peak_run.restype = ct.c_int
    lib.fse_peak_run.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                 ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.zeros(16, dtype=torch.float64, device=dev)
    out = {}
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        pass
    for kind, name, iters in ((0, "fp64_dfma", 2000), (1, "fp32_ffma", 100000), (2, "fp32_ffma2", 50000)):
        ms, fl = ct.c_double(), ct.c_double()
        blocks = sms * 8
        lib.fse_peak_run(kind, blocks, max(1, iters // 10), ct.c_void_p(scratch.data_ptr()),
                         ct.c_void_p(stream.cuda_stream), ct.byref(ms), ct.byref(fl))
        best = None
        with ClockSampler(uuid) as clk:
            for _ in range(3):
                rc = lib.fse_peak_run(kind, blocks, iters, ct.c_void_p(scratch.data_ptr()),
                                      ct.c_void_p(stream.cuda_stream), ct.byref(ms), ct.byref(fl))
                if rc != 0:
                    raise RuntimeError(f"fse_peak_run({kind}) failed: CUDA error {rc}")
                tf = fl.value / (ms.value / 1000.0) / 1e12
                best = tf if best is None or tf > best else best
        out[name + "_tflops"] = best
        out[name + "_clocks"] = clk.summary()
    out["how"] = ("8 independent fma chains per thread, %d blocks x 256 threads, best of 3 CUDA-event-timed "
                  "launches; fma = 2 flops, packed float2 fma = 4" % (sms * 8))
    return out


def fft_flops_per_step(d: dict) -> float:
    """Flops of one split step in the 5 N log2 N convention of FFT benchmarks
    (complex transforms; a real transform counts half), unpruned: the two
    full-grid kinetic transforms and the zero-padded R2C / C2R convolution."""
    nx, ny, nz = d["n"]
    n = nx * ny * nz
    kin = 2 * 5.0 * n * math.log2(n)
    lx, ly, lz = 2 * nx, 2 * ny, 2 * nz
    cols = nx + 1
    conv = (2 * 2.5 * lx * math.log2(lx) * ny * nz            # R2C and C2R along x
            + 2 * 5.0 * ly * math.log2(ly) * cols * nz        # y forward and inverse (n_z planes)
            + 2 * 5.0 * lz * math.log2(lz) * cols * ly)       # z forward and inverse (2 n_y planes)
    return kin + conv


def cufft_step_timing(torch, d: dict, psi0, dev, stream, steps: int):
    """The same split step assembled from cuFFT (torch.fft) and plain
    elementwise torch kernels, as a comparison for the hand-written passes.
    Its kernel transform is the FFT of the sampled, cube-truncated kernel on
    the padded grid rather than the Gaussian-sum one: the values differ
    slightly, the cost does not."""
    nx, ny, nz = d["n"]
    L = [d["hi"][j] - d["lo"][j] for j in range(3)]
    h = [L[j] / d["n"][j] for j in range(3)]
    f32, c64 = torch.float32, torch.complex64
    with torch.cuda.stream(stream):
        k = [2 * math.pi * torch.fft.fftfreq(d["n"][j], d=h[j], device=dev, dtype=torch.float64) for j in range(3)]
        K2 = k[2][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[0][None, None, :] ** 2
        theta = (d["dt"] / 4) * K2 ** d["s"]
        kin_half = torch.exp(-1j * theta).to(c64)
        kin_full = torch.exp(-2j * theta).to(c64)
        del K2, theta
        # padded-grid kernel: samples of 1/(4 pi |x|) on the doubled box, zero at the origin
        xs = [torch.fft.fftfreq(2 * d["n"][j], d=1.0 / (2 * L[j]), device=dev, dtype=f32) for j in range(3)]
        r = torch.sqrt(xs[2][:, None, None] ** 2 + xs[1][None, :, None] ** 2 + xs[0][None, None, :] ** 2)
        U = torch.where(r > 0, 1.0 / (4 * math.pi * r.clamp_min(1e-30)), torch.zeros_like(r))
        chat = (torch.fft.rfftn(U) * (h[0] * h[1] * h[2])).real.contiguous()
        del r, U
        kp = [2 * math.pi * torch.fft.fftfreq(2 * d["n"][j], d=h[j], device=dev, dtype=f32) for j in range(3)]
        kxr = kp[0][: nx + 1].abs()
        ax = [d["lo"][j] + h[j] * torch.arange(d["n"][j], device=dev, dtype=f32) for j in range(3)]
        psi = torch.as_tensor(psi0).to(dev, c64)
        n3 = d["dip_n"]
        om = d["omega"]

        def step(n, first):
            ta, tb = n * d["dt"], (n + 1) * d["dt"]
            X = torch.fft.fftn(psi)
            X *= kin_half if first else kin_full
            u1 = torch.fft.ifftn(X)
            rho = u1.real ** 2 + u1.imag ** 2
            R = torch.fft.rfftn(rho, s=(2 * nz, 2 * ny, 2 * nx))
            # time-integrated dipole matrix M (midpoint rule) and the DDI multiplier
            tm = 0.5 * (ta + tb)
            c, sn = math.cos(om * tm), math.sin(om * tm)
            m = (c * n3[0] - sn * n3[1], sn * n3[0] + c * n3[1], n3[2])
            dt = tb - ta
            qk = (m[0] * kxr[None, None, :] + m[1] * kp[1][None, :, None] + m[2] * kp[2][:, None, None]) ** 2
            khat = (-dt) + 3 * dt * qk * chat
            R *= khat
            phi = torch.fft.irfftn(R, s=(2 * nz, 2 * ny, 2 * nx))[:nz, :ny, :nx]
            g = d["gamma"]
            P = 0.5 * dt * (g[0] ** 2 * (ax[0] ** 2)[None, None, :] + g[1] ** 2 * (ax[1] ** 2)[None, :, None]
                            + g[2] ** 2 * (ax[2] ** 2)[:, None, None])
            th = (d["beta"] * dt) * rho + d["lam"] * phi + P
            return u1 * torch.polar(torch.ones_like(th), -th)

        for n in range(3):
            psi = step(n, n == 0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for n in range(steps):
            psi = step(3 + n, False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        # the transforms alone: 3D C2C of psi (256^3) and the padded R2C / C2R (512^3)
        def timed(fn, reps=5):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            return a.elapsed_time(b) / reps
        rho = psi.real ** 2
        R = torch.fft.rfftn(rho, s=(2 * nz, 2 * ny, 2 * nx))
        out = {"split_steps_per_s": 1000.0 / ms, "ms_per_step": ms, "steps": steps,
               "c2c_256cubed_ms": timed(lambda: torch.fft.fftn(psi)),
               "r2c_padded_512cubed_ms": timed(lambda: torch.fft.rfftn(rho, s=(2 * nz, 2 * ny, 2 * nx))),
               "c2r_padded_512cubed_ms": timed(lambda: torch.fft.irfftn(R, s=(2 * nz, 2 * ny, 2 * nx))),
               "note": "torch.fft (cuFFT) plus elementwise torch kernels; not the product path"}
    return out


# ---------------------------------------------------------------------------

def run_reference(args, rank: int):
    if rank != 0:
        return 0
    nst = max(1, min(args.steps, 2))
    proc, q = start_oracle(nst)
    r = finish_oracle(proc, q)
    cb = oracle_baseline_dict(r)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": r.get("steps"), "warmup": 0,
            "ms_per_step": (1000.0 * r["seconds"] / r["steps"]) if r.get("ok") else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [256, 256, 256],
                                             "padded": [512, 512, 512], "kernel": "ddi3d"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """Slowest rank's timed-region length (ms); the job is done when it is."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput: every replica advances its own grid `steps` times."""
    return world * steps / (ms_max / 1000.0)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fse", choices=["fse", "reference"])
    ap.add_argument("--f64-steps", type=int, default=40)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--oracle-steps", type=int, default=1)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--gs-steps", type=int, default=20)
    ap.add_argument("--others", type=int, default=1, help="1: also time the other workloads")
    ap.add_argument("--peaks", type=int, default=1, help="1: measure DFMA/FFMA/FFMA2 throughput")
    ap.add_argument("--cufft-steps", type=int, default=20, help="steps of the cuFFT comparison (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    import fse_inputs as I
    import paper_1512_03210_gb300 as fse

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    d = I.workload(WORKLOAD)
    psi0 = I.psi0(WORKLOAD)
    stream = torch.cuda.current_stream(dev)
    plan = fse.Plan(d, stream=stream, device=dev)
    x = plan.to_device(psi0)
    t = 0.0
    plan.step(x, t, args.warmup)
    t += args.warmup * d["dt"]
    torch.cuda.synchronize(dev)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        pass
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = plan.launches
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(uuid) as clk:
        ev0.record(stream)
        plan.step(x, t, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = plan.launches - l0
    t += args.steps * d["dt"]
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    value = job_value(args.steps, ms, world)

    # per-kernel event timing over a second region of the same length
    fse.fse_plan_profile(plan.handle, True)
    plan.step(x, t, args.steps)
    torch.cuda.synchronize(dev)
    prof = fse.fse_plan_profile_read(plan.handle)
    fse.fse_plan_profile(plan.handle, False)
    t += args.steps * d["dt"]
    tot = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    pb = pass_bytes(d)
    peak, peak_kind = measured_peak()
    avg_ms = prof[dom][0] / max(1, prof[dom][1])
    achieved = pb[dom] / (avg_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"of {peak_kind} (copy bandwidth)",
                "traffic": traffic_for(dom, WORKLOAD), "algorithmic_bytes": pb[dom],
                "avg_launch_ms": avg_ms,
                "share": prof[dom][0] / tot if tot > 0 else None}
    step_bytes = step_model_bytes(d)
    kernels = {k: {"ms": v[0], "launches": v[1], "share": v[0] / tot if tot else 0.0,
                   "gbs": (pb[k] * v[1] / (v[0] / 1000.0) / 1e9) if (v[1] and k in pb and v[0] > 0) else None}
               for k, v in prof.items() if v[1]}

    # float64 GPU path on the same workload (same scheme, same accuracy class)
    f64 = None
    if args.f64_steps > 0:
        d64 = dict(d, prec="f64")
        plan64 = fse.Plan(d64, stream=stream, device=dev)
        x64 = plan64.to_device(psi0)
        plan64.step(x64, 0.0, 3)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan64.step(x64, 3 * d["dt"], args.f64_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        v64 = args.f64_steps / (e0.elapsed_time(e1) / 1000.0)
        f64 = {"value": v64, "unit": UNIT, "steps": args.f64_steps, "speedup_f32_over_f64": value / world / v64}
        del plan64, x64

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if args.e2e_steps > 0:
        host = torch.from_numpy(np.ascontiguousarray(psi0.astype(np.complex64))).pin_memory().numpy()
        plan.step_host(host, 0.0, 1)
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            plan.step_host(host, i * d["dt"], 1)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * args.e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(host.nbytes),
               "calls": args.e2e_steps, "note": "one fse_step_host call (1 split step) per step"}

    # batched 2D workload: 256 independent runs of mixed sizes advanced together
    batched = None
    if args.batched_steps > 0:
        runs = I.batched_runs()
        bt = fse.Batch(runs, stream=stream, device=dev)
        xs = bt.to_device([I.psi0(r) for r in runs])
        # the first call with this step count captures the launch graph; the
        # timed call replays it
        bt.step(xs, 0.0, args.batched_steps)
        torch.cuda.synchronize(dev)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lb = bt.launches
        b0.record(stream)
        bt.step(xs, args.batched_steps * 1e-3, args.batched_steps)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        bms = b0.elapsed_time(b1)
        pts = sum(r["n"][0] * r["n"][1] for r in runs)
        bb = sum(step_model_bytes(dict(r, prec="f32")) for r in runs)
        batched = {"workload": "batched_2d", "runs": len(runs), "steps": args.batched_steps,
                   "run_steps_per_s": len(runs) * args.batched_steps / (bms / 1000.0),
                   "grid_point_steps_per_s": pts * args.batched_steps / (bms / 1000.0),
                   "ms_per_batch_step": bms / args.batched_steps, "launches": bt.launches - lb,
                   "model_bytes_per_batch_step": bb,
                   "model_frac_of_hbm": bb * args.batched_steps / (bms / 1000.0) / 1e9 / peak,
                   "graph": "launches captured once per step count, replayed",
                   "sizes": sorted({r["n"][0] for r in runs})}
        del bt, xs

    # the other configurations: steps/s of the 2D Coulomb (float64) and 128^3
    # dipolar (float32) runs, and forward + adjoint steps/s of the gradient run
    others = None
    if args.others:
        others = {}
        for name in ("2d_coulomb_128", "3d_dipolar_128"):
            dc = I.workload(name)
            pc = fse.Plan(dc, stream=stream, device=dev)
            xc = pc.to_device(I.psi0(name))
            pc.step(xc, 0.0, 5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pc.step(xc, 5 * dc["dt"], dc["steps"])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            others[name] = {"split_steps_per_s": dc["steps"] / (e0.elapsed_time(e1) / 1000.0),
                             "steps": dc["steps"], "dtype": dc["prec"]}
            del pc, xc
        from paper_1512_03210_gb300 import autograd as AG
        da = I.workload("adjoint_2d_256")
        pa = fse.Plan(da, stream=stream, device=dev)
        gam = torch.tensor(I.adjoint_gammas(da["steps"]), dtype=torch.float64)
        tgt = pa.to_device(I.adjoint_target(da))
        cell = float(np.prod([(da["hi"][j] - da["lo"][j]) / da["n"][j] for j in range(2)]))

        def fwd_bwd():
            x0 = pa.to_device(I.psi0("adjoint_2d_256")).requires_grad_(True)
            g = gam.clone().requires_grad_(True)
            J = AG.overlap_objective(AG.evolve(pa, x0, g), tgt, cell)
            J.backward()
            return J
        fwd_bwd()
        torch.cuda.synchronize(dev)
        t0a = time.perf_counter()
        fwd_bwd()
        torch.cuda.synchronize(dev)
        sa = time.perf_counter() - t0a
        others["adjoint_2d_256"] = {"gradient_steps_per_s": da["steps"] / sa, "steps": da["steps"],
                                     "dtype": da["prec"],
                                     "note": "forward with sqrt(T) checkpoints, recomputation and adjoint; host-timed"}
        del pa

    # GF-GauSum ground state (Section 3.2): normalised gradient-flow steps, each a
    # BiCGStab solve through the library's FFT passes (the call synchronises)
    gs = None
    if args.gs_steps > 0:
        dg = I.workload(GS_WORKLOAD)
        pg = fse.Plan(dg, stream=stream, device=dev)
        xg = pg.to_device(I.psi0(GS_WORKLOAD))
        nbg = fse.fse_ground_state_workspace(pg.handle)
        wsg = torch.empty(nbg, dtype=torch.uint8, device=dev)
        fse.fse_ground_state(pg.handle, xg, wsg, nbg, dg["dt"], 2, 0.0, 500, GS_INNER_TOL)
        lg = pg.launches
        t0g = time.perf_counter()
        info = fse.fse_ground_state(pg.handle, xg, wsg, nbg, dg["dt"], args.gs_steps, 0.0, 500, GS_INNER_TOL)
        sec = time.perf_counter() - t0g
        gs = {"workload": GS_WORKLOAD, "grid": list(dg["n"]), "dtype": "f64", "gf_steps": info["outer"],
              "gf_steps_per_s": info["outer"] / sec, "ms_per_gf_step": 1000 * sec / max(1, info["outer"]),
              "inner_iterations": info["inner"], "ms_per_inner_iteration": 1000 * sec / max(1, info["inner"]),
              "last_change": info["change"], "launches": pg.launches - lg,
              "note": "host-timed around the call; BiCGStab scalars stay on the device, each inner iteration is a replayed CUDA graph, the host polls the residual one iteration behind"}
        del pg, xg, wsg

    # arithmetic ceilings of this GPU, and the same step built from cuFFT
    peaks = measure_peaks(torch, dev, stream) if args.peaks else None
    if f64 is not None:
        fl = fft_flops_per_step(d)
        f64["fft_flops_per_step"] = fl
        f64["tflops_5nlogn"] = fl * f64["value"] / 1e12
        if peaks:
            f64["frac_of_dfma_peak"] = f64["tflops_5nlogn"] / peaks["fp64_dfma_tflops"]
        f64["flops_note"] = ("5 N log2 N flops per complex transform (half for real), unpruned, "
                             "against the measured DFMA throughput")
    cufft = cufft_step_timing(torch, d, psi0, dev, stream, args.cufft_steps) if args.cufft_steps > 0 else None

    if rank != 0:
        return 0
    # the oracle runs after the GPU legs (spawned, single-threaded), so that it
    # never shares the host with the timed regions
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        ro = finish_oracle(*start_oracle(args.oracle_steps, 2 if args.gs_steps > 0 else 0))
        cb = oracle_baseline_dict(ro)
        if gs is not None and ro.get("gs"):
            g0 = ro["gs"]
            gs["oracle"] = {"gf_steps_per_s": g0["steps"] / g0["seconds"], "steps": g0["steps"],
                            "inner_iterations": g0["inner"], "cores": 1, "kind": "oracle"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [256, 256, 256], "padded": [512, 512, 512],
                   "kernel": "ddi3d", "s": d["s"], "omega": d["omega"], "dt": d["dt"],
                   "l2": "inputs larger than L2 (psi 134 MB, padded spectrum 279 MB); no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "grid_point_steps_per_s": value * 256 ** 3,
        "model_bytes_per_step": step_bytes,
        "step_roofline_frac": step_bytes * value / world / 1e9 / peak,
        "roofline": roofline, "kernels": kernels, "f64": f64, "e2e": e2e, "batched_2d": batched, "ground_state": gs, "other_workloads": others,
        "peaks": peaks, "cufft": cufft,
        "cpu_baseline": cb, "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
