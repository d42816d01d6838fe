"""Benchmark of the GDM hot path on GB300.

One step = assemble A = I - G alpha + LU factorisation + FP64-refined solve of both plane-wave
illuminations for the 40 x 30 x 10 cell cuboid (N = 12,000, 3N = 36,000, lambda = 500 nm).
The metric is seconds per (lambda, N) solve (lower is better).

    python bench.py [--gpus N --steps K --warmup W --precision tf32|fp32|fp64 --impl ours|reference]

Under torchrun each rank solves its own copy of the problem (independent units, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# refinement stop: the last relative correction (False) or the error estimated from the contraction of the last
# two corrections (True, the default); set from --stop
ERR_EST = True
METRIC = "GDM assemble+solve s per (λ,N) vs FP64 GPU path at 1e-9 rel err; adjoint grad s"
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop/FMA x max clock
# FP32 thread instructions per (target, source) pair, 2 right-hand sides, of the GMRES FP32 operator
# k_green_sum_f32 (ncu count: profiles/green_sum_f32_gmres_cuboid20x15x10_ncu.md)
FP32_OPERATOR_INST_PER_PAIR = 204.0
# FP32 thread instructions per ordered pair of the adjoint's double-float gradient pair sum k_dgreen_sum_ff (G s,
# dG/dr s, dG/dk s; one right-hand side; ncu count: profiles/dgreen_sum_ff_cylinder_ncu.md)
DGREEN_FF_INST_PER_PAIR = 3627.0
# FP32 thread instructions per ordered pair, 2 right-hand sides, of the double-float residual sum
# k_green_sum_ff<3, 3, 2> (ncu count)
RESIDUAL_FF_INST_PER_PAIR = 1406.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: a scratch file (GDM_CLOCKS_DIR, default the system temporary directory); the summary
        # goes into the JSON line
        self.path = os.path.join(os.environ.get("GDM_CLOCKS_DIR", tempfile.gettempdir()), f"gdm_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[2] > 300.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_sample(nx=18, ny=14, nz=10, target_n=12000):
    """The CPU FP64 oracle as it stands on a bounded sample of the workload: the same cuboid
    recipe at nx*ny*nz cells, assembly + dense solve (LAPACK zgesv through numpy), scaled to N = target_n
    by N^2 (assembly) and N^3 (solve)."""
    import numpy as np
    import gdm_workloads as W
    import oracle as O
    s = W.cuboid_precision(nx, ny, nz)
    pr = O.Problem(s.pos, float(s.wavelengths[0]), 3, eps=s.eps, step=s.step)
    t0 = time.perf_counter()
    A = pr.matrix()
    F0 = pr.plane_wave(s.e0)
    t1 = time.perf_counter()
    np.linalg.solve(A, F0)
    t2 = time.perf_counter()
    ratio = target_n / s.n
    est = (t1 - t0) * ratio ** 2 + (t2 - t1) * ratio ** 3
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if os.environ.get("OPENBLAS_NUM_THREADS") == "1":
        cores = 1
    return {"value": est, "unit": "s", "cores": cores, "kind": "oracle",
            "assembly_s": (t1 - t0) * ratio ** 2, "zgesv_s": (t2 - t1) * ratio ** 3,
            "sample": f"oracle assemble+solve of the same cuboid recipe at {nx}x{ny}x{nz} cells (N={s.n}, "
                      f"{t2 - t0:.2f} s measured: assembly {t1 - t0:.2f} s, LAPACK zgesv {t2 - t1:.2f} s), "
                      f"scaled to N={target_n} by N^2 (assembly) and N^3 (solve)"}


def cpu_oracle_one_core(nx=12, ny=10, nz=10):
    """The same sample on one host core: a child process with one BLAS thread (the oracle's assembly is
    single-threaded numpy already), so that the parent's BLAS pool is untouched."""
    code = ("import json, bench; print(json.dumps(bench.cpu_oracle_sample(%d, %d, %d)))" % (nx, ny, nz))
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # the one-core figure is context only
        return {"unavailable": f"{type(e).__name__}: {e}"}


def oracle_full_size_records():
    """Wall times of the oracle's full-size solve of the 40 x 30 x 10 cuboid (N = 12,000), measured once per
    host by oracle/make_golden_cuboid.py and stored beside its golden fields."""
    out = {}
    for tag, name in (("dev_host_x86", "cuboid40x30x10_oracle.json"),
                      ("gb300_host", "cuboid40x30x10_oracle_gb300_host.json")):
        try:
            with open(os.path.join(ROOT, "tests", "golden", name)) as f:
                r = json.load(f)
            out[tag] = {"total_s": r["total_s"], "assembly_s": r["assembly_s"], "zgesv_s": r["solve_s"],
                        "host": r["host"], "runs": 1}
        except (OSError, KeyError, ValueError):
            pass
    return out


def cpu_baseline_leg():
    """cpu_baseline of the bench line: the bounded sample on all host cores (the value), its one-core
    counterpart, and the stored full-size measurements."""
    cb = cpu_oracle_sample()
    cb["one_core"] = cpu_oracle_one_core()
    cb["full_size_measured"] = oracle_full_size_records()
    return cb


def golden_fields():
    """The oracle's dense FP64 solution of the 40 x 30 x 10 cuboid (tests/golden), or None."""
    try:
        import numpy as np
        return np.load(os.path.join(ROOT, "tests", "golden", "cuboid40x30x10_oracle.npz"))["F"]
    except Exception:
        return None


def adjoint_leg(G, ctx, dev, precision, warmup, steps):
    """Differentiation workload: dielectric cylinder r = 80 nm, h = 100 nm, d = 10 nm, eps = 12.25 + 0.05i,
    8 wavelengths 450-800 nm, x-polarised plane wave; L = sum over the wavelengths of |E|^2 at a probe
    50 nm above the top face plus sigma_sca; gradients with respect to every cell position, every cell
    eps and each wavelength through the autograd wrappers (forward solve + adjoint backward)."""
    import torch
    import gdm_workloads as W
    from paper_2505_09545_gb300 import autograd as AG
    cyl = W.cylinder_diff()
    pos = torch.tensor(cyl.pos, device=dev, requires_grad=True)
    eps = torch.tensor(cyl.eps, device=dev, requires_grad=True)
    rp = torch.tensor(cyl.r_eval, device=dev)
    wls = torch.tensor([float(l) for l in cyl.wavelengths], dtype=torch.float64, device=dev, requires_grad=True)

    def run():
        pos.grad = None
        eps.grad = None
        wls.grad = None
        t0 = time.perf_counter()
        # all wavelengths solved (and, in the backward, adjoint-solved) concurrently
        F, sig = AG.scatter_spectrum(pos, eps, wls, ctx, cyl.step, cyl.e0, precision=precision)
        L = 0.0
        for i in range(wls.shape[0]):
            E = AG.nearfield(pos, eps, wls[i], F[i], rp, ctx, cyl.step, cyl.e0)
            L = L + (E.abs() ** 2).sum() + sig[i, :, 1].sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1

    for _ in range(max(3, warmup)):
        run()
    fw, bw = [], []
    for _ in range(max(1, steps)):
        a, b = run()
        fw.append(a)
        bw.append(b)
    f, b = statistics.median(fw), statistics.median(bw)
    # one wavelength's backward with phase accounting on this context: the adjoint solve (triangular solves
    # with the forward factors and its refinement residuals) and the gradient pair sums dG/dr, dG/dk (FP64,
    # two launches over the n (n - 1) ordered pairs)
    wl0 = wls[:1].detach().clone().requires_grad_(True)
    F1, sig1 = AG.scatter(pos, eps, wl0[0], ctx, cyl.step, cyl.e0, precision=precision)
    E1 = AG.nearfield(pos, eps, wl0[0], F1, rp, ctx, cyl.step, cyl.e0)
    L1 = (E1.abs() ** 2).sum() + sig1[:, 1].sum()
    torch.cuda.synchronize()
    ctx.phases(True)
    L1.backward()
    ph = ctx.phases(False)
    pairs = 2.0 * cyl.n * (cyl.n - 1)
    grad = {"gradient_ms": ph["gradient"], "adjoint_solves_ms": ph["correction_solves"],
            "adjoint_residual_ms": ph["residual"], "pairs": pairs,
            "note": "one wavelength's gdm_backward on one context (the timed spectrum runs the 8 concurrently)"}
    if DGREEN_FF_INST_PER_PAIR and ph["gradient"] > 0:
        peak = 152 * 128 * 2.07e9
        ach = pairs * DGREEN_FF_INST_PER_PAIR / (ph["gradient"] / 1e3)
        grad["roofline"] = {"bound": "alu", "kernel": "k_dgreen_sum_ff (double-float pair sums of G, dG/dr, dG/dk)",
                            "achieved": ach, "peak": peak, "unit": "FP32 inst/s", "frac": ach / peak,
                            "inst_per_pair": DGREEN_FF_INST_PER_PAIR,
                            "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock)"}
    return {"value": f + b, "unit": "s", "forward_s": f, "backward_s": b, "precision": precision,
            "backward_one_wavelength": grad,
            "workload": f"cylinder r=80 h=100 d=10 nm (N={cyl.n}), eps=12.25+0.05i, {wls.shape[0]} wavelengths "
                        "450-800 nm, x-pol; L = sum |E(probe)|^2 + sigma_sca; grads wrt all positions, eps, lambda",
            "timing": "wall clock with device synchronisation, median of the timed repetitions"}


def fp64_compare(G, ctx, dev, precision, cuboid, tol, golden=None):
    """The plain FP64 GPU path (FP64 assembly, FP64 LU, FP64 solve) against the mixed-precision path on
    the same cuboid: seconds per assemble+solve and the relative field difference between the two (and,
    where the oracle's stored solution of this cuboid exists, each path's error against it). The FP64
    path is warmed up on a 3N = 1,800 cuboid (allocations, module loading) and timed once: one full-size
    FP64 solve takes minutes, so its launch overheads are far below the timer's resolution."""
    import torch
    import gdm_workloads as W
    nx, ny, nz = (int(v) for v in cuboid.split("x"))
    out = {}
    fields = {}

    def run(prec, nxyz, reps, t):
        s = W.cuboid_precision(*nxyz)
        lam = float(s.wavelengths[0])
        pos = torch.tensor(s.pos, device=dev)
        prob = G.GDMProblem(pos, lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
        F0 = G.incident_planewave(ctx, pos, lam, s.e0)
        A = torch.empty((prob.size, G.padded_lda(prob.size)),
                        dtype=torch.complex128 if prec == "fp64" else torch.complex64, device=dev)
        ipiv = torch.empty(prob.size, dtype=torch.int32, device=dev)
        F = torch.empty_like(F0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            G.assemble(ctx, prob, prec, out=A)
            G.solve(ctx, prob, A, F0, prec, ipiv=ipiv, F=F, tol=t, err_estimate=ERR_EST and prec != "fp64")
        e1.record()
        torch.cuda.synchronize()
        del A
        return e0.elapsed_time(e1) / reps / 1e3, F, s

    run("fp64", (10, 6, 10), 1, 0.0)                     # warm-up
    out["fp64"], fields["fp64"], s = run("fp64", (nx, ny, nz), 1, 0.0)
    run(precision, (nx, ny, nz), 1, tol)                 # warm-up
    out[precision], fields[precision], _ = run(precision, (nx, ny, nz), 3, tol)
    d = (fields[precision] - fields["fp64"]).norm(dim=1) / fields["fp64"].norm(dim=1)
    res = {"workload": f"cuboid {nx}x{ny}x{nz} (3N={3 * s.n})", "fp64_s": out["fp64"],
           f"{precision}_s": out[precision], "speedup": out["fp64"] / out[precision],
           "rel_field_diff_vs_fp64": float(d.max()), "tol": tol,
           "fp64_tflops": 8.0 / 3.0 * (3.0 * s.n) ** 3 / out["fp64"] / 1e12,
           "timing": "CUDA events; FP64 one timed run (after a warm-up on a 3N=1,800 cuboid), "
                     "mixed precision the mean of three after one warm-up"}
    if golden is not None and (nx, ny, nz) == (40, 30, 10):
        import numpy as np
        for prec in ("fp64", precision):
            Fh = fields[prec].cpu().numpy().T
            res[f"{prec}_field_err_vs_oracle"] = float(np.max(np.linalg.norm(Fh - golden, axis=0)
                                                              / np.linalg.norm(golden, axis=0)))
    return res


def precision_leg(G, ctx, dev, precision, tol, golden, reps=3):
    """The headline cuboid step (assemble + LU + refined solve) in another factor precision: seconds per step
    (CUDA events, mean of `reps` after one warm-up), refinement steps, the fields' error against the stored
    oracle solution, and the trailing update's rate (CUDA events on its launch stream)."""
    import numpy as np
    import torch
    import gdm_workloads as W
    s = W.cuboid_precision()
    lam = float(s.wavelengths[0])
    pos = torch.tensor(s.pos, device=dev)
    prob = G.GDMProblem(pos, lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0)
    A = torch.empty((prob.size, G.padded_lda(prob.size)), dtype=torch.complex64, device=dev)
    ipiv = torch.empty(prob.size, dtype=torch.int32, device=dev)
    F = torch.empty_like(F0)

    def step():
        G.assemble(ctx, prob, precision, out=A)
        return G.solve(ctx, prob, A, F0, precision, ipiv=ipiv, F=F, tol=tol, err_estimate=ERR_EST)[2]

    step()
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        info = step()
    e1.record()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    out = {"precision": precision, "s": e0.elapsed_time(e1) / reps / 1e3, "refine_iters": info["iterations"],
           "rel_residual_fp64": info["rel_residual"],
           "trailing_update_tflops": prof["flops"] / (prof["ms"] / 1e3) / 1e12 if prof["ms"] > 0 else None}
    if golden is not None:
        Fh = F.cpu().numpy().T
        out["field_err_vs_oracle"] = float(np.max(np.linalg.norm(Fh - golden, axis=0) / np.linalg.norm(golden, axis=0)))
    del A
    return out


def traffic_record(kernel_src, algorithmic_bytes_per_launch):
    """Per-launch DRAM traffic of the trailing update: the ratio of DRAM bytes to algorithmic bytes from the
    committed ncu capture of one launch of the 3N = 9,000 case, times this run's algorithmic bytes per launch
    (C, the largest term, scales with m^2 in both); None unless the capture was taken on the kernel source as
    it is now (sha256 of the file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "tc_update_pair_tf32_cuboid20x15x10_ncu.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = dict(re.findall(r"^- (\w+): (\S+)$", txt, flags=re.M))
    src = os.path.join(ROOT, "paper_2505_09545_gb300", "csrc", kernel_src)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if vals.get("source_sha256") != sha:
        return None
    try:
        return float(vals["traffic_over_algorithmic"]) * algorithmic_bytes_per_launch
    except (KeyError, ValueError):
        return None


# FP32 thread instructions per (evaluation point, dipole) pair, 2 right-hand sides, E and H, of the near-field
# kernel k_green_sum_ff<3, 6, 2> (ncu count: profiles/green_sum_ff_nearfield_cuboid20x15x10_ncu.md)
NEARFIELD_INST_PER_PAIR = 2175.0


def nearfield_leg(G, ctx, dev, prob, F, n_side=320, reps=5):
    """Near field of the solved cuboid on a map above it: n_side^2 points (102,400 by default) on the plane
    z = 100 nm (50 nm above the top face) spanning +-400 nm, E and H for both illuminations, by one
    gdm_nearfield call (double-float Green sums over every (point, dipole) pair). Against the FP32 issue
    peak: ncu instructions per pair x pairs / CUDA-event time of the whole call (moment and target
    preparation, O(N + M), included)."""
    import torch
    import gdm_workloads as W
    r = torch.tensor(W.nearfield_plane(n_side, 400.0, 100.0), device=dev)
    m = r.shape[0]
    G.nearfield(ctx, prob, F, r)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        E, H = G.nearfield(ctx, prob, F, r)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / reps / 1e3
    pairs = float(m) * prob.n
    peak = 152 * 128 * 2.07e9
    out = {"workload": f"{m} points (plane z=100 nm, +-400 nm) x {prob.n} dipoles, E and H, {F.shape[0]} RHS",
           "s": s, "pairs_per_s": pairs / s}
    if NEARFIELD_INST_PER_PAIR:
        ach = pairs * NEARFIELD_INST_PER_PAIR / s
        out["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "FP32 inst/s", "frac": ach / peak,
                           "inst_per_pair": NEARFIELD_INST_PER_PAIR,
                           "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock)"}
    return out


def run_nearfield(args):
    """Near-field map of the solved 40 x 30 x 10 cuboid (N = 12,000): one step = one gdm_nearfield call over
    320 x 320 points, E and H, both illuminations."""
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nx, ny, nz = (int(v) for v in args.cuboid.split("x"))
    s = W.cuboid_precision(nx, ny, nz)
    lam = float(s.wavelengths[0])
    ctx = G.Context(local)
    pos = torch.tensor(s.pos, device=dev)
    prob = G.GDMProblem(pos, lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0)
    A = G.assemble(ctx, prob, args.precision)
    F, _, _ = G.solve(ctx, prob, A, F0, args.precision)
    del A
    for _ in range(max(1, args.warmup)):
        nearfield_leg(G, ctx, dev, prob, F, args.nearfield_side, 1)
    leg = nearfield_leg(G, ctx, dev, prob, F, args.nearfield_side, args.steps)
    line = {"metric": "near-field map s", "value": leg["s"], "unit": "s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": leg["s"] * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2 (double-float)", "data": "synthetic",
            "config": {"workload": f"cuboid {nx}x{ny}x{nz} (N={s.n}) solved fields; " + leg["workload"]},
            "pairs_per_s": leg["pairs_per_s"], "roofline": leg.get("roofline")}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def metasurface_leg(G, ctx, dev, precision, tol, eps_env, warmup, steps, peaks, units=None):
    """ED/MD metasurface: 64 x 64 dipoles (6N = 24,576), Lorentzian 6x6 polarisabilities, 32 wavelengths
    500-800 nm, x- and y-polarised normal incidence; per wavelength on the GPU: polarisabilities, incident
    field, assemble + mixed-precision LU + FP64-refined solve + cross sections. One step = all 32
    wavelengths; the value is seconds per (lambda, N) solve. Also: the assembly kernel alone against HBM,
    and the whole wavelength's (8/3)(6N)^3 LU flops against the TF32 denominator. units = (lo, hi): only the
    wavelengths [lo, hi) (this rank's share of the spectrum)."""
    import numpy as np
    import torch
    import gdm_workloads as W
    s = W.metasurface_edmd()
    if units is not None:
        s.wavelengths = s.wavelengths[units[0]:units[1]]
    pos = torch.tensor(s.pos, device=dev)
    ns = 6 * s.n
    A = torch.empty((ns, G.padded_lda(ns)), dtype=torch.complex64, device=dev)
    ipiv = torch.empty(ns, dtype=torch.int32, device=dev)
    w0e = torch.tensor(s.omega0_e, device=dev)
    w0m = torch.tensor(s.omega0_m, device=dev)
    al = torch.empty((s.n, 6, 6), dtype=torch.complex128, device=dev)
    sig = torch.empty((len(s.wavelengths), 3, 2), dtype=torch.float64, device=dev)
    infos = []

    def step():
        infos.clear()
        for i, lam in enumerate(s.wavelengths):
            lam = float(lam)
            G.alpha6_lorentz(ctx, w0e, w0m, s.gamma_ev, s.amp_nm, lam, out=al, eps_env=eps_env)
            prob = G.GDMProblem(pos, lam, 6, alpha6=al, eps_env=eps_env)
            F0 = G.incident_planewave(ctx, pos, lam, s.e0, kind_out=6, eps_env=eps_env)
            G.assemble(ctx, prob, "fp32", out=A)
            F, _, info = G.solve(ctx, prob, A, F0, precision, ipiv=ipiv, tol=tol, err_estimate=ERR_EST)
            e, c, b = G.cross_sections(ctx, prob, F0, F, np.ones(2))
            sig[i, 0], sig[i, 1], sig[i, 2] = e, c, b
            infos.append(info)

    for _ in range(max(1, warmup)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nl = len(s.wavelengths)
    # one extra (untimed) wavelength with per-phase device-time accounting, plus its assembly alone
    lam = float(s.wavelengths[0])
    G.alpha6_lorentz(ctx, w0e, w0m, s.gamma_ev, s.amp_nm, lam, out=al, eps_env=eps_env)
    prob = G.GDMProblem(pos, lam, 6, alpha6=al, eps_env=eps_env)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0, kind_out=6, eps_env=eps_env)
    G.assemble(ctx, prob, "fp32", out=A)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record()
    for _ in range(5):
        G.assemble(ctx, prob, "fp32", out=A)
    eb.record()
    torch.cuda.synchronize()
    asm_ms = ea.elapsed_time(eb) / 5
    asm_bytes = float(ns) * ns * 8
    ctx.phases(True)
    G.solve(ctx, prob, A, F0, precision, ipiv=ipiv, tol=tol, err_estimate=ERR_EST)
    phases = {k: round(v, 2) for k, v in ctx.phases(False).items()}
    per_lam = ms / 1e3 / nl
    tf32_peak = peaks["bf16_tflops_sustained"] * NOMINAL_TF32_OVER_BF16
    lu_flops = 8.0 / 3.0 * float(ns) ** 3
    del A
    return {"value": per_lam, "unit": "s", "steps": steps, "ms_per_step": ms,
            "workload": f"ED/MD metasurface 64x64, pitch 400 nm (6N={ns}), Lorentzian alpha_e, alpha_m omega0~U[2,3] "
                        f"eV, width 0.1 eV, seed 4; {nl} wavelengths 500-800 nm, x/y-pol; assemble + LU + "
                        f"FP64-refined solve + cross sections per wavelength; host eps_env={eps_env:g}; relative "
                        f"correction <= {tol:g}",
            "accuracy": {"max_refine_iters": max(i["iterations"] for i in infos),
                         "max_rel_residual_fp64": max(i["rel_residual"] for i in infos),
                         "refactored": int(sum(bool(i["refactored"]) for i in infos))},
            "sigma_ext_range_nm2": [float(sig[:, 0].min()), float(sig[:, 0].max())], "sigma": sig,
            "phases_ms_one_wavelength": phases,
            "assembly_roofline": {"bound": "hbm", "achieved": asm_bytes / (asm_ms / 1e3) / 1e9,
                                  "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": asm_bytes / (asm_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "ms": asm_ms,
                                  "bytes": asm_bytes, "kernel": "assemble A = I - G alpha, 6x6 blocks"},
            "lu_tensor_frac_whole_wavelength": {"flops": lu_flops, "tflops": lu_flops / per_lam / 1e12,
                                                "peak": tf32_peak, "frac": lu_flops / per_lam / 1e12 / tf32_peak,
                                                "note": "(8/3)(6N)^3 over the whole wavelength's time (assembly, "
                                                        "panels, solves and refinement included)"}}


def run_adjoint(args):
    """The differentiation workload as its own line (see adjoint_leg)."""
    import torch
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = G.Context(local)
    leg = adjoint_leg(G, ctx, dev, args.precision, args.warmup, args.steps)
    line = {"metric": "adjoint gradient s (8 wavelengths, forward + backward)", "value": leg.pop("value"),
            "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic", "config": {"workload": leg.pop("workload")}, **leg}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def run_metasurface(args):
    """The ED/MD metasurface workload as its own line (see metasurface_leg). Under torchrun the 32 wavelengths
    are split contiguously across the ranks (independent units, no collective on the data path); the job's
    time is the slowest rank's and the cross sections are gathered once at the end."""
    import torch
    import paper_2505_09545_gb300 as G
    from paper_2505_09545_gb300 import shard
    import gdm_workloads as W
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    n_units = len(W.metasurface_edmd().wavelengths)
    lo, hi = shard.unit_range(n_units, ws, rank)
    ctx = G.Context(local)
    peaks, _ = load_peaks()
    clk = ClockSampler(local)
    clk.start()
    leg = metasurface_leg(G, ctx, dev, args.precision, args.tol, args.eps_env, args.warmup, args.steps, peaks,
                          units=(lo, hi))
    clocks = clk.stop()
    ms = max_over_ranks(leg.pop("ms_per_step"), ws, dev)
    sig = shard.gather_units(leg.pop("sigma"), lo, n_units)
    leg.pop("value")
    line = {"metric": METRIC, "value": ms / 1e3 / n_units, "unit": leg.pop("unit"), "n_gpus": ws,
            "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None,
            "dtype": "c64-tf32+f64" if args.precision == "tf32" else args.precision, "data": "synthetic",
            "config": {"workload": leg.pop("workload"), "precision": args.precision,
                       "parallelism": f"wavelengths split contiguously over {ws} rank(s)",
                       "l2": "inputs larger than L2 (4.8 GB complex64 matrix rewritten per wavelength)"},
            **leg, "sigma_ext_range_nm2": [float(sig[:, 0].min()), float(sig[:, 0].max())], "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def batch_roofline_sum(ss, infos, ms, precision):
    """The batch's time against the sum of its kernels' rooflines: every structure's assembly (HBM store of
    (3N)^2 complex64), LU ((8/3)(3N)^3 flops at the TF32 tensor rate), triangular solves (one pass over the
    factors per solve, initial plus one per refinement iteration, at HBM rate) and refinement residuals (one
    FP32 Green sum, then double-float ones, at the FP32 issue rate with the ncu instruction counts per pair),
    with each structure's own iteration count. frac = summed roofline time / measured time."""
    peaks, src = load_peaks()
    hbm = peaks["hbm_gbs"] * 1e9
    tc = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * 1e12
    if precision == "tf32":
        tc *= NOMINAL_TF32_OVER_BF16
    issue = 152 * 128 * 2.07e9
    asm = lu = sol = res = 0.0
    for s, info in zip(ss, infos):
        n3 = 3.0 * s.n
        it = max(1, int(info["iterations"]))
        asm += n3 * n3 * 8.0 / hbm
        lu += 8.0 / 3.0 * n3 ** 3 / tc
        sol += n3 * n3 * 8.0 * (it + 1) / hbm
        res += float(s.n) ** 2 * (FP32_OPERATOR_INST_PER_PAIR + (it - 1) * RESIDUAL_FF_INST_PER_PAIR) / issue
    ideal = asm + lu + sol + res
    return {"assembly_ms": asm * 1e3, "lu_ms": lu * 1e3, "solves_ms": sol * 1e3, "residuals_ms": res * 1e3,
            "ideal_ms": ideal * 1e3, "measured_ms": ms, "frac": ideal * 1e3 / ms,
            "peaks": f"{src}: HBM {peaks['hbm_gbs']:.0f} GB/s, tensor {tc / 1e12:.0f} TFLOP/s, "
                     f"FP32 issue {issue / 1e12:.1f} T inst/s"}


def batch_leg(G, ctx, dev, ss, precision, tol, streams, autotune, warmup, steps, ws=1):
    """The batch of structures ss through gdm_solve_batched: tuned widths (the grouped factorisation's for
    TF32, the per-problem table otherwise), warm-up, then steps timed with CUDA events. Returns the timing,
    the results' accuracy record and the batch against its summed per-kernel rooflines."""
    import torch
    probs = [G.GDMProblem(torch.tensor(s.pos, device=dev), float(s.wavelengths[0]), 3,
                          eps=torch.tensor(s.eps, device=dev), step=s.step) for s in ss]
    sizes = [p.size for p in probs]
    table, glu_nb = None, None
    if autotune and precision != "fp64":
        table = G.autotune(ctx, sizes, precision=precision)
        if precision == "tf32" and len(sizes) > 1:
            glu_nb = G.autotune_batched(ctx, sizes)
    e0s = [s.e0 for s in ss]

    def step():
        return G.solve_batched(ctx, probs, e0s, precision=precision, n_streams=streams, tol=tol,
                               err_estimate=ERR_EST)

    for _ in range(max(1, warmup)):
        out = step()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index or 0)
    clk.start()
    l0 = ctx.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batch_timed")  # profilers can select exactly the timed steps
    e0.record()
    for _ in range(steps):
        out = step()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, ws, dev)
    infos = out[2]
    return {"ms": ms, "launches": ctx.launches - l0, "clocks": clocks, "lu_block_table": table,
            "grouped_lu_block": glu_nb, "factor_ms": infos[0]["factor_ms"] if glu_nb or precision == "tf32" else None,
            "roofline_sum": batch_roofline_sum(ss, infos, ms, precision),
            "accuracy": {"tol": tol, "max_refine_iters": max(i["iterations"] for i in infos),
                         "max_rel_residual_fp64": max(i["rel_residual"] for i in infos),
                         "refactored": int(sum(i["refactored"] for i in infos))},
            "sizes_gb": sum(n * n for n in sizes) * 8 / 1e9}


BATCH_WORKLOAD = ("{n} Eden blobs, N~U{{50..1500}} cells (sum N={sum_n}), d=15 nm, eps~U[2,16], own "
                  "lambda~U[400,1000] nm each, x/y-pol; plane wave + assemble + LU + FP64-refined solve + cross "
                  "sections, one gdm_solve_batched call")


def run_batch(args):
    """Batching workload: 256 independent Eden blobs of N ~ U{50..1500} cells on a 15 nm mesh
    (3N = 150 ... 4500), eps ~ U[2,16], each at its own wavelength ~ U[400,1000] nm with x- and
    y-polarised plane waves; one step = plane wave + assemble + LU + FP64-refined solve + cross sections
    of all 256 through one gdm_solve_batched call. The value is seconds per (lambda, N) solve."""
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    from paper_2505_09545_gb300 import shard
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    ss_all = W.blob_batch(n_struct=args.batch_structs)
    # under torchrun: contiguous ranges of structures with near-equal LU work (3N)^3 per rank
    lo, hi = shard.weighted_unit_range([(3.0 * s.n) ** 3 for s in ss_all], ws, rank)
    ss = ss_all[lo:hi]
    ctx = G.Context(local)
    leg = batch_leg(G, ctx, dev, ss, args.precision, args.tol, args.streams, not args.no_autotune, args.warmup,
                    args.steps, ws)
    ms = leg["ms"]
    flops = sum(8.0 / 3.0 * (3.0 * s.n) ** 3 for s in ss_all)
    line = {"metric": METRIC, "value": ms / 1e3 / len(ss_all), "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None, "dtype": "c64-tf32+f64" if args.precision == "tf32" else args.precision,
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD.format(n=len(ss_all), sum_n=sum(s.n for s in ss_all)),
                       "precision": args.precision, "streams": args.streams or 8,
                       "lu_block_table": leg["lu_block_table"], "grouped_lu_block": leg["grouped_lu_block"],
                       "parallelism": f"structures split contiguously over {ws} rank(s) by LU work",
                       "l2": f"inputs larger than L2 ({leg['sizes_gb']:.1f} GB of complex64 "
                             "matrices rewritten every step)"},
            "batch_s": ms / 1e3, "lu_tflops_effective": flops / (ms / 1e3) / 1e12,
            "grouped_factor_ms": leg["factor_ms"], "roofline_sum": leg["roofline_sum"],
            "accuracy": leg["accuracy"], "gpu_launches": leg["launches"], "clocks": leg["clocks"]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_gpm(args):
    """Effective-model extraction: global polarizability matrix of the dielectric sphere (R = 60 nm,
    d = 10 nm, N = 925, eps = 12.25, lambda = 600 nm) with 15 effective dipole pairs at farthest-point
    sites, fitted at 200 probes on a 120 nm sphere for 80 plane waves (40 directions x 2 polarisations)
    and 16 dipole sources on a 180 nm sphere. One step = one gdm_gpm_extract call (illumination fields,
    one factorisation, 96 refined solves, probe fields, both least-squares fits)."""
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = W.sphere_plain_fp64()
    lam = float(s.wavelengths[0])
    khat, e0, ds_pos, ds_mom = W.gpm_illumination_set(n_angles=40, n_sources=16, source_radius=180.0, seed=1)
    r_gpm = W.farthest_points(s.pos, 15, 1)
    r_probe = W.sphere_points(200, 120.0, seed=2)
    ctx = G.Context(local)
    t = lambda x: torch.tensor(x, device=dev)
    prob = G.GDMProblem(t(s.pos), lam, 3, eps=t(s.eps), step=s.step)
    args_d = (t(r_gpm), t(r_probe), khat, e0, t(ds_pos), t(ds_mom))

    def step():
        return G.gpm_extract(ctx, prob, *args_d, precision=args.precision)

    for _ in range(max(1, args.warmup)):
        out = step()
    torch.cuda.synchronize()
    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0_.record()
    for _ in range(args.steps):
        out = step()
    e1_.record()
    torch.cuda.synchronize()
    ms = e0_.elapsed_time(e1_) / args.steps
    line = {"metric": "GPM extraction s (15 dipole pairs, 96 illuminations)", "value": ms / 1e3, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64-tf32+f64" if args.precision == "tf32" else args.precision, "data": "synthetic",
            "config": {"workload": f"GPM of the sphere R=60 d=10 nm (N={s.n}), eps=12.25, lambda={lam:g} nm: 15 sites, "
                                   "80 plane waves + 16 dipole sources, 200 probes"},
            "rel_fit": out[2]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def run_farfield(args):
    """Far-field scattering cross section of the solved cuboid (N = 12,000, both polarisations): one step =
    one gdm_sigma_farfield call on a 64 x 128 (Gauss-Legendre cos theta x uniform phi) grid, i.e.
    8,192 directions x 12,000 cells x 2 illuminations of phased sums in FP64."""
    import numpy as np
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = W.cuboid_precision(40, 30, 10)
    lam = float(s.wavelengths[0])
    ctx = G.Context(local)
    pos = torch.tensor(s.pos, device=dev)
    prob = G.GDMProblem(pos, lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0)
    A = G.assemble(ctx, prob, args.precision)
    F, _, _ = G.solve(ctx, prob, A, F0, args.precision)
    del A
    e2 = np.ones(2)
    for _ in range(max(1, args.warmup)):
        sig = G.sigma_farfield(ctx, prob, F, e2, 64, 128)
    torch.cuda.synchronize()
    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0_.record()
    for _ in range(args.steps):
        sig = G.sigma_farfield(ctx, prob, F, e2, 64, 128)
    e1_.record()
    torch.cuda.synchronize()
    ms = e0_.elapsed_time(e1_) / args.steps
    ext, sca, ab = G.cross_sections(ctx, prob, F0, F, e2)
    pairs = 64 * 128 * s.n * 2
    line = {"metric": "far-field sigma_sca s", "value": ms / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"cuboid 40x30x10 (N={s.n}) solved fields, 64x128 far-field grid, 2 illuminations"},
            "pairs_per_s": pairs / (ms / 1e3),
            "sigma_sca_ff_nm2": sig.cpu().tolist(), "sigma_ext_minus_abs_nm2": (ext - ab).cpu().tolist()}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def run_ldos(args):
    """Electric LDOS around the dielectric sphere (R = 60 nm, d = 10 nm, N = 925, eps = 12.25, lambda =
    600 nm) at 32 emitter positions 15 nm outside its surface: one step = one gdm_ldos call (96 dipole
    illuminations, one factorisation, refined solves, scattered fields at the emitters)."""
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = W.sphere_plain_fp64()
    lam = float(s.wavelengths[0])
    ctx = G.Context(local)
    prob = G.GDMProblem(torch.tensor(s.pos, device=dev), lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
    r0 = torch.tensor(W.sphere_points(32, 80.0, seed=3), device=dev)
    for _ in range(max(1, args.warmup)):
        out = G.ldos(ctx, prob, r0, precision=args.precision)
    torch.cuda.synchronize()
    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0_.record()
    for _ in range(args.steps):
        out = G.ldos(ctx, prob, r0, precision=args.precision)
    e1_.record()
    torch.cuda.synchronize()
    ms = e0_.elapsed_time(e1_) / args.steps
    line = {"metric": "LDOS s (32 emitter positions x 3 orientations)", "value": ms / 1e3, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64-tf32+f64" if args.precision == "tf32" else args.precision, "data": "synthetic",
            "config": {"workload": f"sphere R=60 d=10 nm (N={s.n}), eps=12.25, lambda={lam:g} nm, 32 emitters on an "
                                   "80 nm sphere, electric LDOS along x, y, z"},
            "ldos_range": [float(out.min()), float(out.max())]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def run_gmres(args):
    """Matrix-free preconditioned GMRES on a cuboid larger than the dense workload (default 80 x 60 x 10 cells,
    N = 48,000, 3N = 144,000: its dense complex64 matrix alone would take 166 GB): one step = one
    gdm_solve_gmres call (partition, coarse-model and block factorisations, FGMRES to a relative residual of
    1e-12 for both polarisations) from device-resident inputs."""
    import numpy as np
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G
    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nx, ny, nz = (int(v) for v in args.gmres_cuboid.split("x"))
    s = W.cuboid_precision(nx, ny, nz)
    lam = float(s.wavelengths[0])
    ctx = G.Context(local)
    pos = torch.tensor(s.pos, device=dev)
    prob = G.GDMProblem(pos, lam, 3, eps=torch.tensor(s.eps, device=dev), step=s.step)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0)
    F = torch.empty_like(F0)
    for _ in range(max(1, args.warmup)):
        F, info = G.solve_gmres(ctx, prob, F0, precision=args.precision if args.precision != "fp64" else "tf32", F=F)
    torch.cuda.synchronize()
    e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = G.lib().gdm_launch_count(ctx.h)
    e0_.record()
    for _ in range(args.steps):
        F, info = G.solve_gmres(ctx, prob, F0, precision=args.precision if args.precision != "fp64" else "tf32", F=F)
    e1_.record()
    torch.cuda.synchronize()
    launches = (G.lib().gdm_launch_count(ctx.h) - launches0) // args.steps
    ms = e0_.elapsed_time(e1_) / args.steps
    # operator throughput: each GMRES step (FP32 operator) and each true residual (double-float operator, at
    # the start of every restart cycle but the first, whose iterate is 0, and once at the end) is one pass over
    # all N^2 pairs for both right-hand sides
    passes = info["iterations"] + info["cycles"]
    # one more solve with phase accounting (CUDA events on the context stream around every operator
    # application): the operator kernel k_green_sum_ff (double-float pair sums on the FP32 pipes) against
    # the FP32 issue rate of 152 SMs x 128 lanes x 2.07 GHz; 1,406 FP32 thread instructions per
    # (target, source) pair for two right-hand sides (ncu count, profiles/green_sum_ff_gmres_cuboid20x15x10_ncu.md)
    ctx.phases(True)
    G.solve_gmres(ctx, prob, F0, precision=args.precision if args.precision != "fp64" else "tf32", F=F)
    ph = ctx.phases(False)
    # the dominant kernel is the FP32 operator of the Arnoldi steps (k_green_sum_f32); the double-float one
    # (k_green_sum_ff) evaluates the true residual once per restart cycle
    fast_ms, ff_ms = ph["operator_f32"], ph["residual"]
    cycles = info["cycles"]
    fast_passes = info["iterations"]
    ff_passes = passes - fast_passes
    peak_inst = 152 * 128 * 2.07e9
    inst_fast = FP32_OPERATOR_INST_PER_PAIR
    achieved = fast_passes * float(s.n) ** 2 * inst_fast / (fast_ms / 1e3) if fast_ms > 0 else 0.0
    it_ms = fast_ms + ff_ms + ph["correction_solves"] + ph["other"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_inst, "unit": "FP32 inst/s",
                "frac": achieved / peak_inst, "traffic": None, "kernel": "k_green_sum_f32 (GMRES Arnoldi operator)",
                "inst_per_pair": inst_fast, "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock)",
                "share_of_iterations": fast_ms / max(it_ms, 1e-9),
                "double_float_operator": {"passes": ff_passes, "ms": ff_ms,
                                          "fp32_inst_per_s": ff_passes * float(s.n) ** 2 * RESIDUAL_FF_INST_PER_PAIR / (ff_ms / 1e3)
                                          if ff_ms > 0 else 0.0},
                "phases_ms": {"fp32_operator": fast_ms, "double_float_operator": ff_ms,
                              "preconditioner": ph["correction_solves"], "orthogonalisation": ph["other"]},
                "restart_cycles": cycles}
    line = {"metric": "GMRES solve s per (lambda, N)", "value": ms / 1e3, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 operator, tf32 preconditioner", "data": "synthetic",
            "config": {"workload": f"cuboid {nx}x{ny}x{nz} cells, d=10 nm, N={s.n} (3N={3 * s.n}), eps~U[2,16]+iU[0,0.5] "
                                   "seed 2, lambda=500 nm, x- and y-polarised; FGMRES(60), coarse model + 512-cell blocks, "
                                   "tol 1e-12"},
            "iterations": info["iterations"], "rel_residual": info["rel_residual"],
            "setup_ms": info["factor_ms"], "iterate_ms": info["refine_ms"],
            "pair_evals_per_s": passes * float(s.n) ** 2 * 2 / (info["refine_ms"] / 1e3),
            "roofline": roofline, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()


def max_over_ranks(value, ws, device):
    """The job's time is the slowest rank's: all-reduce MAX over the process group (any backend; the
    tensor lives on `device`). Single process: the value itself."""
    if ws <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def per_unit_seconds(job_ms, ws, units_per_rank=1):
    """Replicas: every rank solves its own units; whole-job seconds per unit = slowest rank's time / all
    units of the job."""
    return job_ms / 1e3 / (ws * units_per_rank)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    cpu_oracle_sample(8, 6, 5)  # warm numpy / BLAS
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        last = cpu_oracle_sample()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(last["value"])
    v = statistics.mean(times)
    cb = dict(last)
    cb["value"] = v
    cb["full_size_measured"] = oracle_full_size_records()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(args):
    nx, ny, nz = (int(v) for v in getattr(args, "cuboid", "40x30x10").split("x"))
    n = nx * ny * nz
    return {"workload": f"cuboid {nx}x{ny}x{nz} cells, d=10 nm, N={n} (3N={3 * n}), eps~U[2,16]+iU[0,0.5] seed 2, "
                        "lambda=500 nm, x- and y-polarised plane waves; assemble + LU + FP64-refined solve "
                        + (f"(estimated relative error <= {getattr(args, 'tol', 1e-10):g}, from the contraction of "
                           "the last two corrections)" if getattr(args, "stop", "correction") == "estimate" else
                           f"(relative correction <= {getattr(args, 'tol', 1e-10):g})"),
            "precision": args.precision, "n_rhs": 2,
            "l2": "inputs larger than L2 (10.4 GB complex64 matrix rewritten every step)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="tf32", choices=["tf32", "fp32", "fp64", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10,
                    help="refinement stop: max relative correction; the fields' error is about 0.03 x tol "
                         "(measured and reported in 'accuracy'), inside the metric's 1e-9")
    ap.add_argument("--stop", default="estimate", choices=["correction", "estimate"],
                    help="refinement stop rule: the last relative correction <= tol, or the relative error "
                         "estimated from the contraction of the last two corrections <= tol")
    ap.add_argument("--cuboid", default="40x30x10",
                    help="cells per axis of the cuboid workload (smaller cases are for profiling only)")
    ap.add_argument("--fp64-cuboid", default="40x30x10",
                    help="cuboid of the FP64-GPU-path comparison (default the full workload, ~2 min)")
    ap.add_argument("--workload", default="cuboid",
                    choices=["cuboid", "metasurface", "batch", "gpm", "farfield", "ldos", "gmres", "nearfield",
                             "adjoint"],
                    help="cuboid: the headline assemble+solve line; metasurface: 64x64 ED/MD array, 32 wavelengths; "
                         "batch: 256 uneven blobs, each at its own wavelength; gpm: effective-model extraction; "
                         "farfield: far-field sigma_sca of the solved cuboid; ldos: electric LDOS around the sphere; "
                         "gmres: matrix-free preconditioned GMRES on a larger cuboid; nearfield: E and H map of the "
                         "solved cuboid; adjoint: the differentiation workload alone")
    ap.add_argument("--nearfield-side", type=int, default=320, help="nearfield workload: points per side of the map")
    ap.add_argument("--gmres-cuboid", default="80x60x10", help="gmres workload: cells per axis")
    ap.add_argument("--eps-env", type=float, default=1.0, help="metasurface workload: host permittivity")
    ap.add_argument("--streams", type=int, default=0, help="batch workload: concurrent streams (0 = default)")
    ap.add_argument("--no-autotune", action="store_true", help="batch workload: keep the default LU block width")
    ap.add_argument("--batch-structs", type=int, default=256,
                    help="batch workload: structures in the batch (256 = the workload; fewer for profiler captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint leg and the FP64 comparison (profiling runs)")
    args = ap.parse_args()
    global ERR_EST
    ERR_EST = args.stop == "estimate"
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import gdm_workloads as W
    import paper_2505_09545_gb300 as G

    if args.workload == "metasurface":
        return run_metasurface(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "gpm":
        return run_gpm(args)
    if args.workload == "farfield":
        return run_farfield(args)
    if args.workload == "ldos":
        return run_ldos(args)
    if args.workload == "gmres":
        return run_gmres(args)
    if args.workload == "nearfield":
        return run_nearfield(args)
    if args.workload == "adjoint":
        return run_adjoint(args)

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cpu_base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu_base = cpu_baseline_leg()  # before any GPU work of this process

    nx, ny, nz = (int(v) for v in args.cuboid.split("x"))
    s = W.cuboid_precision(nx, ny, nz)
    lam = float(s.wavelengths[0])
    ctx = G.Context(local)
    pos = torch.tensor(s.pos, device=dev)
    eps = torch.tensor(s.eps, device=dev)
    prob = G.GDMProblem(pos, lam, 3, eps=eps, step=s.step)
    ns = prob.size
    A = torch.empty((ns, G.padded_lda(ns)), dtype=torch.complex128 if args.precision == "fp64" else torch.complex64,
                    device=dev)
    ipiv = torch.empty(ns, dtype=torch.int32, device=dev)
    F0 = G.incident_planewave(ctx, pos, lam, s.e0)
    F = torch.empty_like(F0)

    def step():
        G.assemble(ctx, prob, args.precision, out=A)
        return G.solve(ctx, prob, A, F0, args.precision, ipiv=ipiv, F=F, tol=args.tol, err_estimate=ERR_EST)[2]

    for _ in range(max(3, args.warmup)):
        info = step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(local)
    barrier()
    clk.start()
    ctx.profile(True)
    l0 = ctx.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    infos = []
    for _ in range(args.steps):
        infos.append(step())
    e1.record()
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ctx.launches - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws, dev)

    # error of the timed fields: against a solve refined to 1e-12 with the same factors (A and ipiv hold
    # the last timed step's factorisation)
    F_ref = torch.empty_like(F)
    G.solve(ctx, prob, A, F0, args.precision, ipiv=ipiv, F=F_ref, factored=True, tol=1e-12)
    field_err = float(((F - F_ref).norm(dim=1) / F_ref.norm(dim=1)).max())
    # and against the oracle's dense FP64 solution of the same system, where it is stored
    golden = golden_fields() if args.cuboid == "40x30x10" else None
    oracle_err = None
    if golden is not None:
        Fh = F.cpu().numpy().T
        oracle_err = float(np.max(np.linalg.norm(Fh - golden, axis=0) / np.linalg.norm(golden, axis=0)))

    # one extra (untimed) step with per-phase device-time accounting
    ctx.phases(True)
    step()
    phases = {k: round(v, 2) for k, v in ctx.phases(False).items()}

    # end to end through the public API: host inputs -> device, solve, fields back to the host
    h_pos = torch.tensor(s.pos).pin_memory()
    h_eps = torch.tensor(s.eps).pin_memory()
    h_F = torch.empty(F.shape, dtype=F.dtype).pin_memory()
    d_pos = torch.empty_like(pos)
    d_eps = torch.empty_like(eps)

    def e2e_step():
        d_pos.copy_(h_pos, non_blocking=True)
        d_eps.copy_(h_eps, non_blocking=True)
        pr2 = G.GDMProblem(d_pos, lam, 3, eps=d_eps, step=s.step)
        f0 = G.incident_planewave(ctx, d_pos, lam, s.e0)
        G.assemble(ctx, pr2, args.precision, out=A)
        G.solve(ctx, pr2, A, f0, args.precision, ipiv=ipiv, F=F, tol=args.tol, err_estimate=ERR_EST)
        h_F.copy_(F, non_blocking=True)

    e2e_step()
    barrier()
    k_e2e = max(1, min(3, args.steps))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / k_e2e, ws, dev)

    # assembly kernel alone against HBM: (3N)^2 complex entries written once
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    G.assemble(ctx, prob, args.precision, out=A)
    torch.cuda.synchronize()
    ea.record()
    for _ in range(5):
        G.assemble(ctx, prob, args.precision, out=A)
    eb.record()
    torch.cuda.synchronize()
    asm_ms = ea.elapsed_time(eb) / 5
    asm_bytes = float(ns) * ns * A.element_size()

    extras = {}
    if not args.no_extras:
        extras["adjoint"] = adjoint_leg(G, ctx, dev, args.precision, args.warmup, args.steps)
        extras["nearfield"] = nearfield_leg(G, ctx, dev, prob, F)
        if args.precision == "tf32" and args.cuboid == "40x30x10":
            extras["bf16_refine"] = precision_leg(G, ctx, dev, "bf16", args.tol, golden)
        extras["metasurface"] = metasurface_leg(G, ctx, dev, args.precision, args.tol, 1.0, 1, 1, load_peaks()[0])
        extras["metasurface"].pop("sigma")
        extras["fp64_gpu_path"] = fp64_compare(G, ctx, dev, args.precision, args.fp64_cuboid, args.tol, golden)
        if ws == 1:
            import gdm_workloads as W
            ss_b = W.blob_batch()
            bl = batch_leg(G, ctx, dev, ss_b, args.precision, args.tol, 0, True, 2, 3)
            extras["batch"] = {"workload": BATCH_WORKLOAD.format(n=len(ss_b), sum_n=sum(s.n for s in ss_b)),
                               "batch_s": bl["ms"] / 1e3, "s_per_solve": bl["ms"] / 1e3 / len(ss_b),
                               "lu_tflops_effective": sum(8.0 / 3.0 * (3.0 * s.n) ** 3 for s in ss_b) /
                               (bl["ms"] / 1e3) / 1e12,
                               "grouped_factor_ms": bl["factor_ms"], "grouped_lu_block": bl["grouped_lu_block"],
                               "roofline_sum": bl["roofline_sum"], "accuracy": bl["accuracy"],
                               "gpu_launches_per_step": bl["launches"] / 3}

    peaks, peak_src = load_peaks()
    per_launch_ms = prof["ms"] / max(1, prof["launches"])
    flops_per_launch = prof["flops"] / max(1, prof["launches"])
    if args.precision == "fp64":
        rl = {"bound": "alu", "peak": 1.05, "peak_src": "FP64 rate measured with torch float64 matmul on GB300"}
    elif args.precision == "bf16":
        rl = {"bound": "tensor", "peak": peaks["bf16_tflops_sustained"],
              "peak_src": f"{peak_src} sustained bf16 (cuBLAS)"}
    elif os.environ.get("GDM_TC_DISABLE") or prof.get("tc", True) is False:
        rl = {"bound": "alu", "peak": FP32_SIMT_PEAK_TFLOPS, "peak_src": "FP32 SIMT: 152 SMs x 128 lanes x 2 x 2.07 GHz"}
    else:
        rl = {"bound": "tensor", "peak": peaks["bf16_tflops_sustained"] * NOMINAL_TF32_OVER_BF16,
              "peak_src": f"{peak_src} sustained bf16 x nominal TF32/BF16 ratio 1.1/2.25"}
    achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12 if per_launch_ms > 0 else 0.0
    traffic = traffic_record("lu_tc.cu", prof["bytes"] / max(1, prof["launches"])) if (
        rl["bound"] == "tensor" and args.precision == "tf32" and args.cuboid == "40x30x10") else None
    roofline = {"bound": rl["bound"], "achieved": achieved, "peak": rl["peak"], "unit": "TFLOP/s",
                "frac": achieved / rl["peak"], "traffic": traffic, "kernel": "LU trailing update A22 -= A21 U12",
                "algorithmic_bytes_per_launch": prof["bytes"] / max(1, prof["launches"]),
                "flops_per_launch": flops_per_launch,
                "launches_per_step": prof["launches"] / args.steps, "ms_per_step_in_kernel": prof["ms"] / args.steps,
                "peak_source": rl["peak_src"]}
    assembly = {"bound": "hbm", "achieved": asm_bytes / (asm_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": asm_bytes / (asm_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "ms": asm_ms,
                "bytes": asm_bytes, "peak_source": f"{peak_src} copy bandwidth",
                "kernel": "assemble A = I - G alpha (one launch, every entry written once)"}
    units = ws * 1
    value = per_unit_seconds(ms, ws)
    it = infos[-1]
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": {"tf32": "c64-tf32+f64", "fp32": "c64-3xtf32+f64",
                                           "bf16": "c64-bf16+f64"}.get(args.precision, "f64"),
            "data": "synthetic", "config": workload_config(args),
            "accuracy": {"tol": args.tol, "field_err_vs_oracle": oracle_err,
                         "field_err_vs_solve_to_1e-12": field_err,
                         "refine_iters": it["iterations"], "rel_correction": it["rel_correction"],
                         "rel_residual_fp64": it["rel_residual"], "factor_ms": it["factor_ms"],
                         "refine_ms": it["refine_ms"]},
            "roofline": roofline, "assembly_roofline": assembly, **extras,
            "gpu_launches": launches, "phases_ms": phases,
            "e2e": {"value": e2e_s / units, "unit": "s", "h2d_bytes_per_step": int(h_pos.numel() * 8 + h_eps.numel() * 16),
                    "d2h_bytes_per_step": int(h_F.numel() * 16)},
            "clocks": clocks, "cpu_baseline": cpu_base}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
