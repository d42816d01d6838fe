"""Stored oracle solution of the 40 x 30 x 10 cell cuboid (N = 12,000, 3N = 36,000): test infrastructure.

Writes tests/golden/cuboid40x30x10_oracle.npz (the oracle's fields F, 36,000 x 2 complex128, and its
cross sections) and tests/golden/cuboid40x30x10_oracle.json (the same cross sections, the oracle's own
relative residual and the wall time of each phase with the host it ran on). Only the oracle and the
seeded input generators are called: the system is built by `Problem.matrix_blocks` a band of rows at a
time (the full-size temporaries of `Problem.matrix` would need about 150 GB of host memory; the entries
are the same) and solved by LAPACK zgesv through numpy, as `Problem.solve` does (Sec. "Numerical
solution": A F = F0 of Eq. GDM_system_of_equations).

    python oracle/make_golden_cuboid.py                      # write the golden files (~45 GB of RAM)
    python oracle/make_golden_cuboid.py --check OUT.json     # re-run, compare with the stored fields,
                                                             # write only a timing record
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gdm_workloads as W  # noqa: E402
import oracle as O  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")
STEM = "cuboid40x30x10_oracle"


def build_matrix(prob, rows_per_band=400):
    """Dense dipole-interleaved system (row 3i + a, column 3j + b) from the oracle's 3x3 blocks
    A_ij = delta_ij I - G_ij alpha_j, one band of target cells at a time."""
    n, k = prob.n, prob.kind
    A = np.empty((k * n, k * n), np.complex128)
    for r0 in range(0, n, rows_per_band):
        rows = np.arange(r0, min(n, r0 + rows_per_band))
        blk = prob.matrix_blocks(rows)                       # (band, n, k, k)
        A[k * r0:k * (r0 + len(rows))] = blk.transpose(0, 2, 1, 3).reshape(k * len(rows), k * n)
    return A


def solve_cuboid():
    s = W.cuboid_precision(40, 30, 10)
    prob = O.Problem(s.pos, float(s.wavelengths[0]), 3, eps=s.eps, step=s.step)
    t0 = time.perf_counter()
    A = build_matrix(prob)
    F0 = prob.plane_wave(s.e0)
    t1 = time.perf_counter()
    F = np.linalg.solve(A, F0)
    t2 = time.perf_counter()
    rel_res = np.linalg.norm(F0 - A @ F, axis=0) / np.linalg.norm(F0, axis=0)
    del A
    ext, sca, ab = prob.cross_sections(F0, F, s.e0)
    host = {"machine": platform.machine(), "cores": len(os.sched_getaffinity(0)),
            "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS", "default (all cores)")}
    rec = {"workload": "cuboid 40x30x10 cells, d=10 nm, N=12000 (3N=36000), eps~U[2,16]+iU[0,0.5] seed 2, "
                       "lambda=500 nm, x- and y-polarised plane waves along +z",
           "n": int(prob.n), "sigma_ext": ext.tolist(), "sigma_sca": sca.tolist(), "sigma_abs": ab.tolist(),
           "rel_residual": rel_res.tolist(),
           "assembly_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "host": host}
    return F, rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", metavar="OUT_JSON", help="compare with the stored fields; write a timing record")
    args = ap.parse_args()
    F, rec = solve_cuboid()
    if args.check:
        ref = np.load(os.path.join(GOLDEN, STEM + ".npz"))["F"]
        rec["rel_diff_vs_stored"] = (np.linalg.norm(F - ref, axis=0) / np.linalg.norm(ref, axis=0)).tolist()
        os.makedirs(os.path.dirname(os.path.abspath(args.check)), exist_ok=True)
        with open(args.check, "w") as f:
            json.dump(rec, f, indent=1)
    else:
        os.makedirs(GOLDEN, exist_ok=True)
        np.savez_compressed(os.path.join(GOLDEN, STEM + ".npz"), F=F,
                            sigma=np.array([rec["sigma_ext"], rec["sigma_sca"], rec["sigma_abs"]]))
        with open(os.path.join(GOLDEN, STEM + ".json"), "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
