"""The N > 1 paths on CPU. Replicas (bench.py): two gloo ranks agree on the slowest rank's time, the whole-job
per-unit value follows from it, and the reference arm does no work on ranks other than 0. Partition
(paper_2505_09545_gb300.shard): two gloo ranks each take half of a spectrum's wavelengths and the joined loss,
shared gradients and per-wavelength gradients equal the single-rank result."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws, torch.device("cpu"))
    out[rank] = (t, bench.per_unit_seconds(t, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == pytest.approx(15.0 / 1e3 / 2)


def test_reference_arm_skips_other_ranks(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, cuboid="40x30x10", precision="tf32")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    """The reference arm at N = 1 (rank 0) prints one JSON line with the contract's keys: the oracle timed on
    the host cores, its own e2e with no host-device traffic, the same config as the GPU arm."""
    import argparse
    import json
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda *a, **k: {
        "value": 1.5, "unit": "s", "cores": 4, "kind": "oracle", "sample": "stub sample"})
    args = argparse.Namespace(gpus=1, steps=2, warmup=1, cuboid="40x30x10", precision="tf32", tol=1e-10)
    bench.run_reference(args)
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["higher_is_better"] is False
    assert line["value"] == 1.5 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 4
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"] == bench.workload_config(args)


def test_unit_range_partitions_contiguously():
    from paper_2505_09545_gb300.shard import unit_range
    for n in (0, 1, 7, 8, 32, 256):
        for ws in (1, 2, 3, 4, 8):
            ranges = [unit_range(n, ws, r) for r in range(ws)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        unit_range(4, 2, 2)



def test_weighted_unit_range_balances_uneven_structures():
    """The 256-blob batch's LU work (3N)^3 split over 2, 4 and 8 ranks: contiguous, complete, and every rank's
    share within one largest item of the mean."""
    import gdm_workloads as W
    from paper_2505_09545_gb300.shard import weighted_unit_range
    w = [(3.0 * s.n) ** 3 for s in W.blob_batch()]
    for ws in (1, 2, 4, 8):
        ranges = [weighted_unit_range(w, ws, r) for r in range(ws)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(w)
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        share = [sum(w[lo:hi]) for lo, hi in ranges]
        assert max(abs(x - sum(w) / ws) for x in share) <= max(w)

def _spectrum_unit_fn(lo, hi):
    """Oracle loss |E(probe)|^2 + sigma_sca and its gradients for the wavelengths [lo, hi) of a small cylinder
    (the units a rank owns)."""
    import numpy as np
    import gdm_workloads as W
    import oracle as O
    cyl = W.cylinder_diff(radius=20.0, height=20.0, step=10.0, n_lambda=5)
    L, gp, ge = 0.0, np.zeros((cyl.n, 3)), np.zeros(cyl.n, np.complex128)
    gl = []
    for lam in cyl.wavelengths[lo:hi]:
        pr = O.Problem(cyl.pos, float(lam), 3, eps=cyl.eps, step=cyl.step)
        Lo, gpo, geo, glo = O.loss_and_grad_probe_sca(pr, cyl.e0, cyl.r_eval[0])
        L, gp, ge = L + Lo, gp + gpo, ge + geo
        gl.append(glo)
    return (torch.tensor(L, dtype=torch.float64), torch.tensor(gp), torch.tensor(ge),
            torch.tensor(np.array(gl, np.float64).reshape(-1)))


def _spectrum_rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2505_09545_gb300.shard import spectrum_loss_and_grads
    L, gp, ge, gl = spectrum_loss_and_grads(_spectrum_unit_fn, 5)
    out[rank] = (float(L), gp.numpy(), ge.numpy(), gl.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_a_spectrum():
    import numpy as np
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_spectrum_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    L1, gp1, ge1, gl1 = _spectrum_unit_fn(0, 5)
    for r in range(ws):
        L, gp, ge, gl = res[r]
        assert L == pytest.approx(float(L1), rel=1e-13)
        np.testing.assert_allclose(gp, gp1.numpy(), rtol=1e-12, atol=1e-12 * np.abs(gp1.numpy()).max())
        np.testing.assert_allclose(ge, ge1.numpy(), rtol=1e-12, atol=1e-12 * np.abs(ge1.numpy()).max())
        np.testing.assert_allclose(gl, gl1.numpy(), rtol=1e-13)
