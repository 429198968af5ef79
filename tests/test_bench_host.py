"""Host logic of bench.py that needs no GPU: the replica workloads of the
ranks, the max-over-ranks timing on a world-size-2 gloo process group, the
reference arm (one full oracle step per timed step) with its JSON line on
rank 0 and no output on the other ranks, and the oracle leg with its error
summary against given results."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_replica_workloads_are_seeded_by_rank():
    a = bench.workload("channels64", 0).coefficient()
    b = bench.workload("channels64", 1).coefficient()
    assert a.shape == b.shape and not np.array_equal(a, b)
    assert np.array_equal(a, bench.workload("channels64", 0).coefficient())


def test_max_over_ranks_without_process_group():
    assert bench.max_over_ranks(3.25) == 3.25


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(1.5 + rank, dist)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, "r%d" % rank), "w") as f:
        f.write(repr(v))


def test_max_over_ranks_gloo_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert [float(open(tmp_path / ("r%d" % r)).read()) for r in range(2)] == [2.5, 2.5]


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--workload", "channels64"],
                          capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_json_line_on_rank_0():
    p = _run_reference(0, 1)
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0
    # same config object as the GPU arm's
    w = bench.workload("channels64", 0)
    assert d["config"] == bench.workload_config(w, 4160, 1)
    assert d["step_seconds"][0] <= d["value"] * 1.0001


def test_reference_arm_other_ranks_exit_silently():
    p = _run_reference(1, 2)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


class _FakeHierarchy:
    def __init__(self, fail_gmres):
        self.fail_gmres = fail_gmres
        self.calls = {"solve": 0, "solve_gmres": 0}

    def solve(self, b, tol=1e-8, allow_maxit=False):
        self.calls["solve"] += 1
        return None, 66, 9e-9

    def solve_gmres(self, b, tol=1e-8, allow_maxit=False):
        self.calls["solve_gmres"] += 1
        if self.fail_gmres:
            raise RuntimeError("no convergence")
        return None, 35, 8e-7


def test_solver_leg_times_both_solvers_and_records_failures():
    H = _FakeHierarchy(fail_gmres=False)
    syncs = []
    out = bench.solver_leg(H, None, steps=3, warmup=2, sync=lambda: syncs.append(1))
    assert H.calls == {"solve": 5, "solve_gmres": 5} and len(syncs) == 12
    assert out["pcg_additive"]["iterations"] == 66 and out["gmres_hybrid"]["iterations"] == 35
    assert out["gmres_hybrid"]["rel_residual"] == 8e-7 and out["pcg_additive"]["ms"] >= 0.0
    out = bench.solver_leg(_FakeHierarchy(fail_gmres=True), None, steps=1, warmup=0, sync=lambda: None)
    assert "error" in out["gmres_hybrid"] and out["pcg_additive"]["iterations"] == 66


def test_oracle_leg_error_summary(tmp_path):
    """The oracle leg on the 64 x 64 workload, given the dense oracle's results
    in the place of the GPU's: eigenvalue errors at the subspace iteration's
    accuracy, equal counts, dimensions and iterations; a planted count
    difference is reported."""
    from oracle import fem, method
    w = bench.workload("channels64", 0)
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    H = method.Hierarchy(mesh, w.coefficient(), w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta)
    b = fem.load_vector(mesh)
    x, it, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-8)
    subs = H.levels[H.L].subs
    lam = np.full((len(subs), 32), np.nan)
    for i, s in enumerate(subs):
        k = min(32, len(s["lam"]))
        lam[i, :k] = s["lam"][:k]
    ms = np.array([s["m"] for s in subs])
    ms[3] += 1                                            # planted difference
    dims = [H.coarse_dims()[0], H.n]
    path = tmp_path / "gpu.npz"
    np.savez(path, level_dim=np.array(dims), iterations=np.array(it), x=x, fine_lam=lam, fine_m=ms)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-leg", str(path),
                        "--workload", "channels64"], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    d = json.loads(p.stdout.strip().splitlines()[-1])
    assert d["seconds"] > 0 and d["cores"] >= 1 and d["iterations"] == it
    e = d["error_vs_oracle"]
    assert e["fine"]["max_rel_eig_err"] < 1e-8
    assert e["fine"]["count_mismatch"] == [[3, int(ms[3]), int(ms[3]) - 1]]
    assert e["coarse_dims"]["gpu"] == e["coarse_dims"]["oracle"]
    assert e["iterations"]["gpu"] == e["iterations"]["oracle"]
    assert e["solution_gpu"]["rel_err_A"] < 1e-6 and e["solution_oracle"]["rel_err_A"] < 1e-6


def test_measured_traffic_holds_only_for_its_workload_and_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from the committed capture only for the
    workload and the kernel source it was taken from."""
    import hashlib
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment = ignored\nfamily=fine_gevp_solve\nkernel=k\nworkload=w512\nsource=kernel.cu\n"
        "source_sha256=%s\ndram_bytes_per_launch=1000\nalgorithmic_bytes_captured_launch=1200\n" % digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.measured_traffic("fine_gevp_solve", "w512")
    assert got["traffic"] == 1000.0 and got["traffic_launch_algorithmic_bytes"] == 1200.0
    assert bench.measured_traffic("fine_gevp_solve", "other_workload") == {}
    assert bench.measured_traffic("fine_gevp_apply", "w512") == {}
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("fine_gevp_solve", "w512")["traffic"] is None
