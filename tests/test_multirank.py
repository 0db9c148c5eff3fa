"""The N > 1 path on the CPU: two `gloo` ranks.

Under torchrun every rank steps its own full replica of the workload and the
ranks exchange nothing on the data path; they meet only to time the job (a
barrier on both sides and the maximum of the ranks' durations).  These tests
run that timing reduction, the whole-job rate, the independence of the seeded
replicas, and the reference arm under `torch.distributed.run` with two ranks,
all on the CPU.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=WORLD)


def _timing_worker(rank, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, port)
    try:
        # rank r "took" 1.5 + r seconds; every rank must see the slowest
        tdist.barrier()
        t = bench.max_over_ranks(torch, tdist, 1.5 + rank, "cpu")
        rate = bench.whole_job_rate(WORLD, 1000.0, t)
        tdist.barrier()
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"t": t, "rate": rate}, f)
    finally:
        tdist.destroy_process_group()


def _replica_worker(rank, port, out_dir):
    """Each rank builds the seeded 2-D bubble and takes one oracle RHS on its
    own copy; the ranks then compare checksums (the only exchange)."""
    sys.path.insert(0, ROOT)
    from oracle import dg, initial
    from oracle.mesh import Mesh
    from paper_2305_13847_gb300 import inputs
    _init(rank, port)
    try:
        w = inputs.workload("adjoint2d_q4", n=(8, 4), order=2)
        mesh = Mesh(w["dim"], w["n"], w["L"], w["order"], w["periodic"])
        node, face, _ = initial.base_tables(mesh, H=w["H"])
        prob = dg.Problem(mesh, node, face, rain=w["rain"])
        noise = inputs.node_noise(w, mesh.Ne, mesh.Np)
        U = initial.bubble_state(prob, w["A"], w["centre"], w["radius"], noise=noise, H=w["H"])
        R = dg.rhs(prob, U)
        mine = torch.tensor([float(np.sum(np.abs(R))), float(np.sum(R * np.arange(R.size).reshape(R.shape)))],
                            dtype=torch.float64)
        got = [torch.zeros_like(mine) for _ in range(WORLD)]
        tdist.all_gather(got, mine)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"sums": [g.tolist() for g in got]}, f)
    finally:
        tdist.destroy_process_group()


def _spawn(fn, tmp_path):
    port = _free_port()
    tmp.spawn(fn, args=(port, str(tmp_path)), nprocs=WORLD, join=True)
    return [json.load(open(os.path.join(tmp_path, "rank%d.json" % r))) for r in range(WORLD)]


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    res = _spawn(_timing_worker, tmp_path)
    for r in res:
        assert r["t"] == 2.5                    # the slower rank's duration, on both ranks
        assert r["rate"] == pytest.approx(WORLD * 1000.0 / 2.5)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 0.75, "cpu") == 0.75
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0


def test_replicas_are_identical_and_independent(tmp_path):
    res = _spawn(_replica_worker, tmp_path)
    sums = res[0]["sums"]
    assert res[1]["sums"] == sums
    assert sums[0] == sums[1]                  # bitwise: same seeded input, same arithmetic
    assert sums[0][0] > 0.0


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(WORLD),
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(WORLD),
           "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1                      # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == WORLD and d["value"] > 0
