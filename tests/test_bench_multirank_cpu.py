"""The multi-rank path of bench.py on the host with the gloo backend, world size 2: the
whole-job figures take the slowest rank's time and the DOF-updates of all ranks, the
reference arm launched by torchrun prints one line from rank 0 while the other rank exits 0,
and the one-GPU batch workload refuses a multi-rank launch."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 10 (r + 1) ms over 1000 (r + 1) DOF-updates
    ms, dof = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
    with open(out_path + ".%d" % rank, "w") as f:
        json.dump([ms, dof], f)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "red")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        with open(out + ".%d" % r) as f:
            ms, dof = json.load(f)
        assert ms == 20.0 and dof == 3000.0


def test_reference_arm_under_torchrun_world2():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0


def test_batch_workload_refuses_multirank():
    env = dict(os.environ, WORLD_SIZE="2", RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "batch64"],
                       capture_output=True, text=True, cwd=ROOT, env=env, timeout=300)
    assert r.returncode != 0
    assert "one GPU" in r.stderr
    assert not any(ln.strip().startswith("{") for ln in r.stdout.splitlines())
