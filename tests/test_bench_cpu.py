"""bench.py on the host: the reference arm (the FP64 oracle on the host cores) prints one JSON
line with the keys of the bench contract, and the GPU arm fails loudly without a GPU instead
of falling back to the host."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                          text=True, cwd=ROOT, env=env, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference"
    assert out["metric"] == "DOF-updates/s" and out["unit"] == "DOF-updates/s"
    assert out["value"] > 0 and out["ms_per_step"] > 0 and out["higher_is_better"] is True
    assert out["warmup"] >= 3 and out["steps"] == 1 and out["n_gpus"] == 1
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["workload"].startswith("slab3d_q2_128x48x20")


def test_gpu_arm_fails_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU arm runs")
    r = _run("--steps", "1", "--warmup", "3", "--no-cpu-baseline", timeout=300)
    assert r.returncode != 0
    assert not any(ln.strip().startswith("{") for ln in r.stdout.splitlines())


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_lat_difference_is_zero_for_an_affine_activation_field(dim, order):
    """The serving accuracy measure interpolates the plain run's activation times (Gauss-Legendre
    nodes of its uniform fine grid) to the adaptive run's probes: an affine field is
    reproduced exactly, probes where a neighbouring plain probe never activated are left out,
    and a shift of the adaptive times by c shows up as a difference of c."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import workloads as W
    prob = W.Problem(dim=dim, order=order, extent=(0.5, 0.3, 0.2), base=(5, 3, 2), max_refine=2)
    plain = bench.plain_version(prob)
    g = np.array([3.0, -2.0, 1.5][:dim])
    lat_p = bench.probe_points(plain) @ g + 7.0
    pts = bench.probe_points(prob)
    assert pts.shape == (int(np.prod(prob.base[:dim])) * (order + 1) ** dim, dim)
    lat_a = pts @ g + 7.0
    d = bench.lat_difference(prob, lat_a, plain, lat_p)
    assert d["probes"] == len(lat_a) and d["max_ms"] < 1e-12
    d = bench.lat_difference(prob, lat_a + 0.25, plain, lat_p)
    assert abs(d["mean_ms"] - 0.25) < 1e-12 and abs(d["max_ms"] - 0.25) < 1e-12
    # the plain run never activated beyond a plane: adaptive probes next to it are not compared
    lat_p2 = np.where(bench.probe_points(plain)[:, 0] < 0.25, lat_p, np.inf)
    d = bench.lat_difference(prob, lat_a, plain, lat_p2)
    assert 0 < d["probes"] < len(lat_a) and d["max_ms"] < 1e-12 and d["adaptive_only"] > 0
