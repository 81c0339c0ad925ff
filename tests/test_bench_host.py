"""Host-side logic of bench.py across ranks, on CPU with two gloo ranks: the job time is
the slowest rank's, the value counts every rank's sites (weak scaling), and the
reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    v = bench.whole_job_mlups(1000, 10, world, t)
    out.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(1000 * 10 * 2 / 15.0 / 1e6)


def test_reference_arm_rank_gating():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
                        "--workload", "droplet2d"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
                        "--workload", "droplet2d"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_recorded_traffic_follows_the_kernel_code(tmp_path, monkeypatch):
    """The DRAM traffic recorded from an ncu capture is reported only while the code of the
    kernel's translation unit and the headers it includes is unchanged: comments and
    whitespace do not count, any code change does, and files the unit does not include do
    not either."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_2003_11069_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text('#include "h.cuh"\n// a kernel\n__global__ void k(int* a) { a[0] = 1; }\n')
    (csrc / "h.cuh").write_text("#pragma once\n/* helper */ inline int two() { return 2; }\n")
    (csrc / "other.cuh").write_text("inline int three() { return 3; }\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._unit_closure("k.cu") == ["h.cuh", "k.cu"]
    h0 = bench.kernel_source_hash("k.cu")
    (prof / "traffic.json").write_text(json.dumps({"w/fp32": {"kernel_unit": "k.cu", "kernel_sources": h0,
                                                                "dram_bytes_per_step": 123}}))
    assert bench.recorded_traffic("w", "fp32") == 123
    (csrc / "k.cu").write_text('#include "h.cuh"\n// the kernel, reworded\n__global__ void k(int* a)\n{ a[0] = 1; }\n')
    (csrc / "other.cuh").write_text("inline int three() { return 4; }\n")
    assert bench.kernel_source_hash("k.cu") == h0
    assert bench.recorded_traffic("w", "fp32") == 123
    (csrc / "h.cuh").write_text("#pragma once\n/* helper */ inline int two() { return 3; }\n")
    assert bench.kernel_source_hash("k.cu") != h0
    assert bench.recorded_traffic("w", "fp32") is None
    assert bench.recorded_traffic("w", "fp64") is None


def test_algorithmic_bytes_per_site():
    """B_alg per site update (one read and one write of the stored state), which the bench's
    roofline fractions divide by: two populations per direction in FP64/FP32 (2 Q values),
    FP16-dev deviations (Q half2 and a float2 of reference densities), and the D3Q27 total +
    recolouring form (26 totals in FP32 or FP16, two FP32 rest populations, a float4)."""
    import bench

    assert bench.alg_bytes_per_site(0, "fp32") == 2 * 2 * 9 * 4 == 144
    assert bench.alg_bytes_per_site(0, "fp16dev") == 2 * (9 * 4 + 8) == 88
    assert bench.alg_bytes_per_site(1, "fp64") == 2 * 2 * 27 * 8 == 864
    assert bench.alg_bytes_per_site(1, "fp32") == 432
    assert bench.alg_bytes_per_site(1, "fp16dev") == 232
    assert bench.alg_bytes_per_site(1, "fp32", 1) == 2 * (26 * 4 + 2 * 4 + 16) == 256
    assert bench.alg_bytes_per_site(1, "fp16dev", 1) == 2 * (26 * 2 + 2 * 4 + 16) == 152
