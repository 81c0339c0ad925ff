"""Benchmark of the fused NCI colour-gradient lattice Boltzmann step on GB300.

One "step" is one full lattice Boltzmann time step (stream, moments, gradient, NCI,
collide, recolour) over the whole lattice. Default workload: the 3D packed emulsion in
a square duct, D3Q27, 512 x 128 x 128 sites, walls in y and z, periodic in x, FCC-packed
droplets of radius 10, body force 2e-6, A_h = 0.03, FP16-deviation storage and FP32
arithmetic (--precision fp32: FP32 storage), with the same duct in FP32 storage timed
beside it (fp32_compare: the total + recolouring form and the two-population layout).
Metric: MLUPS (million lattice-site updates per second), whole job. The duct's state
(1.9 GB for the two FP16-dev buffers, 3.6 GB in FP32) is far larger than L2, so K steps
are timed back to back with CUDA events on the library's stream. Lattices that fit in L2 (the 2048 x 256 channel) are flushed
before every timed step (a 512 MB write, then a 256 MB read so that the write's dirty
lines go back to memory before, not during, the step) and each step is timed alone.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload duct3d|duct3d_small|channel2d|channel2d_large|droplet2d|ensemble|warmstart]
                  [--precision fp32|fp64|fp16dev]

--impl reference times the FP64 CPU oracle on the host cores (the deliberately slow
correctness reference, not a tuned CPU code). Under torchrun every rank runs its own
replica of the workload on its own GPU (the step does not shard here); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2003_11069_gb300 import inputs  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    # name: lattice, sizes, walls, physics, generator
    "channel2d": dict(lattice=0, nx=2048, ny=256, nz=1, wall_y=1, wall_z=0, tau=1.0, A_s=0.01, beta=0.7,
                      A_h=0.05, force=(1e-5, 0.0, 0.0),
                      gen=lambda nx, ny, nz, seed: inputs.channel_emulsion_2d(nx, ny, seed=seed),
                      desc="D2Q9 soft-flowing-crystal channel 2048x256, walls y, packed droplets R 12-16 "
                           "(hexagonal rows, +-1 jitter, film >= 1: area fraction 0.73 of the 0.8 requested), "
                           "G=1e-5, A_h=0.05"),
    "channel2d_large": dict(lattice=0, nx=8192, ny=1024, nz=1, wall_y=1, wall_z=0, tau=1.0, A_s=0.01, beta=0.7,
                            A_h=0.05, force=(1e-5, 0.0, 0.0),
                            gen=lambda nx, ny, nz, seed: inputs.channel_emulsion_2d(nx, ny, seed=seed),
                            desc="D2Q9 soft-flowing-crystal channel 8192x1024 (the 2048x256 channel's generator "
                                 "at 16x the sites, state 2.4 GB in FP32: larger than L2), walls y, packed "
                                 "droplets R 12-16, G=1e-5, A_h=0.05"),
    "duct3d": dict(lattice=1, nx=512, ny=128, nz=128, wall_y=1, wall_z=1, tau=1.0, A_s=0.01, beta=0.7,
                   A_h=0.03, force=(2e-6, 0.0, 0.0),
                   gen=lambda nx, ny, nz, seed: inputs.duct_emulsion_3d(nx, ny, nz, seed=seed),
                   desc="D3Q27 packed-emulsion square duct 512x128x128, walls y,z, FCC droplets R 10 "
                        "(film >= 1: volume fraction 0.54, the most R 10 spheres reach in this duct; 0.7 "
                        "requested), G=2e-6, A_h=0.03"),
    "ensemble": dict(lattice=0, nx=0, ny=0, nz=1, wall_y=1, wall_z=0, tau=1.0, A_s=0.01, beta=0.7,
                     A_h=0.05, force=(1e-5, 0.0, 0.0), members=96,
                     gen=lambda nx, ny, nz, seed: inputs.channel_emulsion_2d(nx, ny, seed=seed),
                     desc="96 independent D2Q9 channels, length 512-2048, width 64-256, area fraction "
                          "0.7-0.9 requested (packings reach about 0.73), G log-uniform 1e-6..1e-4, A_h "
                          "uniform 0..0.1, one batched launch per step (CUDA graph), autotuned L2 "
                          "promotion and static tiles of the batched kernel"),
    "duct3d_small": dict(lattice=1, nx=384, ny=96, nz=96, wall_y=1, wall_z=1, tau=1.0, A_s=0.01, beta=0.7,
                         A_h=0.03, force=(2e-6, 0.0, 0.0),
                         gen=lambda nx, ny, nz, seed: inputs.duct_emulsion_3d(nx, ny, nz, seed=seed),
                         desc="D3Q27 packed-emulsion square duct 384x96x96 (profiling size: 3 GB of FP32 "
                              "state), walls y,z, FCC droplets R 10, G=2e-6, A_h=0.03"),
    "duct3d_profile": dict(lattice=1, nx=512, ny=128, nz=48, wall_y=1, wall_z=1, tau=1.0, A_s=0.01, beta=0.7,
                           A_h=0.03, force=(2e-6, 0.0, 0.0),
                           gen=lambda nx, ny, nz, seed: inputs.duct_emulsion_3d(nx, ny, nz, seed=seed),
                           desc="D3Q27 packed-emulsion duct 512x128x48 (profiling size: the bench duct's 256 "
                                "columns of 32x8 sites, 1.4 GB of FP32 state), walls y,z, FCC droplets R 10, "
                                "G=2e-6, A_h=0.03"),
    "warmstart": dict(lattice=0, nx=0, ny=0, nz=1, wall_y=1, wall_z=0, tau=1.0, A_s=0.01, beta=0.7,
                      A_h=0.0, force=(0.0, 0.0, 0.0), gen=None,
                      desc="U-Net warm start: D2Q9 packed-emulsion channels, length 512-1024, width 64-96, "
                           "area fraction 0.7-0.9 target, A_h 0-0.01, Poiseuille velocity 2e-3..2e-2 "
                           "(log-uniform); network 4 levels, base 32, BF16, trained on LB snapshots "
                           "resampled to 64x256; held-out channels run cold, cold-perturbed and warm"),
    "droplet2d": dict(lattice=0, nx=128, ny=128, nz=1, wall_y=0, wall_z=0, tau=1.0, A_s=0.01, beta=0.7,
                      A_h=0.05, force=(0.0, 0.0, 0.0),
                      gen=lambda nx, ny, nz, seed: inputs.droplet(nx, ny, radius=30),
                      desc="D2Q9 periodic 128x128, one droplet R 30, A_h=0.05"),
}

# The kernels lb_step launches, by lb_step_path().
STEP_KERNELS = {0: "fused2d_kernel (one-pass D2Q9 step)",
                1: "tma2d_kernel (persistent TMA-fed D2Q9 step, one launch per step)",
                2: "moments_kernel + march3d_kernel (D3Q27 two-pass step, two launches)",
                3: "interface3d_kernel + nci3d_kernel + carry3d_kernel (D3Q27 single-read step: densities "
                   "carried by the previous collision, interface pass, NCI ray pass, TMA-fed collision; three "
                   "launches)",
                4: "moments_kernel + normals3d_kernel + collide3d_kernel (D3Q27 streaming step: psi, per-site "
                   "normals, then the NCI ray, pull, collision and store without shared memory; three launches)"}
STATE_FORMS = {0: "pairs: the populations of both components",
               1: "total + recolouring: the total populations f*_i of the 26 moving directions (FP32, or FP16 "
                  "deviations from w_i rho_0), the rest population of each component and (rho_1/rho, beta "
                  "rho_1 rho_2/rho m) per site: FP32 128 B (pairs 216 B), FP16-dev 76 B (pairs 116 B); the "
                  "moments pass is moments3_kernel<TotalRecol/TotalRecolHalf> and the collision collide3t_kernel"}


# Bytes of state moved per site update (1 read + 1 write): FP64/FP32 populations are
# 2 components x Q values; FP16-dev stores Q half2 deviations plus a float2 of
# reference densities per site; the total + recolouring form (state form 1, D3Q27) Q - 1
# total populations (FP32, or FP16 deviations), 2 FP32 rest populations and a float4 of
# coefficients.
def alg_bytes_per_site(lattice: int, precision: str, form: int = 0) -> int:
    Q = 9 if lattice == 0 else 27
    if form == 1:
        return 2 * ((Q - 1) * (2 if precision == "fp16dev" else 4) + 8 + 16)
    per_site = {"fp64": 2 * Q * 8, "fp32": 2 * Q * 4, "fp16dev": Q * 4 + 8}[precision]
    return 2 * per_site


L2_BYTES = 129 << 20


def state_bytes(lattice: int, precision: str, N: int) -> int:
    """Bytes of one population state (one of the two buffers)."""
    return alg_bytes_per_site(lattice, precision) // 2 * N


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def _unit_closure(unit: str) -> list:
    """A translation unit of the CUDA library and the local headers it includes,
    transitively (sorted names)."""
    import re
    d = os.path.join(ROOT, "paper_2003_11069_gb300", "csrc")
    seen, todo = set(), [unit]
    while todo:
        name = todo.pop()
        if name in seen or not os.path.exists(os.path.join(d, name)):
            continue
        seen.add(name)
        with open(os.path.join(d, name)) as fh:
            todo += re.findall(r'^\s*#include\s+"([^"]+)"', fh.read(), re.M)
    return sorted(seen)


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace collapsed (a change to a
    comment is not a change to the kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(unit: str = None) -> str:
    """Hash of the CUDA code (comments and whitespace ignored): of one translation unit
    and its headers (the sources a kernel is built from), or of every file when unit is
    None."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2003_11069_gb300", "csrc")
    for name in (_unit_closure(unit) if unit else sorted(os.listdir(d))):
        with open(os.path.join(d, name), encoding="utf-8") as fh:
            h.update(name.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current sources of the kernel's translation unit (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        ent = rec.get(f"{workload}/{precision}")
        if ent and ent.get("kernel_sources") == kernel_source_hash(ent.get("kernel_unit")):
            return ent.get("dram_bytes_per_step")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [v for v in sm if v > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_run(w: dict, budget_s: float, nthreads: int, crop=None):
    """Time the FP64 CPU oracle on (a crop of) the workload for about budget_s seconds."""
    import oracle
    nx, ny, nz = (crop or (w["nx"], w["ny"], w["nz"]))
    fl = w["gen"](nx, ny, nz, 1234)
    p = oracle.make_params(lattice=w["lattice"], nx=nx, ny=ny, nz=nz, wall_y=w["wall_y"], wall_z=w["wall_z"],
                           tau=w["tau"], A_s=w["A_s"], beta=w["beta"], A_h=w["A_h"], force=w["force"])
    f = oracle.init(p, fl.rho1, fl.rho2)
    steps, t0 = 0, time.perf_counter()
    chunk = 1
    while True:
        oracle.step_inplace(p, f, chunk, nthreads)
        steps += chunk
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
        chunk = max(1, min(chunk * 2, int(steps * (budget_s - el) / max(el, 1e-9)) or 1))
    el = time.perf_counter() - t0
    n = nx * ny * nz
    return {"mlups": n * steps / el / 1e6, "steps": steps, "seconds": el, "sites": n,
            "sample": f"{nx}x{ny}x{nz} crop of the same generator, {steps} steps, FP64 oracle"}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the slowest rank sets the whole job's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(sites_per_rank: int, steps: int, world_size: int, seconds: float) -> float:
    """Million site updates per second of all ranks together (weak scaling: every rank
    advances its own replica of the workload)."""
    return sites_per_rank * steps * world_size / seconds / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    if w is WORKLOADS["warmstart"]:
        cpu = unet_cpu_baseline()
        line = {"impl": "reference", "metric": "U-Net training throughput (FP64 oracle)", "value": cpu["value"],
                "unit": cpu["unit"], "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": {"workload": w["desc"], "sample": cpu["sample"]},
                "cpu_baseline": cpu,
                "e2e": {"value": cpu["value"], "unit": cpu["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import oracle
    if w["nx"] == 0:  # the ensemble: one 1024 x 128 member stands in for the sample
        w = dict(w, nx=1024, ny=128)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    sites = nx * ny * nz
    # each step: one full oracle step on a bounded sample of the workload
    budget_sites = 600_000 if w["lattice"] == 0 else 120_000
    if sites > budget_sites:
        if w["lattice"] == 0:
            crop = (nx, max(16, budget_sites // nx), 1)
        else:
            crop = (max(32, budget_sites // (ny * nz) // 32 * 32) if budget_sites // (ny * nz) >= 32 else 32,
                    min(ny, 48), min(nz, 48))
    else:
        crop = (nx, ny, nz)
    fl = w["gen"](*crop, 1234)
    p = oracle.make_params(lattice=w["lattice"], nx=crop[0], ny=crop[1], nz=crop[2], wall_y=w["wall_y"],
                           wall_z=w["wall_z"], tau=w["tau"], A_s=w["A_s"], beta=w["beta"], A_h=w["A_h"],
                           force=w["force"])
    f = oracle.init(p, fl.rho1, fl.rho2)
    for _ in range(args.warmup):
        oracle.step_inplace(p, f, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step_inplace(p, f, 1, cores)
    el = time.perf_counter() - t0
    n = crop[0] * crop[1] * crop[2]
    mlups = n * args.steps / el / 1e6
    sample = f"{crop[0]}x{crop[1]}x{crop[2]} sample of the workload per step"
    line = {
        "impl": "reference", "metric": "MLUPS", "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "sample": sample, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args, w, lbnci, torch, prec, ws, rank, local, dist):
    """The ensemble workload: every member advanced by one batched launch per step."""
    members = inputs.ensemble_channels(w["members"], seed=1234 + rank)
    stream = torch.cuda.Stream()
    cfgs = [lbnci.lb_config_make(nx=m.nx, ny=m.ny, wall_y=1, tau=w["tau"], A_s=w["A_s"], beta=w["beta"],
                                 A_h=m.A_h, force=(m.force, 0.0, 0.0), precision=prec,
                                 stream=stream.cuda_stream) for m in members]
    N = sum(m.nx * m.ny for m in members)
    ens = lbnci.Ensemble(cfgs)
    n_tma = sum(1 for mv in ens.members if mv.step_path() == lbnci.LB_PATH_TMA2D)
    for mv, m in zip(ens.members, members):
        mv.init_fields(m.fields.rho1, m.fields.rho2)
    spt = ens.tune()
    t32x16, t32x32 = ens.tune_times()
    tma_tune = None
    if n_tma:
        promo, nstatic, table = ens.tma_choice()
        tma_tune = {"l2_promotion_bytes": promo, "static_tiles_per_cta": nstatic,
                    "ms_per_step": {f"promo{k[0]}_static{k[1]}": round(v, 4) for k, v in table.items()}}
    ens.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = ens.launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        ens.step(args.steps)  # the state (2.9 GB in FP32) is far larger than L2
        end.record(stream)
        torch.cuda.synchronize()
    launches = ens.launches() - launches0
    total_ms = max_over_ranks(start.elapsed_time(end), dist, "cuda")
    obs = [mv.observables(allow_numeric=True) for mv in ens.members]
    study = flow_study(ens, members, args.study_steps, obs) if rank == 0 else None
    # the same lattices stepped one launch per member per step, for comparison
    seq_ms = None
    if not args.no_e2e:
        sims = [lbnci.Sim(c) for c in cfgs]  # on the same stream as the ensemble
        for sm, m in zip(sims, members):
            sm.init_fields(m.fields.rho1, m.fields.rho2)
        ks = max(3, args.steps // 4)
        for sm in sims:
            sm.step(2)
        torch.cuda.synchronize()
        s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s2.record(stream)
        for _ in range(ks):
            for sm in sims:
                sm.step(1)
        e2.record(stream)
        torch.cuda.synchronize()
        seq_ms = s2.elapsed_time(e2) / ks
        for sm in sims:
            sm.close()
    ens.close()
    kern = []
    if n_tma:
        kern.append(f"tma2d_kernel batched over {n_tma} members")
    if n_tma < len(members):
        kern.append(f"fused2d_batch_kernel over {len(members) - n_tma} members (tile 32x{8 * spt})")
    extra = {"step_kernels": "; ".join(kern), "one_launch_per_member_ms_per_step": seq_ms,
             "autotune": {"tma_kernel": tma_tune,
                          "one_pass_kernel": {"tile": f"32x{8 * spt}", "ms_per_step":
                                              {"32x16": round(t32x16, 4), "32x32": round(t32x32, 4)}}
                          if n_tma < len(members) else None}}
    return N, total_ms, launches, clk.summary(), obs, extra, study


def flow_study(ens, members, study_steps, obs):
    """The study an ensemble runs for (the flow rate of the dispersed phase against the
    body force G and the near-contact strength A_h, Results, Fig. 3): per member G, A_h,
    width, target area fraction and the flow rates, time-averaged over the second half of
    `study_steps` further steps (sampled every study_steps / 40), or the values after the
    timed steps when study_steps is 0 (null where a member's state went non-finite: with
    G up to 1e-4 in channels up to 256 wide the Poiseuille speed G W^2 / (8 nu) passes
    the lattice's low-Mach range, and with A_h near 0.1 the near-contact kicks grow
    without bound; "diverged" counts them); and the least-squares fit
    log Q_d = a + b log G + c A_h + d log ny over the members with finite Q_d > 0."""
    if study_steps > 0:
        ens.step(study_steps // 2)
        every = max(1, study_steps // 40)
        acc = np.zeros((len(members), 2))
        ns = 0
        for _ in range((study_steps - study_steps // 2) // every):
            ens.step(every)
            o = [mv.observables(allow_numeric=True) for mv in ens.members]
            acc += [[x["flow_rate"], x["flow_rate_disp"]] for x in o]
            ns += 1
        q = acc / max(ns, 1)
    else:
        q = np.array([[x["flow_rate"], x["flow_rate_disp"]] for x in obs])
    finite = np.isfinite(q).all(axis=1)
    rows = [[float(f"{m.force:.4g}"), round(m.A_h, 4), m.ny, round(m.fields.meta["target_area_fraction"], 3),
             float(f"{q[k, 0]:.5g}") if finite[k] else None, float(f"{q[k, 1]:.5g}") if finite[k] else None]
            for k, m in enumerate(members)]
    ok = finite & (q[:, 1] > 0)
    fit = None
    if ok.sum() >= 5:
        X = np.column_stack([np.ones(ok.sum()), np.log([m.force for m in members])[ok],
                             np.array([m.A_h for m in members])[ok], np.log([m.ny for m in members])[ok]])
        coef, *_ = np.linalg.lstsq(X, np.log(q[ok, 1]), rcond=None)
        fit = {"dlogQd_dlogG": round(float(coef[1]), 4), "dlogQd_dA_h": round(float(coef[2]), 4),
               "dlogQd_dlogny": round(float(coef[3]), 4), "members_fitted": int(ok.sum())}
    return {"steps_after_timing": study_steps,
            "average": "second half, 40 samples" if study_steps > 0 else "none (state after the timed steps)",
            "columns": ["G", "A_h", "ny", "area_fraction", "Q", "Q_disp"], "members": rows,
            "diverged": int((~finite).sum()), "fit": fit}


def time_other_storage(lbnci, torch, w, prec, rho1, rho2, steps, warmup, env):
    """ms per step of `steps` back-to-back steps of workload w in another storage (a fresh
    sim; `env` is set while it is created, which is when the library reads it)."""
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        stream = torch.cuda.Stream()
        cfg = lbnci.lb_config_make(lattice=w["lattice"], nx=w["nx"], ny=w["ny"], nz=w["nz"], wall_y=w["wall_y"],
                                   wall_z=w["wall_z"], tau=w["tau"], A_s=w["A_s"], beta=w["beta"], A_h=w["A_h"],
                                   force=w["force"], precision=prec, stream=stream.cuda_stream)
        sim = lbnci.Sim(cfg, workspace="torch")
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    form = sim.state_form()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        sim.init_fields(rho1, rho2)
        sim.step(warmup)
        stream.synchronize()
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sim.close()
    return ms, form


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="duct3d", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp16dev", choices=["fp32", "fp64", "fp16dev"])
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="duct with FP16-dev storage: skip timing the FP32 storages on the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ws-train", type=int, default=2048,
                    help="warmstart: training channels (2048: about 20k snapshots, 8 minutes on GB300)")
    ap.add_argument("--ws-test", type=int, default=64, help="warmstart: held-out channels")
    ap.add_argument("--ws-horizon", type=int, default=60000, help="warmstart: lattice steps per run")
    ap.add_argument("--study-steps", type=int, default=0,
                    help="ensemble: further steps after timing over which the flow rates are averaged")
    ap.add_argument("--flush-mb", type=int, default=L2_FLUSH_BYTES >> 20,
                    help="L2 flush buffer written before every timed step (MB)")
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    from paper_2003_11069_gb300 import lbnci

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lbnci.load()
    if args.workload == "ensemble":
        return main_ensemble(args, w, lbnci, torch, ws, rank, local, dist)
    if args.workload == "warmstart":
        return main_warmstart(args, w, torch, ws, rank, local, dist)
    stream = torch.cuda.Stream()
    prec = {"fp32": lbnci.LB_FP32, "fp64": lbnci.LB_FP64, "fp16dev": lbnci.LB_FP16DEV}[args.precision]
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    N = nx * ny * nz
    cfg = lbnci.lb_config_make(lattice=w["lattice"], nx=nx, ny=ny, nz=nz, wall_y=w["wall_y"], wall_z=w["wall_z"],
                               tau=w["tau"], A_s=w["A_s"], beta=w["beta"], A_h=w["A_h"], force=w["force"],
                               precision=prec, stream=stream.cuda_stream)
    fl = w["gen"](nx, ny, nz, 1234 + rank)
    rho1 = torch.from_numpy(fl.rho1).cuda()
    rho2 = torch.from_numpy(fl.rho2).cuda()
    flush = torch.empty(max(1, args.flush_mb if state_bytes(w["lattice"], args.precision, N) * 2 <= 4 * L2_BYTES
                            else 1) << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    sim = lbnci.Sim(cfg, workspace="torch")
    # a state larger than four times L2 (129 MB) is its own flush: steps run back to back
    big = state_bytes(w["lattice"], args.precision, N) * 2 > 4 * L2_BYTES
    flush_mb = 0 if big else args.flush_mb
    with torch.cuda.stream(stream):
        sim.init_fields(rho1, rho2)
        sim.step(args.warmup)
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = sim.launches()
        with ClockSampler(local) as clk:
            if big:
                starts[0].record(stream)
                sim.step(args.steps)
                ends[0].record(stream)
            else:
                for k in range(args.steps):
                    if flush_mb > 0:
                        flush.fill_(k & 0xFF)  # evict the lattice from L2 before each timed step
                        # then read half of it back: the write left L2 full of the flush's dirty
                        # lines, whose write-back would otherwise land in the timed step
                        flush[: flush.numel() // 2].max()
                    starts[k].record(stream)
                    sim.step(1)
                    ends[k].record(stream)
            torch.cuda.synchronize()
        launches = sim.launches() - launches0
        path = sim.step_path()
        form = sim.state_form()
        if big:
            step_ms = [starts[0].elapsed_time(ends[0])]
        else:
            step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        total_ms = max_over_ranks(float(sum(step_ms)), dist, "cuda")
        if dist:
            dist.barrier()
        obs = sim.observables(allow_numeric=True)
    clocks = clk.summary()
    ms_per_step = total_ms / args.steps
    value = whole_job_mlups(N, args.steps, ws, total_ms * 1e-3)

    # FP16-deviation storage against FP32 storage on the same duct: fresh sims, the same
    # generated fields, K steps back to back (rank 0's figures; every rank runs its own)
    fp32_compare = None
    if big and args.precision == "fp16dev" and w["lattice"] == 1 and not args.no_fp32_compare:
        fp32_compare = {}
        for name, env in (("fp32", {}), ("fp32_pairs", {"LBNCI_D3_STATE": "pairs"})):
            ms, form_v = time_other_storage(lbnci, torch, w, lbnci.LB_FP32, rho1, rho2, args.steps, args.warmup, env)
            b = alg_bytes_per_site(1, "fp32", form_v)
            b2 = alg_bytes_per_site(1, "fp32", 0)
            pk, _ = measured_hbm_peak()
            fp32_compare[name] = {"ms_per_step": round(ms, 5), "value": round(N / (ms * 1e-3) / 1e6, 2),
                                  "state_form": STATE_FORMS.get(form_v, "?").split(":")[0],
                                  "alg_bytes_per_site": b,
                                  "frac": round(b * N / (ms * 1e-3) / 1e9 / pk, 4),
                                  "frac_two_population": round(b2 * N / (ms * 1e-3) / 1e9 / pk, 4)}
            fp32_compare[f"speedup_vs_{name}"] = round(ms / ms_per_step, 3)
        fp32_compare["env"] = "fp32_pairs: LBNCI_D3_STATE=pairs"

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h1 = torch.from_numpy(fl.rho1).pin_memory()
        h2 = torch.from_numpy(fl.rho2).pin_memory()
        psi_h = torch.empty(N, dtype=torch.float64).pin_memory()
        u_h = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_fields(h1.numpy(), h2.numpy())
        sim.step(args.steps)
        o2 = sim.observables(psi_h.numpy(), u_h.numpy(), allow_numeric=True)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": round(whole_job_mlups(N, args.steps, ws, el), 3), "unit": "MLUPS",
               "h2d_bytes_per_step": round(2 * 8 * N / args.steps, 1),
               "d2h_bytes_per_step": round((4 * 8 * N + 80) / args.steps, 1),
               "note": "lb_init_fields from pinned host rho1/rho2, lb_step(K), lb_observables with psi "
                       "and u copied back to host; bytes per step = totals / K"}
    sim.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0

    peak, peak_kind = measured_hbm_peak()
    bpsite = alg_bytes_per_site(w["lattice"], args.precision, form)
    achieved = bpsite * N / (ms_per_step * 1e-3) / 1e9
    traffic = recorded_traffic(args.workload, args.precision)
    cpu = None
    if not args.no_cpu_baseline:
        crop = (512, 64, 1) if w["lattice"] == 0 else (64, 32, 32)
        if args.workload == "droplet2d":
            crop = None
        r = cpu_oracle_run(w, args.cpu_budget, os.cpu_count() or 1, crop)
        cpu = {"value": round(r["mlups"], 4), "unit": "MLUPS", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": r["sample"]}
    line = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16 storage / f32 compute"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w["desc"], "sites": N, "precision": args.precision,
                   "l2": (f"state {2 * state_bytes(w['lattice'], args.precision, N) / 1e9:.2f} GB (two buffers), "
                          f"larger than L2 (129 MB): not flushed, {args.steps} steps timed back to back" if big else
                          f"flushed before every timed step ({flush_mb} MB write, then a "
                          f"{flush_mb // 2} MB read so the flush's dirty lines are written back "
                          f"before the step); each step timed alone" if flush_mb > 0 else "not flushed"),
                   "step_kernel": STEP_KERNELS.get(path, "?"),
                   "state_form": STATE_FORMS.get(form, "?"),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "droplets": fl.meta.get("droplets"),
                   "fraction": fl.meta.get("area_fraction", fl.meta.get("volume_fraction"))},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "kernel": STEP_KERNELS.get(path, "?"), "alg_bytes_per_site": bpsite},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "observables": {"n_nci": obs["n_nci"], "n_interface": obs["n_interface"], "n_bad": obs["n_bad"]},
    }
    if form == 1:  # the fraction at the two-population storage's bytes, for comparison
        b2 = alg_bytes_per_site(w["lattice"], args.precision, 0)
        line["roofline"]["two_population_equivalent"] = {
            "alg_bytes_per_site": b2, "frac": round(b2 * N / (ms_per_step * 1e-3) / 1e9 / peak, 4)}
    if fp32_compare is not None:
        line["fp32_compare"] = fp32_compare
    print(json.dumps(line), flush=True)
    return 0


def main_ensemble(args, w, lbnci, torch, ws, rank, local, dist):
    prec = {"fp32": lbnci.LB_FP32, "fp64": lbnci.LB_FP64, "fp16dev": lbnci.LB_FP16DEV}[args.precision]
    N, total_ms, launches, clocks, obs, extra, study = run_ensemble(args, w, lbnci, torch, prec, ws, rank, local,
                                                                    dist)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    ms_per_step = total_ms / args.steps
    value = whole_job_mlups(N, args.steps, ws, total_ms * 1e-3)
    peak, peak_kind = measured_hbm_peak()
    bpsite = alg_bytes_per_site(0, args.precision)
    achieved = bpsite * N / (ms_per_step * 1e-3) / 1e9
    seq = extra["one_launch_per_member_ms_per_step"]
    line = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16 storage / f32 compute"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w["desc"], "sites": N, "members": w["members"], "precision": args.precision,
                   "l2": "state larger than L2 (not flushed)", **extra,
                   "speedup_vs_one_launch_per_member": round(seq / ms_per_step, 3) if seq else None},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": recorded_traffic(args.workload, args.precision),
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)", "kernel": extra["step_kernels"],
                     "alg_bytes_per_site": bpsite},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clocks,
        "flow_study": study,
    }
    print(json.dumps(line), flush=True)
    return 0


def unet_train_flops_per_sample(H=64, W=256, levels=4, base=32, in_ch=5, out_ch=3) -> float:
    """Algorithmic FLOPs of one training sample (forward + data gradient + weight gradient;
    the first layer needs no data gradient): 2 MACs per weight use per pixel."""
    fwd = first = 0.0
    C = [base << l for l in range(levels)]
    for l in range(levels):
        P = (H >> l) * (W >> l)
        cin = in_ch if l == 0 else C[l - 1]
        fwd += 2 * P * C[l] * 9 * (cin + C[l])
        if l == 0:
            first = 2 * P * C[l] * 9 * cin
    for l in range(levels - 1):
        P = (H >> l) * (W >> l)
        fwd += 2 * P * C[l] * 9 * (C[l + 1] + 2 * C[l] + C[l])
    fwd += 2 * H * W * out_ch * base
    return 3 * fwd - first


def main_warmstart(args, w, torch, ws_, rank, local, dist):
    """Time to steady state of held-out channels started warm from the trained surrogate,
    against cold starts; one JSON line. Replicas under torchrun (each rank its own study)."""
    from paper_2003_11069_gb300 import unet
    from paper_2003_11069_gb300 import warmstart as wst
    stream = torch.cuda.Stream()
    train = wst.channels(args.ws_train, seed=100 + rank, ah_range=(0.0, 0.01))
    test = wst.channels(args.ws_test, seed=999 + rank, ah_range=(0.0, 0.01))
    every = 200
    horizon = args.ws_horizon
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with ClockSampler(local) as clk:
        res = wst.experiment(train, test, steps=horizon, every=every, snap_from=int(0.72 * horizon) // 2000 * 2000,
                             snap_every=2000, epochs=30, batch=32, lr=1e-3, stream=stream.cuda_stream,
                             log=lambda m: print(m, file=sys.stderr))
    wall = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    # the surrogate's training step alone, timed with CUDA events on its stream
    cfg = unet.make_config(max_batch=32, stream=stream.cuda_stream)
    net = unet.Net(cfg)
    X = torch.randn(64, 64, 256, 5, device="cuda")
    T = torch.randn(64, 64, 256, 3, device="cuda")
    idx = torch.arange(32, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        net.train_step(X, T, idx=idx, batch=32, lr=1e-4)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 20
    l0 = net.launches()
    s.record(stream)
    for _ in range(n):
        net.train_step(X, T, idx=idx, batch=32, lr=1e-4)
    e.record(stream)
    torch.cuda.synchronize()
    step_ms = s.elapsed_time(e) / n
    launches = (net.launches() - l0) // n
    net.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    flops = unet_train_flops_per_sample() * 32
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        pk = json.load(fh)
    peak = float(pk.get("bf16_tflops", 1900.0))
    achieved = flops / (step_ms * 1e-3) / 1e12
    sm = res["summary"]
    cpu = None
    if not args.no_cpu_baseline:
        cpu = unet_cpu_baseline()
    line = {
        "metric": "time-to-steady-state speedup (median over held-out channels, warm vs cold start, flow rate "
                  "within 1%)",
        "value": sm["median_speedup_warm"], "unit": "x", "n_gpus": ws_, "steps": horizon, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 network (f32 accumulate), f32 lattice Boltzmann", "data": "synthetic",
        "config": {"workload": w["desc"], "train_channels": len(train), "test_channels": len(test),
                   "snapshots": res["snapshots"], "horizon_steps": horizon, "record_every": every,
                   "window_steps": res["window_steps"], "l2": "not applicable (whole pipeline)",
                   "wall_seconds": round(wall, 1), "data_seconds": round(res["data_seconds"], 1),
                   "train_seconds": round(res["train_seconds"], 1), "train_steps": res["train_steps"],
                   "test_lb_seconds": round(res["lb_seconds_test"], 1)},
        "summary": sm,
        "roofline": {"bound": "tensor", "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                     "kernel": "U-Net training step (batch 32, 64x256, all kernels)",
                     "flops_per_step": flops, "ms_per_train_step": round(step_ms, 4)},
        "cpu_baseline": cpu, "e2e": None, "gpu_launches": int(launches),
        "gpu_launches_note": "kernel launches of one U-Net training step",
        "clocks": clk.summary(),
    }
    print(json.dumps(line, default=float), flush=True)
    return 0


def unet_cpu_baseline(budget_s: float = 15.0) -> dict:
    """The FP64 U-Net oracle (numpy) on the host: forward + backward of single 64x256 samples."""
    from oracle import unet_oracle as U
    shapes = U.layer_shapes(4, 32, 5, 3)
    params = inputs.unet_params(shapes, 0)
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 64, 256, 5))
    t = rng.normal(size=(1, 64, 256, 3))
    n, t0 = 0, time.perf_counter()
    while True:
        U.loss_and_grads(params, x, t, levels=4)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 50:
            break
    el = time.perf_counter() - t0
    return {"value": round(unet_train_flops_per_sample() * n / el / 1e12, 5), "unit": "TFLOP/s",
            "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{n} single-sample forward+backward passes of the 4-level U-Net oracle (numpy FP64)"}


if __name__ == "__main__":
    sys.exit(main())
