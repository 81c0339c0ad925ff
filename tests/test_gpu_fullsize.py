"""Parity at the benchmark's full sizes, through the launches the benchmark times.

Workloads (generators, seeds and physics of `bench.py`):
  * the D2Q9 channel 2048 x 256 (FP32 and FP16-deviation storage; persistent TMA kernel,
    1024 tiles over the resident CTAs, tiles from the counter);
  * the D3Q27 duct 512 x 128 x 128 (FP32 and FP16-deviation storage; the streaming step:
    moments, normals, collision; the steps store the total + recolouring form);
  * the 96-channel ensemble (one batched TMA launch per step over 20.9 M sites).
Each case advances the GPU a few steps from the generated fields (interfaces sharpen
and NCI contacts form), reads the state f0, takes ONE more GPU step and compares it
with one oracle step from f0 (reading leaves the state in the form the steps store it), on the population scale max(|f|, w_i), at every compared
site whose NCI decision is not within 1e-5 of a floating-point tie; decisions must agree
everywhere else.

Compared outputs: every site of the 2-D channel; every site of six sampled ensemble
members; for the duct, every site of two x-slabs, one across the periodic seam
x = 511 | 0. A step's output at a site depends on the input within S + 2 = 6 sites
(pull, psi, its gradient, the NCI ray of S = floor(h_max) = 4 steps, the gradient at
its end, and the pull behind that psi), so the oracle run on a 64-wide slab, periodic
in x, is exact at the slab's 48 central columns, and those are the ones compared.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_2003_11069_gb300 import inputs, lbnci

from test_gpu_parity import _cfg, _near_tie_sites
from test_gpu_precision import step_error

pytestmark = pytest.mark.gpu

WARM_STEPS = 20
SEED = 1234  # rank 0's seed in bench.py
SLAB, SLAB_EDGE = 64, 8  # slab width in x, columns dropped at each end (> S + 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbnci.load()


def _params(name):
    w = bench.WORKLOADS[name]
    return oracle.make_params(lattice=w["lattice"], nx=w["nx"], ny=w["ny"], nz=w["nz"], wall_y=w["wall_y"],
                              wall_z=w["wall_z"], tau=w["tau"], A_s=w["A_s"], beta=w["beta"], A_h=w["A_h"],
                              force=tuple(w["force"])), w


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def _compare(p, f0, got, gpu_hit, precision, sites=None, form=lbnci.LB_STATE_PAIRS):
    """One oracle step from f0 against the GPU's step `got` ([2][Q][N] arrays of the
    lattice p); `gpu_hit` = the GPU's NCI hit map of f0; `sites` = the compared site
    indices (all when None). Returns (max error in units of the precision's per-step
    bound, number of compared sites)."""
    ref = oracle.step(p, f0, 1, nthreads=0)
    near, of = _near_tie_sites(p, f0)
    Q, N = oracle.Q_of(p), oracle.N_of(p)
    sel = np.ones(N, bool) if sites is None else np.isin(np.arange(N), sites)
    differ = (gpu_hit != of["hit"]) & sel
    assert not (differ & ~near).any(), f"{int((differ & ~near).sum())} NCI decisions differ away from ties"
    ok = sel & ~near & ~differ
    assert ok.sum() > 0.95 * sel.sum()
    if p.A_h > 0:
        assert (of["hit"][ok] > 0).sum() > 0, "NCI must be active among the compared sites"
    err = float(step_error(p, got, ref, precision, form)[:, ok].max())
    assert err <= 1.0, err
    return err, int(ok.sum())


@pytest.mark.parametrize("precision", [lbnci.LB_FP32, lbnci.LB_FP16DEV])
def test_channel2048x256_full_size(precision):
    p, w = _params("channel2d")
    fl = w["gen"](p.nx, p.ny, p.nz, SEED)
    with lbnci.Sim(_cfg(p, precision)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_TMA2D
        sim.init_fields(fl.rho1, fl.rho2)
        sim.step(WARM_STEPS)
        f0 = sim.get_populations()
        hit = sim.fields()["hit"]
        sim.step(1)
        got = sim.get_populations()
    err, n = _compare(p, f0, got, hit, precision)
    print(f"channel 2048x256 precision {precision}: max error {err:.3f} of the per-step bound over {n} sites")


def _slab(f, p, xs):
    """Columns xs (in order) of a [2][Q][nz][ny][nx] population array, as a lattice of
    width len(xs), periodic in x."""
    Q = oracle.Q_of(p)
    v = f.reshape(2 * Q, p.nz, p.ny, p.nx)[..., xs]
    return np.ascontiguousarray(v).reshape(-1)


@pytest.mark.parametrize("precision", [lbnci.LB_FP32, lbnci.LB_FP16DEV])
def test_duct512x128x128_full_size_slabs(precision):
    if _mem_available_gb() < 16:
        pytest.skip("needs several GB of host memory (the 3.6 GB FP64 state, fields, slabs)")
    p, w = _params("duct3d")
    fl = w["gen"](p.nx, p.ny, p.nz, SEED)
    slabs = [np.arange(-SLAB // 2, SLAB // 2) % p.nx, np.arange(200, 200 + SLAB)]  # the seam, the middle
    form = lbnci.LB_STATE_TOTAL_RECOLOUR
    with lbnci.Sim(_cfg(p, precision)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_D3Q27_STREAM and sim.state_form() == form
        sim.init_fields(fl.rho1, fl.rho2)
        sim.step(WARM_STEPS)
        f0 = sim.get_populations()
        f0s = [_slab(f0, p, xs) for xs in slabs]
        del f0
        hit = sim.fields()["hit"].reshape(p.nz, p.ny, p.nx)
        hits = [np.ascontiguousarray(hit[..., xs]).reshape(-1) for xs in slabs]
        del hit
        sim.step(1)
        got = sim.get_populations()
        gots = [_slab(got, p, xs) for xs in slabs]
        del got
    ps = oracle.make_params(lattice=p.lattice, nx=SLAB, ny=p.ny, nz=p.nz, wall_y=p.wall_y, wall_z=p.wall_z,
                            tau=p.tau, A_s=p.A_s, beta=p.beta, A_h=p.A_h, h_min=p.h_min, h_max=p.h_max,
                            g_th=p.g_th, force=tuple(p.force))
    assert SLAB_EDGE > int(np.floor(p.h_max)) + 2
    lx = np.arange(SLAB)
    keep = (lx >= SLAB_EDGE) & (lx < SLAB - SLAB_EDGE)
    sites = np.flatnonzero(np.broadcast_to(keep, (p.nz, p.ny, SLAB)).reshape(-1))
    for k, (a, b, h) in enumerate(zip(f0s, gots, hits)):
        err, n = _compare(ps, a, b, h, precision, sites, form)
        print(f"duct 512x128x128 precision {precision} slab {k}: max error {err:.3f} of the per-step bound over {n} sites")


@pytest.mark.parametrize("precision", [lbnci.LB_FP32, lbnci.LB_FP16DEV])
def test_ensemble96_full_size_sampled_members(precision):
    w = bench.WORKLOADS["ensemble"]
    members = inputs.ensemble_channels(w["members"], seed=SEED)
    cfgs = [lbnci.lb_config_make(nx=m.nx, ny=m.ny, wall_y=1, tau=w["tau"], A_s=w["A_s"], beta=w["beta"],
                                 A_h=m.A_h, force=(m.force, 0.0, 0.0), precision=precision) for m in members]
    sizes = [m.nx * m.ny for m in members]
    rng = np.random.default_rng(5)
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argmax([m.A_h for m in members])),
                   *rng.choice(len(members), 3, replace=False).tolist()})
    with lbnci.Ensemble(cfgs) as ens:
        assert all(m.step_path() == lbnci.LB_PATH_TMA2D for m in ens.members)
        for mv, m in zip(ens.members, members):
            mv.init_fields(m.fields.rho1, m.fields.rho2)
        ens.tune()
        ens.step(WARM_STEPS)
        f0 = {k: ens.members[k].get_populations() for k in pick}
        hits = {k: ens.members[k].fields()["hit"] for k in pick}
        ens.step(1)
        got = {k: ens.members[k].get_populations() for k in pick}
    for k in pick:
        m = members[k]
        p = oracle.make_params(lattice=oracle.D2Q9, nx=m.nx, ny=m.ny, wall_y=1, tau=w["tau"], A_s=w["A_s"],
                               beta=w["beta"], A_h=m.A_h, force=(m.force, 0.0, 0.0))
        err, n = _compare(p, f0[k], got[k], hits[k], precision)
        print(f"ensemble member {k} ({m.nx}x{m.ny}, A_h {m.A_h:.3f}): max error {err:.3f} of the per-step bound over {n} sites")
