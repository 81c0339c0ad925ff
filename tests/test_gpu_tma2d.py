"""The persistent TMA-fed D2Q9 FP32 step, against the FP64 oracle.

The kernel reads each tile's 48 x 28 population neighbourhood from a TMA copy in shared
memory, patches the cells beyond a periodic edge with their images, and hands tiles out
through an atomic counter that alternates between launches; the cases cover walls,
periodic y, ragged tiles, fewer NCI probes, NCI off and the exact difference method. Each case runs several steps one at a time; after every step the GPU state is
compared with one oracle step from the GPU's own previous state (errors do not
accumulate), on the population scale max(|f|, w_i), at every site whose NCI decision
is not within 1e-5 of a floating-point tie.
"""
import numpy as np
import pytest

import oracle
from paper_2003_11069_gb300 import inputs, lbnci

from test_gpu_parity import FP32_TOL, _cfg, _near_tie_sites, _scale
from test_gpu_precision import step_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbnci.load()


CASES = {
    # walls in y, 6 x 5 tiles of which 20 take the TMA path
    "channel192x80_walls": dict(p=dict(nx=192, ny=80, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                                       force=(1e-5, 0, 0)),
                                gen=lambda: inputs.channel_emulsion_2d(192, 80, seed=21, r_lo=9, r_hi=12)),
    # periodic in y: the neighbourhood wraps for the first and last tile rows (slow path)
    "periodic160x96": dict(p=dict(nx=160, ny=96, tau=0.9, A_s=0.01, beta=0.7, A_h=0.05, force=(1e-5, 2e-6, 0)),
                           gen=lambda: inputs.channel_emulsion_2d(160, 96, seed=22, r_lo=9, r_hi=12)),
    # ragged last tile row, periodic y, h_max = 3.5 (three probes)
    "ragged128x50": dict(p=dict(nx=128, ny=50, tau=0.8, A_s=0.02, beta=0.5, A_h=0.1, h_min=1.5, h_max=3.5,
                                force=(2e-5, -1e-5, 0)),
                         gen=lambda: inputs.channel_emulsion_2d(128, 50, seed=23, r_lo=7, r_hi=9, film=0.5)),
    # NCI off: the kernel built for a psi halo of radius 1
    "nci_off160x64": dict(p=dict(nx=160, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.0,
                                 force=(1e-5, 0, 0)),
                          gen=lambda: inputs.channel_emulsion_2d(160, 64, seed=24, r_lo=9, r_hi=12)),
    # the paper's forcing: exact difference method, NCI on the dispersed phase only
    "edm192x64": dict(p=dict(nx=192, ny=64, wall_y=1, tau=0.9, A_s=0.01, beta=0.7, A_h=0.05,
                             force=(1e-5, 0, 0), forcing=1),
                      gen=lambda: inputs.channel_emulsion_2d(192, 64, seed=25, r_lo=9, r_hi=12)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_tma2d_steps(name):
    case = CASES[name]
    p = oracle.make_params(lattice=oracle.D2Q9, **case["p"])
    fl = case["gen"]()
    Q, N = 9, p.nx * p.ny
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_TMA2D
        sim.init_fields(fl.rho1, fl.rho2)
        sim.step(20)  # let interfaces and flow develop
        checked = 0
        for _ in range(6):
            f0 = sim.get_populations()
            sim.step(1)
            got = sim.get_populations()
            ref = oracle.step(p, f0, 1)
            near, of = _near_tie_sites(p, f0)
            rel = (np.abs(got - ref) / _scale(p, ref)).reshape(2 * Q, N)
            ok = ~near
            assert ok.mean() > 0.97
            err = rel[:, ok].max()
            assert err <= FP32_TOL, f"{name}: max rel err {err:.3e}"
            if p.A_h > 0:
                assert (of["hit"][ok] > 0).sum() > 0  # NCI acts on compared sites
            checked += 1
        obs = sim.observables()
    assert checked == 6 and obs["n_bad"] == 0


@pytest.mark.parametrize("name", ["channel192x80_walls", "periodic160x96", "ragged128x50", "edm192x64"])
def test_fp16dev_tma2d_steps(name):
    """FP16-deviation storage on the TMA kernel (deviation planes and reference densities
    copied by TMA, decoded in shared memory): each step within the FP16-dev per-step bound
    (step_error) of one oracle step from the GPU's own previous state."""
    case = CASES[name]
    p = oracle.make_params(lattice=oracle.D2Q9, **case["p"])
    fl = case["gen"]()
    Q, N = 9, p.nx * p.ny
    with lbnci.Sim(_cfg(p, lbnci.LB_FP16DEV)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_TMA2D
        sim.init_fields(fl.rho1, fl.rho2)
        sim.step(20)
        for _ in range(4):
            f0 = sim.get_populations()
            sim.step(1)
            got = sim.get_populations()
            ref = oracle.step(p, f0, 1)
            near, _ = _near_tie_sites(p, f0)
            err = step_error(p, got, ref, lbnci.LB_FP16DEV)
            assert (~near).mean() > 0.97
            assert err[:, ~near].max() <= 1.0, f"{name}: {err[:, ~near].max():.3f}"
        assert sim.observables()["n_bad"] == 0


def test_fp32_tma2d_after_set_populations():
    """A state set from the host after some steps is what the next step reads (the
    tensor maps follow the buffer swap)."""
    p = oracle.make_params(lattice=oracle.D2Q9, nx=192, ny=80, wall_y=1, tau=1.0, A_s=0.01, beta=0.7,
                           A_h=0.05, force=(1e-5, 0, 0))
    fa = inputs.channel_emulsion_2d(192, 80, seed=31, r_lo=9, r_hi=12)
    fb = inputs.channel_emulsion_2d(192, 80, seed=32, r_lo=9, r_hi=12)
    f_b = oracle.step(p, oracle.init(p, fb.rho1, fb.rho2), 5).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.init_fields(fa.rho1, fa.rho2)
        sim.step(3)
        sim.set_populations(f_b)
        sim.step(1)
        got = sim.get_populations()
    ref = oracle.step(p, f_b, 1)
    near, _ = _near_tie_sites(p, f_b)
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(18, -1)
    assert rel[:, ~near].max() <= FP32_TOL


def test_step_path_selection(monkeypatch):
    def path(**kw):
        cfg = lbnci.lb_config_make(**kw)
        with lbnci.Sim(cfg) as sim:
            return sim.step_path()

    base = dict(nx=64, ny=32, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05)
    assert path(**base, precision=lbnci.LB_FP32) == lbnci.LB_PATH_TMA2D
    assert path(**dict(base, nx=37), precision=lbnci.LB_FP32) == lbnci.LB_PATH_FUSED2D
    assert path(**base, precision=lbnci.LB_FP64) == lbnci.LB_PATH_FUSED2D
    assert path(**base, precision=lbnci.LB_FP16DEV) == lbnci.LB_PATH_TMA2D
    assert path(**dict(base, nx=38), precision=lbnci.LB_FP16DEV) == lbnci.LB_PATH_FUSED2D
    assert path(lattice=1, nx=16, ny=8, nz=8, wall_y=1, wall_z=1, tau=1.0, A_s=0.01, beta=0.7,
                precision=lbnci.LB_FP32) == lbnci.LB_PATH_D3Q27
    d3 = dict(lattice=1, nx=32, ny=8, nz=8, wall_y=1, wall_z=1, tau=1.0, A_s=0.01, beta=0.7)
    assert path(**d3, precision=lbnci.LB_FP32) == lbnci.LB_PATH_D3Q27_STREAM
    assert path(**d3, precision=lbnci.LB_FP16DEV) == lbnci.LB_PATH_D3Q27_STREAM
    assert path(**d3, precision=lbnci.LB_FP64) == lbnci.LB_PATH_D3Q27
    assert path(**dict(d3, ny=12), precision=lbnci.LB_FP32) == lbnci.LB_PATH_D3Q27
    monkeypatch.setenv("LBNCI_FUSED", "classic")
    assert path(**base, precision=lbnci.LB_FP32) == lbnci.LB_PATH_FUSED2D
    monkeypatch.setenv("LBNCI_D3_KERNEL", "march")
    assert path(**d3, precision=lbnci.LB_FP16DEV) == lbnci.LB_PATH_D3Q27
    monkeypatch.setenv("LBNCI_D3_KERNEL", "carry")
    assert path(**d3, precision=lbnci.LB_FP32) == lbnci.LB_PATH_D3Q27_CARRY
    assert path(**d3, precision=lbnci.LB_FP16DEV) == lbnci.LB_PATH_D3Q27_CARRY


def test_fp32_tma2d_and_classic_agree():
    """The TMA-fed kernel and the one-pass fused kernel compute the same FP32 step (the
    NCI probe offsets round ties differently, and the compilers contract differently):
    over 50 steps of the channel emulsion their states stay close, and mass is kept."""
    import os
    fl = inputs.channel_emulsion_2d(256, 64, seed=41, r_lo=10, r_hi=13)
    cfg = lbnci.lb_config_make(nx=256, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0, 0), precision=lbnci.LB_FP32)
    out = {}
    for mode in ("tma", "classic"):
        if mode == "classic":
            os.environ["LBNCI_FUSED"] = "classic"
        try:
            with lbnci.Sim(cfg) as sim:
                sim.init_fields(fl.rho1, fl.rho2)
                m0 = sim.observables()["mass"]
                sim.step(50)
                out[mode] = (sim.get_populations(), sim.observables(), m0, sim.step_path())
        finally:
            os.environ.pop("LBNCI_FUSED", None)
    assert out["tma"][3] == lbnci.LB_PATH_TMA2D and out["classic"][3] == lbnci.LB_PATH_FUSED2D
    fc, fk = out["tma"][0], out["classic"][0]
    d = np.abs(fc - fk) / np.maximum(np.abs(fk), 1.0 / 36.0)
    assert np.median(d) < 1e-5 and np.quantile(d, 0.99) < 1e-3
    for mode in out:
        obs, m0 = out[mode][1], out[mode][2]
        assert np.all(np.abs(obs["mass"] - m0) / m0 < 1e-5) and obs["n_bad"] == 0


@pytest.mark.parametrize("nx,ny,walls", [(8, 8, 0), (12, 5, 1), (36, 20, 0), (40, 19, 1), (64, 33, 0)])
def test_fp32_tma2d_tiny_and_ragged(nx, ny, walls):
    """Lattices smaller than one tile or with ragged tiles: every box cell beyond the
    lattice is the periodic image (x, and y without walls) or lies beyond a wall; own
    positions beyond the lattice hold psi of their image or mirror. One step within
    FP32_TOL of the oracle at sites away from NCI ties, on the TMA path."""
    p = oracle.make_params(lattice=oracle.D2Q9, nx=nx, ny=ny, wall_y=walls, tau=0.8, A_s=0.02, beta=0.5,
                           A_h=0.1, h_min=1.5, h_max=3.5, force=(2e-5, -1e-5, 0))
    rng = np.random.default_rng(nx * 100 + ny)
    rho1 = rng.uniform(0.05, 0.95, nx * ny)
    f0 = oracle.init(p, rho1, 1.0 - rho1).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_TMA2D
        sim.set_populations(f0)
        sim.step(1)
        got = sim.get_populations()
    ref = oracle.step(p, f0, 1)
    near, _ = _near_tie_sites(p, f0)
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(18, nx * ny)
    assert (~near).mean() > 0.8
    assert rel[:, ~near].max() <= FP32_TOL, rel[:, ~near].max()


@pytest.mark.parametrize("precision", [lbnci.LB_FP32, lbnci.LB_FP16DEV])
@pytest.mark.parametrize("nx,ny,walls", [(160, 96, 0), (192, 80, 1), (2048, 256, 1)])
def test_chained_steps_equal_separate_steps(precision, nx, ny, walls):
    """lb_step(n) launches n steps back to back, and each launch may begin while the
    previous one finishes (programmatic dependent launch: a CTA's prologue overlaps the
    previous grid's tail, and it waits for that grid before touching global memory). The
    chained steps must give exactly the state of the same steps taken one at a time with
    the stream drained in between, on a periodic-y lattice (every edge tile reads the
    periodic images of its box with plain loads), a walled one, and the 2048 x 256
    channel (1024 tiles, several per CTA)."""
    fl = inputs.channel_emulsion_2d(nx, ny, seed=nx + ny, r_lo=9, r_hi=12)
    cfg = lbnci.lb_config_make(nx=nx, ny=ny, wall_y=walls, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0, 0), precision=precision)
    with lbnci.Sim(cfg) as chained, lbnci.Sim(cfg) as single:
        assert chained.step_path() == lbnci.LB_PATH_TMA2D
        chained.init_fields(fl.rho1, fl.rho2)
        single.init_fields(fl.rho1, fl.rho2)
        chained.step(30)
        for _ in range(30):
            single.step(1)
            single.observables()  # ends with a stream synchronisation
        assert np.array_equal(chained.get_populations(), single.get_populations())
        assert chained.observables()["n_nci"] > 0


def test_tma_wait_failure_is_reported_and_context_survives(monkeypatch):
    """Failure path of the TMA kernel's bounded waits, without a GPU fault: with
    LBNCI_TMA_STALL_TEST=1 every CTA expects 16 bytes more than its first copy brings, so
    its mbarrier wait runs out after about a second; the kernel records the failure and
    returns, lb_observables reports LB_ECUDA, and the context stays usable (a new sim
    steps and matches the oracle)."""
    import time
    p = oracle.make_params(lattice=oracle.D2Q9, nx=64, ny=32, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                           force=(1e-5, 0, 0))
    fl = inputs.channel_emulsion_2d(64, 32, seed=51, r_lo=6, r_hi=8)
    monkeypatch.setenv("LBNCI_TMA_STALL_TEST", "1")
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        t0 = time.time()
        sim.step(1)
        with pytest.raises(lbnci.LBError) as ei:
            sim.observables()
        elapsed = time.time() - t0
    assert ei.value.status == lbnci.LB_ECUDA and "gave up waiting" in str(ei.value)
    assert 0.5 < elapsed < 30.0
    monkeypatch.delenv("LBNCI_TMA_STALL_TEST")
    f0 = oracle.init(p, fl.rho1, fl.rho2).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.set_populations(f0)
        sim.step(1)
        got = sim.get_populations()
        assert sim.observables()["n_bad"] == 0
    ref = oracle.step(p, f0, 1)
    near, _ = _near_tie_sites(p, f0)
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(18, -1)
    assert rel[:, ~near].max() <= FP32_TOL
