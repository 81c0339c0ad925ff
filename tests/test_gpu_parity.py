"""GPU (CUDA, through the C ABI) versus the FP64 CPU oracle, element by element.

FP64 path: from identical states, every population after 1, 10 and 100 steps within
1e-12 relative to the population's own scale max(|f|, w_i rho0); NCI hit maps
bit-exact. FP32 path: per-step error within the FP32 tolerance derived in the design
notes, decisions compared where they are not near a floating-point tie.
"""
import numpy as np
import pytest

import oracle
from paper_2003_11069_gb300 import inputs, lbnci

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbnci.load()


def _cfg(p, precision=lbnci.LB_FP64):
    return lbnci.lb_config_make(
        lattice=p.lattice, nx=p.nx, ny=p.ny, nz=p.nz, wall_y=p.wall_y, wall_z=p.wall_z,
        tau=p.tau, A_s=p.A_s, beta=p.beta, A_h=p.A_h, h_min=p.h_min, h_max=p.h_max, g_th=p.g_th,
        force=tuple(p.force), precision=precision, forcing=p.forcing)


def _scale(p, f):
    """Per-element scale max(|f|, w_i) of a [2][Q][N] population array."""
    _, w, _ = oracle.lattice(p.lattice)
    Q, N = len(w), oracle.N_of(p)
    wq = np.tile(np.repeat(w, N), 2)
    return np.maximum(np.abs(f), wq)


def _max_rel(p, got, ref):
    return float(np.max(np.abs(got - ref) / _scale(p, ref)))


def _run_pair(p, rho1, rho2, steps_list, precision=lbnci.LB_FP64):
    f0 = oracle.init(p, rho1, rho2)
    with lbnci.Sim(_cfg(p, precision)) as sim:
        sim.init_fields(rho1, rho2)
        g0 = sim.get_populations()
        if precision == lbnci.LB_FP64:
            assert _max_rel(p, g0, f0) <= 1e-15  # same equilibrium arithmetic
        f = g0.copy()  # the oracle continues from the GPU's (rounded) state
        done = 0
        out = []
        for n in steps_list:
            sim.step(n - done)
            f = oracle.step(p, f, n - done)
            done = n
            out.append((n, sim.get_populations(), f.copy()))
        fields = sim.fields()
    return out, fields


CASES = {
    "droplet128_nci0": dict(p=dict(nx=128, ny=128, tau=1.0, A_s=0.01, beta=0.7, A_h=0.0),
                            gen=lambda: inputs.droplet(128, 128, radius=30)),
    "droplet128_nci": dict(p=dict(nx=128, ny=128, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05),
                           gen=lambda: inputs.droplet(128, 128, radius=30)),
    "channel128x64_nci": dict(p=dict(nx=128, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                                     force=(1e-5, 0, 0)),
                              gen=lambda: inputs.channel_emulsion_2d(128, 64, seed=7, r_lo=10, r_hi=13)),
    "ragged37x19": dict(p=dict(nx=37, ny=19, wall_y=1, tau=0.8, A_s=0.02, beta=0.5, A_h=0.1,
                               h_min=1.5, h_max=3.5, force=(2e-5, -1e-5, 0)),
                        gen=lambda: inputs.channel_emulsion_2d(37, 19, seed=3, r_lo=4, r_hi=5, film=0.5)),
}


@pytest.mark.parametrize("spt", ["2", "4"])
@pytest.mark.parametrize("name", list(CASES))
def test_fp64_d2q9_parity(name, spt, monkeypatch):
    """Both tilings of the fused D2Q9 kernel (32x16 and 32x32 sites per block)."""
    monkeypatch.setenv("LBNCI_FUSED_SPT", spt)
    case = CASES[name]
    p = oracle.make_params(lattice=oracle.D2Q9, **case["p"])
    fl = case["gen"]()
    out, fields = _run_pair(p, fl.rho1, fl.rho2, [1, 10, 100])
    for n, got, ref in out:
        err = _max_rel(p, got, ref)
        assert err <= FP64_RTOL, f"{name}: step {n}: max rel err {err:.3e}"
    of = oracle.fields(p, out[-1][2])
    assert np.array_equal(fields["hit"], of["hit"])
    if p.A_h > 0 and name != "droplet128_nci":
        assert (of["hit"] > 0).sum() > 0, "NCI must be active in this case"
    for k in ("rho1", "rho2", "psi"):
        assert np.max(np.abs(fields[k] - of[k])) <= 1e-13
    for k in ("grad", "frep", "u"):
        assert np.max(np.abs(fields[k] - of[k])) <= 1e-14


def _duct_fields(nx, ny, nz, seed):
    return inputs.duct_emulsion_3d(nx, ny, nz, seed=seed, radius=5.0, volume_fraction=0.5)


@pytest.mark.parametrize("kernel", ["march", "tiled"])
@pytest.mark.parametrize("walls", [(1, 1), (0, 1), (0, 0)])
def test_fp64_d3q27_parity(walls, kernel, monkeypatch):
    """Both D3Q27 collision kernels (z-marching, default; 3-D tiles)."""
    monkeypatch.setenv("LBNCI_D3_KERNEL", kernel)
    nx, ny, nz = 40, 22, 17  # ragged against the 32x4x2 tile
    p = oracle.make_params(lattice=oracle.D3Q27, nx=nx, ny=ny, nz=nz, wall_y=walls[0], wall_z=walls[1],
                           tau=0.9, A_s=0.01, beta=0.7, A_h=0.03, force=(2e-6, 0, 1e-6))
    fl = _duct_fields(nx, ny, nz, seed=11)
    out, fields = _run_pair(p, fl.rho1, fl.rho2, [1, 10])
    for n, got, ref in out:
        err = _max_rel(p, got, ref)
        assert err <= FP64_RTOL, f"walls {walls}: step {n}: max rel err {err:.3e}"
    of = oracle.fields(p, out[-1][2])
    assert np.array_equal(fields["hit"], of["hit"])
    assert (of["hit"] > 0).sum() > 0


def test_fp64_observables_parity():
    p = oracle.make_params(lattice=oracle.D2Q9, nx=96, ny=48, wall_y=1, tau=1.0, A_s=0.01, beta=0.7,
                           A_h=0.05, force=(1e-5, 0, 0))
    fl = inputs.channel_emulsion_2d(96, 48, seed=5, r_lo=8, r_hi=10)
    with lbnci.Sim(_cfg(p)) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        sim.step(50)
        f = sim.get_populations()
        psi = np.empty(p.nx * p.ny)
        u = np.empty(3 * p.nx * p.ny)
        obs = sim.observables(psi, u)
    ref = oracle.observables(p, f)
    of = oracle.fields(p, f)
    assert obs["step"] == 50
    assert np.allclose(obs["mass"], ref["mass"], rtol=1e-13, atol=0)
    mscale = np.abs((of["rho1"] + of["rho2"]) * of["u"]).sum()
    assert np.max(np.abs(obs["momentum"] - ref["momentum"])) <= 1e-13 * mscale
    assert abs(obs["flow_rate"] - ref["flow_rate"]) <= 1e-13 * mscale / p.nx
    assert abs(obs["flow_rate_disp"] - ref["flow_rate_disp"]) <= 1e-13 * mscale / p.nx
    assert obs["n_nci"] == int((of["hit"] > 0).sum())
    g = np.sqrt((of["grad"] ** 2).sum(axis=0))
    assert obs["n_interface"] == int((g > p.g_th).sum())
    assert obs["n_bad"] == 0
    assert np.max(np.abs(psi - of["psi"])) <= 1e-13
    assert np.max(np.abs(u - of["u"].ravel())) <= 1e-14


def test_fp64_mass_conservation_long():
    """1000 steps with walls, forcing and NCI: each component's mass is kept to rounding."""
    fl = inputs.channel_emulsion_2d(256, 64, seed=2, r_lo=10, r_hi=13)
    cfg = lbnci.lb_config_make(nx=256, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0, 0))
    with lbnci.Sim(cfg) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        m0 = sim.observables()["mass"]
        sim.step(1000)
        o = sim.observables()
    assert np.all(np.abs(o["mass"] - m0) / m0 < 1e-12)
    assert o["n_nci"] > 0


@pytest.mark.parametrize("A_h", [0.0, 0.05])
def test_fp64_droplet_2000_steps_laplace_and_mass(A_h):
    """The plain-method FP64 case: a droplet of radius 30 (tanh profile, width 2) in a
    periodic 128 x 128 box, tau = 1, A_s = 0.01, beta = 0.7, 2000 steps, with and without
    NCI. The GPU state equals the oracle's (1e-12 on the population scale; in practice
    bitwise), each component's mass is kept to rounding, and the pressure jump
    c_s^2 (rho_in - rho_out) is within 20% of sigma/R with sigma = 4 A_s tau/9 (a single
    radius carries the intercept of the fit; the slope is pinned on the oracle across
    radii). With one droplet no interface faces another within h_max: NCI stays off."""
    n, R, A_s, tau = 128, 30.0, 0.01, 1.0
    p = oracle.make_params(nx=n, ny=n, tau=tau, A_s=A_s, beta=0.7, A_h=A_h)
    fl = inputs.droplet(n, n, radius=R)
    with lbnci.Sim(_cfg(p)) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        f0 = sim.get_populations()
        m0 = sim.observables()["mass"]
        sim.step(2000)
        got = sim.get_populations()
        obs = sim.observables()
        fd = sim.fields()
    ref = oracle.step(p, f0, 2000)
    assert _max_rel(p, got, ref) <= FP64_RTOL
    assert np.all(np.abs(obs["mass"] - m0) / m0 < 1e-12)
    rho = (fd["rho1"] + fd["rho2"]).reshape(n, n)
    dp = (rho[n // 2, n // 2] - rho[0, 0]) / 3.0
    sigma = 4 * A_s * tau / 9
    assert abs(dp / (sigma / R) - 1) < 0.2, dp / (sigma / R)
    assert np.max(np.abs(fd["u"])) < 5e-4
    assert obs["n_nci"] == 0


def test_zero_steps_and_tiny_lattices():
    """nsteps = 0 leaves the state unchanged; 1-wide periodic axes and a one-row walled
    channel match the oracle."""
    for dims, walls in (((1, 5), 0), ((6, 1), 1), ((3, 3), 0)):
        nx, ny = dims
        p = oracle.make_params(nx=nx, ny=ny, wall_y=walls, tau=0.9, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-4, 0, 0))
        rng = np.random.default_rng(nx * 10 + ny)
        rho1 = rng.uniform(0.1, 0.9, nx * ny)
        rho2 = 1.0 - rho1
        with lbnci.Sim(_cfg(p)) as sim:
            sim.init_fields(rho1, rho2)
            f0 = sim.get_populations()
            sim.step(0)
            assert np.array_equal(sim.get_populations(), f0)
            sim.step(3)
            got = sim.get_populations()
        ref = oracle.step(p, f0, 3)
        assert _max_rel(p, got, ref) <= FP64_RTOL


def test_set_get_populations_roundtrip_and_workspace():
    p = oracle.make_params(nx=40, ny=24, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05)
    fl = inputs.channel_emulsion_2d(40, 24, seed=1, r_lo=5, r_hi=6)
    f0 = oracle.init(p, fl.rho1, fl.rho2)
    import torch
    with lbnci.Sim(_cfg(p), workspace="torch") as sim:
        sim.set_populations(f0)
        assert np.array_equal(sim.get_populations(), f0)
        sim.step(5)
        got = sim.get_populations()
        # device-side arrays through the same entry points
        fd = torch.empty(f0.size, dtype=torch.float64, device="cuda")
        lbnci.lb_get_populations(sim.h, fd)
        assert np.array_equal(fd.cpu().numpy(), got)
    assert _max_rel(p, got, oracle.step(p, f0, 5)) <= FP64_RTOL


# ----------------------------------------------------------------------------- FP32
FP32_TOL = 2e-6  # per-step error bound on the population scale (see the design notes)


def _near_tie_sites(p, f, margin=1e-5):
    """Sites whose NCI decision is within `margin` of a floating-point tie, judged on the
    oracle's FP64 fields: |grad psi| near g_th at the site, or, at a probe of its ray up
    to the oracle's hit (every probe when there is none), a probe offset s*n near a
    half-integer, |grad psi| near g_th at the probe, or a facing test n(y).n(x) near 0."""
    of = oracle.fields(p, f)
    N = oracle.N_of(p)
    grad = of["grad"]
    g = np.sqrt((grad ** 2).sum(axis=0))
    near = np.abs(g - p.g_th) < margin
    n = np.where(g > 0, -grad / np.where(g > 0, g, 1), 0.0)
    iface = g > p.g_th
    site = np.arange(N)
    x, y, z = site % p.nx, (site // p.nx) % p.ny, site // (p.nx * p.ny)
    hit = of["hit"]
    for s in range(1, int(np.floor(p.h_max)) + 1):
        v = s * n
        near |= iface & (np.abs(np.abs(v) - np.floor(np.abs(v)) - 0.5) < margin).any(axis=0)
        d = (np.sign(v) * np.floor(np.abs(v) + 0.5)).astype(np.int64)  # half away from zero
        if p.lattice == oracle.D2Q9:
            d[2] = 0
        live = iface & ((hit <= 0) | (s <= hit))
        px = (x + d[0]) % p.nx
        py, pz = y + d[1], z + d[2]
        if p.wall_y:
            live &= (py >= 0) & (py < p.ny)
        if p.wall_z:
            live &= (pz >= 0) & (pz < p.nz)
        probe = px + p.nx * ((py % p.ny) + p.ny * (pz % p.nz))
        gp = g[probe]
        dot = (n[:, probe] * n).sum(axis=0)
        near |= live & (np.abs(gp - p.g_th) < margin)
        near |= live & (gp > p.g_th) & (np.abs(dot) < margin)
    return near, of


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_fp32_one_step_tolerance(lat):
    """FP32 storage and arithmetic: one step from the same (FP32-representable) state.
    NCI decisions (hit distances) agree with the FP64 oracle's except at near-tie sites;
    where they agree, every population is within FP32_TOL of the oracle on the
    population scale max(|f|, w_i)."""
    if lat == oracle.D2Q9:
        p = oracle.make_params(lattice=lat, nx=160, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0, 0))
        fl = inputs.channel_emulsion_2d(160, 64, seed=9, r_lo=10, r_hi=13)
    else:
        p = oracle.make_params(lattice=lat, nx=40, ny=22, nz=17, wall_y=1, wall_z=1, tau=1.0, A_s=0.01,
                               beta=0.7, A_h=0.03, force=(2e-6, 0, 0))
        fl = _duct_fields(40, 22, 17, seed=4)
    f0 = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 20).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.set_populations(f0)
        assert np.array_equal(sim.get_populations(), f0)
        fields = sim.fields()
        sim.step(1)
        got = sim.get_populations()
    ref = oracle.step(p, f0, 1)
    near, of = _near_tie_sites(p, f0)
    Q, N = oracle.Q_of(p), oracle.N_of(p)
    differ = fields["hit"] != of["hit"]
    assert not (differ & ~near).any(), f"{int((differ & ~near).sum())} NCI decisions differ away from ties"
    assert differ.sum() <= max(3, near.sum())
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(2 * Q, N)
    ok = ~differ
    assert (of["hit"][ok] > 0).sum() > 0
    assert rel[:, ok].max() <= FP32_TOL, rel[:, ok].max()


def test_fp32_mass_conservation():
    """FP32: each component's mass drifts by no more than rounding over 2000 steps."""
    fl = inputs.channel_emulsion_2d(256, 64, seed=2, r_lo=10, r_hi=13)
    cfg = lbnci.lb_config_make(nx=256, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0, 0), precision=lbnci.LB_FP32)
    with lbnci.Sim(cfg) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        m0 = sim.observables()["mass"]
        sim.step(2000)
        o = sim.observables()
    assert np.all(np.abs(o["mass"] - m0) / m0 < 2e-5), (o["mass"], m0)
    assert o["n_nci"] > 0 and o["n_bad"] == 0


@pytest.mark.parametrize("nx,ny,walls", [(37, 19, 1), (6, 3, 0), (64, 33, 0)])
def test_fp32_ragged_and_tiny(nx, ny, walls):
    """The fused D2Q9 kernel on ragged tiles, lattices smaller than one tile and
    periodic y: one FP32 step within FP32_TOL of the oracle wherever NCI decisions
    agree."""
    p = oracle.make_params(lattice=oracle.D2Q9, nx=nx, ny=ny, wall_y=walls, tau=0.8, A_s=0.02, beta=0.5,
                           A_h=0.1, h_min=1.5, h_max=3.5, force=(2e-5, -1e-5, 0))
    rng = np.random.default_rng(nx * 100 + ny)
    rho1 = rng.uniform(0.05, 0.95, nx * ny)
    f0 = oracle.init(p, rho1, 1.0 - rho1).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.set_populations(f0)
        fields = sim.fields()
        sim.step(1)
        got = sim.get_populations()
    ref = oracle.step(p, f0, 1)
    near, of = _near_tie_sites(p, f0)
    Q, N = 9, nx * ny
    differ = fields["hit"] != of["hit"]
    assert not (differ & ~near).any(), f"{int((differ & ~near).sum())} NCI decisions differ away from ties"
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(2 * Q, N)
    ok = ~near  # a site's new populations depend on its own decision only
    assert ok.mean() > 0.9 and (of["hit"][ok] > 0).sum() > 0
    assert rel[:, ok].max() <= FP32_TOL, rel[:, ok].max()


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_fp64_edm_dispersed_parity(lat):
    """The paper's forcing (exact difference method, NCI on the dispersed phase only):
    FP64 per-step parity with the oracle, NCI active."""
    if lat == oracle.D2Q9:
        p = oracle.make_params(lattice=lat, nx=96, ny=48, wall_y=1, tau=0.9, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 2e-6, 0), forcing=1)
        fl = inputs.channel_emulsion_2d(96, 48, seed=5, r_lo=8, r_hi=10)
        steps = [1, 10, 100]
    else:
        p = oracle.make_params(lattice=lat, nx=40, ny=22, nz=17, wall_y=1, wall_z=1, tau=0.9, A_s=0.01,
                               beta=0.7, A_h=0.03, force=(2e-6, 0, 1e-6), forcing=1)
        fl = _duct_fields(40, 22, 17, seed=11)
        steps = [1, 10]
    out, fields = _run_pair(p, fl.rho1, fl.rho2, steps)
    for n, got, ref in out:
        err = _max_rel(p, got, ref)
        assert err <= FP64_RTOL, f"step {n}: max rel err {err:.3e}"
    of = oracle.fields(p, out[-1][2])
    assert np.array_equal(fields["hit"], of["hit"]) and (of["hit"] > 0).sum() > 0


def test_fp32_edm_one_step():
    p = oracle.make_params(lattice=oracle.D2Q9, nx=96, ny=48, wall_y=1, tau=0.9, A_s=0.01, beta=0.7, A_h=0.05,
                           force=(1e-5, 0, 0), forcing=1)
    fl = inputs.channel_emulsion_2d(96, 48, seed=5, r_lo=8, r_hi=10)
    f0 = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 20).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        sim.set_populations(f0)
        fields = sim.fields()
        sim.step(1)
        got = sim.get_populations()
    ref = oracle.step(p, f0, 1)
    near, of = _near_tie_sites(p, f0)
    differ = fields["hit"] != of["hit"]
    assert not (differ & ~near).any(), f"{int((differ & ~near).sum())} NCI decisions differ away from ties"
    rel = (np.abs(got - ref) / _scale(p, ref)).reshape(18, 96 * 48)
    ok = ~near
    assert (of["hit"][ok] > 0).sum() > 0 and rel[:, ok].max() <= FP32_TOL, rel[:, ok].max()


# ----------------------------------------------------------------------------- failure detection
@pytest.mark.parametrize("lat,prec", [(oracle.D2Q9, lbnci.LB_FP64), (oracle.D2Q9, lbnci.LB_FP32),
                                      (oracle.D2Q9, lbnci.LB_FP16DEV), (oracle.D3Q27, lbnci.LB_FP32),
                                      (oracle.D3Q27, lbnci.LB_FP16DEV)])
def test_injected_nan_and_negative_density(lat, prec):
    """Failure detection with the fault made on the host: lb_init_fields receives one NaN
    site and a 5-wide block (square or cube) of total density -1 inside a uniform mixture
    of density 1, and lb_observables must return LB_ENUMERIC with n_bad counted on the
    streamed state (the densities the next collision would see):
      * the NaN reaches every site that pulls from it: 9 sites (D2Q9), 27 (D3Q27);
      * inside the block every site pulls at least 5/6 of its weight from the block (a
        face site misses only the directions entering through that face, weight 1/6;
        edges and corners miss less than half), so all 25 (125) sites are negative,
        while a site outside pulls at most 1/6 of its weight from it and stays positive.
    The expected count is therefore 9 + 25 (27 + 125); lb_step then still runs."""
    D = 2 if lat == oracle.D2Q9 else 3
    n = 24 if D == 2 else 16
    nz = 1 if D == 2 else n
    shape = (nz, n, n)
    rho1 = np.full(shape, 0.5)
    rho2 = np.full(shape, 0.5)
    c = n // 2
    if D == 2:
        rho1[0, 3, 3] = np.nan
        rho1[0, c - 2:c + 3, c - 2:c + 3] = -0.5
        rho2[0, c - 2:c + 3, c - 2:c + 3] = -0.5
    else:
        rho1[3, 3, 3] = np.nan
        rho1[c - 2:c + 3, c - 2:c + 3, c - 2:c + 3] = -0.5
        rho2[c - 2:c + 3, c - 2:c + 3, c - 2:c + 3] = -0.5
    expected = (9 + 25) if D == 2 else (27 + 125)
    cfg = lbnci.lb_config_make(lattice=lat, nx=n, ny=n, nz=nz, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               precision=prec)
    with lbnci.Sim(cfg) as sim:
        sim.init_fields(rho1.ravel(), rho2.ravel())
        with pytest.raises(lbnci.LBError) as ei:
            sim.observables()
        assert ei.value.status == lbnci.LB_ENUMERIC
        obs = sim.observables(allow_numeric=True)
        assert obs["n_bad"] == expected, obs["n_bad"]
        sim.step(1)  # the library keeps working on a state with bad values
        assert sim.observables(allow_numeric=True)["n_bad"] > 0
    # the oracle's streamed densities agree with the hand count
    p = oracle.make_params(lattice=lat, nx=n, ny=n, nz=nz)
    of = oracle.fields(p, oracle.init(p, rho1.ravel(), rho2.ravel()))
    rho = of["rho1"] + of["rho2"]
    assert int((~(np.isfinite(rho) & (rho > 0))).sum()) == expected
