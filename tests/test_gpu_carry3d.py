"""The single-read D3Q27 step (LB_PATH_D3Q27_CARRY, selected with LBNCI_D3_KERNEL=carry) against
the FP64 oracle.

The step's colour gradient uses densities that the previous step's collision carried
forward (each new population summed into the density of the site it streams to, across
column boundaries through exported rings), so a step is checked both from a state the
library was handed (densities pulled afresh) and from states the library produced itself
(densities carried, the case every step after the first is in). Each step starts from
the GPU's own state and is compared with one oracle step from that state: populations
within the per-step tolerance of the storage at every site whose NCI decision is not at
a floating-point near-tie (judged on the oracle's FP64 fields), and no decision differs
away from one. Lattices: several columns of 32 x 8 sites, walls in y and z, periodic y,
periodic z, one column only (its rings wrap onto itself), the exact difference method.
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


def _duct(nx, ny, nz, seed):
    return inputs.duct_emulsion_3d(nx, ny, nz, seed=seed, radius=5.0, volume_fraction=0.5)


def _check_step(p, f_start, got, precision, what, form=lbnci.LB_STATE_PAIRS):
    ref = oracle.step(p, f_start, 1)
    near, of = _near_tie_sites(p, f_start)
    err = step_error(p, got, ref, precision, form)
    ok = ~near
    assert (of["hit"][ok] > 0).sum() > 0, f"{what}: NCI must be active"
    bad = err[:, ok].max(axis=0) > 1.0
    assert not bad.any(), (f"{what}: {int(bad.sum())} sites beyond the per-step bound (max {err[:, ok].max():.3f}); "
                           f"first at site {int(np.flatnonzero(ok)[np.argmax(bad)])}")
    return float(err[:, ok].max())


CASES = {
    "walls_yz": dict(nx=64, ny=24, nz=12, wall_y=1, wall_z=1),
    "periodic_y": dict(nx=64, ny=24, nz=12, wall_y=0, wall_z=1),
    "periodic_yz": dict(nx=64, ny=16, nz=10, wall_y=0, wall_z=0),
    "one_column": dict(nx=32, ny=8, nz=10, wall_y=0, wall_z=0),
}


@pytest.mark.parametrize("zseg", ["16", "5"])
@pytest.mark.parametrize("precision", [lbnci.LB_FP32, lbnci.LB_FP16DEV])
@pytest.mark.parametrize("name", list(CASES))
def test_carry3d_steps_match_oracle(name, precision, zseg, monkeypatch):
    """zseg: planes per z segment of the collision kernel (16: one segment on these
    lattices; 5: two or three, the last one shorter, so the densities also cross segment
    boundaries through the ghost planes, periodic ones included)."""
    monkeypatch.setenv("LBNCI_C3_ZSEG", zseg)
    monkeypatch.setenv("LBNCI_D3_KERNEL", "carry")  # the streaming step is the default
    geo = CASES[name]
    p = oracle.make_params(lattice=oracle.D3Q27, tau=0.9, A_s=0.01, beta=0.7, A_h=0.03, force=(2e-6, 1e-6, 0),
                           **geo)
    fl = _duct(geo["nx"], geo["ny"], geo["nz"], seed=13)
    f0 = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 20)
    with lbnci.Sim(_cfg(p, precision)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_D3Q27_CARRY
        sim.set_populations(f0)
        start = sim.get_populations()  # the representable state (FP32 or FP16 deviations)
        for k in range(4):  # step 0 from freshly pulled densities, then from carried ones
            sim.step(1)
            got = sim.get_populations()
            err = _check_step(p, start, got, precision, f"{name} step {k}")
            print(f"{name} precision {precision} step {k}: max error {err:.3f} of the per-step bound")
            start = got
        obs = sim.observables()
        assert obs["n_bad"] == 0


def test_carry3d_edm_dispersed(monkeypatch):
    monkeypatch.setenv("LBNCI_C3_ZSEG", "4")
    monkeypatch.setenv("LBNCI_D3_KERNEL", "carry")
    p = oracle.make_params(lattice=oracle.D3Q27, nx=64, ny=24, nz=12, wall_y=1, wall_z=1, tau=0.9, A_s=0.01,
                           beta=0.7, A_h=0.03, force=(2e-6, 0, 1e-6), forcing=1)
    fl = _duct(64, 24, 12, seed=13)
    f0 = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 20).astype(np.float32).astype(np.float64)
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as sim:
        assert sim.step_path() == lbnci.LB_PATH_D3Q27_CARRY
        sim.set_populations(f0)
        start = f0
        for k in range(3):
            sim.step(1)
            got = sim.get_populations()
            _check_step(p, start, got, lbnci.LB_FP32, f"edm step {k}")
            start = got


def test_carry3d_chained_equals_separate_and_march_path(monkeypatch):
    """lb_step(4) equals four lb_step(1) calls bitwise (the carried densities persist
    between calls), and the result stays within the per-step tolerance of the two-pass
    step over the same four steps."""
    p = oracle.make_params(lattice=oracle.D3Q27, nx=64, ny=24, nz=12, wall_y=1, wall_z=1, tau=1.0, A_s=0.01,
                           beta=0.7, A_h=0.03, force=(2e-6, 0, 0))
    fl = _duct(64, 24, 12, seed=21)
    cfg = _cfg(p, lbnci.LB_FP32)
    monkeypatch.setenv("LBNCI_D3_KERNEL", "carry")
    with lbnci.Sim(cfg) as a, lbnci.Sim(cfg) as b:
        assert a.step_path() == lbnci.LB_PATH_D3Q27_CARRY
        a.init_fields(fl.rho1, fl.rho2)
        b.init_fields(fl.rho1, fl.rho2)
        a.step(4)
        for _ in range(4):
            b.step(1)
        fa, fb = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb)
    monkeypatch.setenv("LBNCI_D3_KERNEL", "march")
    with lbnci.Sim(_cfg(p, lbnci.LB_FP32)) as c:
        assert c.step_path() == lbnci.LB_PATH_D3Q27
        c.init_fields(fl.rho1, fl.rho2)
        c.step(4)
        fc = c.get_populations()
    rel = np.abs(fa - fc) / _scale(p, fc)
    # four steps of FP32 rounding differences (and possibly near-tie NCI decisions)
    assert np.quantile(rel, 0.9999) <= 4 * FP32_TOL, np.quantile(rel, 0.9999)
