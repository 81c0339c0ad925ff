"""Ensembles of uneven D2Q9 channels stepped by one batched launch per step (CUDA graph):
every member must evolve exactly as the same lattice stepped alone, in every precision,
whatever the number of steps (graph replays plus a single step) and the tile shape the
autotuner picks; and, in FP64, as the oracle. The member sizes mix lattices that run the
batched TMA kernel (FP32 and FP16-dev with nx % 4 == 0) with lattices that run the one-pass
batch kernel (nx % 4 != 0), and NCI on with NCI off."""
import numpy as np
import pytest

import oracle
from paper_2003_11069_gb300 import inputs, lbnci

pytestmark = pytest.mark.gpu

SIZES = [(64, 24, 1, 1.0, 0.05, 2e-5), (37, 19, 1, 0.8, 0.1, 1e-5), (96, 40, 0, 0.9, 0.0, 3e-5),
         (32, 16, 1, 1.0, 0.03, 1e-4), (130, 33, 1, 0.7, 0.07, 5e-6)]


def _cfgs(precision, forcing=lbnci.LB_FORCE_GUO):
    cfgs, fields = [], []
    for k, (nx, ny, wall, tau, ah, g) in enumerate(SIZES):
        cfgs.append(lbnci.lb_config_make(nx=nx, ny=ny, wall_y=wall, tau=tau, A_s=0.01, beta=0.7, A_h=ah,
                                         force=(g, 0.0, 0.0), precision=precision, forcing=forcing))
        fields.append(inputs.channel_emulsion_2d(nx, ny, seed=100 + k, r_lo=5, r_hi=7, film=0.5))
    return cfgs, fields


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbnci.load()


@pytest.mark.parametrize("precision,forcing", [(lbnci.LB_FP64, 0), (lbnci.LB_FP32, 0), (lbnci.LB_FP16DEV, 0),
                                               (lbnci.LB_FP64, 1), (lbnci.LB_FP32, 1), (lbnci.LB_FP16DEV, 1)])
def test_members_match_standalone(precision, forcing):
    cfgs, fields = _cfgs(precision, forcing)
    with lbnci.Ensemble(cfgs) as ens:
        for m, fl in zip(ens.members, fields):
            m.init_fields(fl.rho1, fl.rho2)
        ens.step(7)  # one single step back to the graph's parity, three graph replays
        ens.step(4)
        got = [m.get_populations() for m in ens.members]
        obs = [m.observables() for m in ens.members]
        assert ens.launches() >= 11
        with pytest.raises(lbnci.LBError):
            ens.members[0].step(1)  # members are stepped by their ensemble only
    for k, (c, fl) in enumerate(zip(cfgs, fields)):
        with lbnci.Sim(c) as sim:
            sim.init_fields(fl.rho1, fl.rho2)
            sim.step(11)
            ref = sim.get_populations()
            assert np.array_equal(got[k], ref), f"member {k}"
            assert obs[k]["step"] == 11


def test_fp64_member_matches_oracle():
    cfgs, fields = _cfgs(lbnci.LB_FP64)
    with lbnci.Ensemble(cfgs) as ens:
        for m, fl in zip(ens.members, fields):
            m.init_fields(fl.rho1, fl.rho2)
        ens.step(20)
        got = [m.get_populations() for m in ens.members]
    for k, (nx, ny, wall, tau, ah, g) in enumerate(SIZES):
        p = oracle.make_params(nx=nx, ny=ny, wall_y=wall, tau=tau, A_s=0.01, beta=0.7, A_h=ah, force=(g, 0, 0))
        ref = oracle.step(p, oracle.init(p, fields[k].rho1, fields[k].rho2), 20)
        _, w, _ = oracle.lattice(0)
        scale = np.maximum(np.abs(ref), np.tile(np.repeat(w, nx * ny), 2))
        assert np.max(np.abs(got[k] - ref) / scale) <= 1e-12, f"member {k}"


def test_autotune_keeps_state_and_results():
    cfgs, fields = _cfgs(lbnci.LB_FP32)
    with lbnci.Ensemble(cfgs) as ens:
        for m, fl in zip(ens.members, fields):
            m.init_fields(fl.rho1, fl.rho2)
        ens.step(3)
        before = [m.get_populations() for m in ens.members]
        assert ens.tma_choice()[:2] == (128, 2) and ens.tma_choice()[2] == {}
        spt = ens.tune()
        assert spt in (2, 4)
        t2, t4 = ens.tune_times()
        assert t2 > 0 and t4 > 0
        promo, nstatic, table = ens.tma_choice()
        assert promo in (0, 64, 128, 256) and nstatic in (1, 2, 3)
        assert len(table) == 12 and all(v > 0 for v in table.values())
        assert table[(promo, nstatic)] == min(table.values())
        after = [m.get_populations() for m in ens.members]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)  # tuning wrote only the back buffers
        ens.step(5)
        got = [m.get_populations() for m in ens.members]
    for k, (c, fl) in enumerate(zip(cfgs, fields)):
        with lbnci.Sim(c) as sim:
            sim.init_fields(fl.rho1, fl.rho2)
            sim.step(8)
            assert np.array_equal(got[k], sim.get_populations()), f"member {k}"


@pytest.mark.parametrize("choice", ["0:1", "64:3", "256:2"])
def test_tma_candidates_give_identical_results(monkeypatch, choice):
    """Every (L2 promotion, static tiles) candidate the autotuner may pick steps the
    members exactly as the lattices stepped alone: the choice moves tiles between CTAs
    and changes cache hints, never the arithmetic of a site."""
    monkeypatch.setenv("LBNCI_TMA_CHOICE", choice)
    cfgs, fields = _cfgs(lbnci.LB_FP16DEV)
    with lbnci.Ensemble(cfgs) as ens:
        pr, st, _ = ens.tma_choice()
        assert f"{pr}:{st}" == choice
        for m, fl in zip(ens.members, fields):
            m.init_fields(fl.rho1, fl.rho2)
        ens.step(6)
        got = [m.get_populations() for m in ens.members]
    monkeypatch.delenv("LBNCI_TMA_CHOICE")
    for k, (c, fl) in enumerate(zip(cfgs, fields)):
        with lbnci.Sim(c) as sim:
            sim.init_fields(fl.rho1, fl.rho2)
            sim.step(6)
            assert np.array_equal(got[k], sim.get_populations()), f"member {k}"


def test_tma_choice_env_is_validated(monkeypatch):
    monkeypatch.setenv("LBNCI_TMA_CHOICE", "96:2")
    cfgs, _ = _cfgs(lbnci.LB_FP32)
    with pytest.raises(lbnci.LBError):
        lbnci.Ensemble(cfgs)


def test_tma_choice_needs_a_tma_member():
    cfgs, _ = _cfgs(lbnci.LB_FP64)
    with lbnci.Ensemble(cfgs) as ens:
        with pytest.raises(lbnci.LBError):
            ens.tma_choice()


def test_flow_rate_grows_with_forcing():
    """Sanity trend of the paper's flow-rate study (not a parity pin): identical channels
    driven harder carry more of both phases after the same time."""
    fl = inputs.channel_emulsion_2d(256, 64, seed=7, r_lo=10, r_hi=13)
    forces = [2e-6, 1e-5, 5e-5]
    cfgs = [lbnci.lb_config_make(nx=256, ny=64, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                                 force=(g, 0, 0), precision=lbnci.LB_FP32) for g in forces]
    with lbnci.Ensemble(cfgs) as ens:
        for m in ens.members:
            m.init_fields(fl.rho1, fl.rho2)
        ens.step(400)
        q = [m.observables()["flow_rate_disp"] for m in ens.members]
    assert q[0] < q[1] < q[2] and q[0] > 0
