"""lb_observables_noalloc: the same observables as lb_observables, computed with no
allocation inside the library (for callers that cannot let it allocate: applications
whose device memory belongs to their own pool, loops that must not risk the
synchronisation a cudaMalloc can cause).

Called through the C ABI on device populations the test owns, twice in a row (the
static scratch keeps the previous call's contents, which must not leak into the next
result), and compared with lb_observables of a sim holding the same state. This file
is collected last on purpose, and runs as well on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2003_11069_gb300 import inputs, lbnci

pytestmark = pytest.mark.gpu


def _close(a, b, scale_mom):
    assert np.allclose(a["mass"], b["mass"], rtol=1e-13, atol=0)
    assert np.max(np.abs(a["momentum"] - b["momentum"])) <= 1e-13 * scale_mom
    assert abs(a["flow_rate"] - b["flow_rate"]) <= 1e-13 * scale_mom
    assert abs(a["flow_rate_disp"] - b["flow_rate_disp"]) <= 1e-13 * scale_mom
    for k in ("n_interface", "n_nci", "n_bad"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("precision", [lbnci.LB_FP64, lbnci.LB_FP32])
def test_noalloc_matches_lb_observables_twice(precision):
    torch = pytest.importorskip("torch")
    nx, ny = 160, 64
    cfg = lbnci.lb_config_make(nx=nx, ny=ny, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                               force=(1e-5, 0.0, 0.0), precision=precision)
    fl = inputs.channel_emulsion_2d(nx, ny, seed=21, r_lo=10, r_hi=13)
    dtype = torch.float64 if precision == lbnci.LB_FP64 else torch.float32
    with lbnci.Sim(cfg) as sim:
        sim.init_fields(fl.rho1, fl.rho2)
        for steps in (25, 40):  # two different states, one call pair each
            sim.step(steps)
            ref = sim.observables()
            f64 = torch.empty(2 * 9 * nx * ny, dtype=torch.float64, device="cuda")
            lbnci.lb_get_populations(sim.h, f64)
            f = f64.to(dtype).contiguous()
            torch.cuda.synchronize()
            first = lbnci.lb_observables_noalloc(cfg, f)
            second = lbnci.lb_observables_noalloc(cfg, f)
            scale = float(np.abs(ref["momentum"]).sum() + abs(ref["flow_rate"])) + 1e-300
            if precision == lbnci.LB_FP64:
                _close(first, ref, scale)
                _close(second, ref, scale)
            else:
                # FP32: the same kernels on the same float state give the same sums
                _close(first, ref, scale)
            for k in ("mass", "momentum"):
                assert np.array_equal(first[k], second[k])
            assert first["n_nci"] > 0 and first["step"] == 0


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    cfg = lbnci.lb_config_make(nx=4096, ny=1024, precision=lbnci.LB_FP64)
    f = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(lbnci.LBError) as ei:
        lbnci.lb_observables_noalloc(cfg, f)
    assert ei.value.status == lbnci.LB_EINVAL
    assert "scratch" in lbnci.lb_last_error(None)
