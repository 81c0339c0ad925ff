"""The U-Net warm start against the method without it (cold starts), end to end on the GPU.

Small, deterministic version of the bench's warm-start study: 96 training channels
(width 64-72, length 512, A_h <= 0.002, Poiseuille velocity 5e-3..1.5e-2) run 30k steps by
the batched lattice Boltzmann ensemble; snapshots after 22k steps train the network with
the library's own BF16 kernels; 16 held-out channels then run cold, cold with a 1e-4 u_P
velocity perturbation (the control) and warm from the network's prediction. In this
regime the flow reaches a 1% steady state by viscous development (t ~ 4.6 W^2/(pi^2 nu)
~ 12k steps), which a good initial velocity field shortens.
"""
import math

import numpy as np
import pytest

from paper_2003_11069_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_warm_start_reaches_steady_state_sooner_at_equal_flow_rate():
    kw = dict(nx_range=(512, 512), ny_range=(64, 72), ah_range=(0.0, 0.002), up_range=(5e-3, 1.5e-2))
    train = ws.channels(96, seed=11, **kw)
    test = ws.channels(16, seed=12, **kw)
    stream = torch.cuda.Stream()
    res = ws.experiment(train, test, steps=30000, every=200, snap_from=22000, snap_every=2000, epochs=15,
                        batch=32, lr=1e-3, stream=stream.cuda_stream, log=print)
    s = res["summary"]
    print(s)
    rows = [r for r in res["channels"] if r["cold"]["steady"] and r["warm"]["steady"]]
    for r in res["channels"]:
        print(r["channel"], r["cold"], r["warm"], r["spread_warm"], r["pred_q_rel_err"])
    assert res["dropped_unstable"] == 0
    assert s["steady_cold"] >= 12
    # the network's own flow-rate estimate is already close
    assert s["median_pred_q_rel_err"] < 0.1
    # warm starts reach their plateau sooner ...
    speed = [r["cold"]["t_ss"] / max(r["warm"]["t_ss"], 200) for r in rows]
    assert np.median(speed) > 1.2, speed
    # ... and the plateau they reach is the cold start's, to the 1% tolerance
    assert np.mean([r["spread_warm"] <= 0.01 for r in rows]) >= 0.75
    assert all(math.isfinite(r["cold"]["plateau"]) for r in res["channels"])
