"""Warm start of packed-emulsion channels from the U-Net surrogate (lbnci_unet.h).

The lattice Boltzmann step (lbnci.h) is the method; the surrogate only proposes an
initial state. A channel starts either cold (its packed droplets at rest) or warm (the
same droplets with the velocity field the network predicts); the lattice Boltzmann run
then continues to the same horizon in both cases and decides: the time to steady state
is the first recorded step after which the flow rate stays within `tol` of the cold run's
converged flow rate.

Pipeline (every step of the network and of the flow runs in the library's kernels; this
module moves arrays and resamples images on the host):
  channels()   seeded channel configurations: width, length, area fraction, A_h, forcing
  run()        one batched ensemble of channels: flow-rate history and relaxed snapshots
  features()   5 input channels on the surrogate's H x W grid (mask, psi0, forcing, A_h,
               area fraction) and 3 targets (psi, u_x / u_P, u_y / u_P), u_P = G W^2/(8 rho nu)
  train()      Adam on the GPU through lbu_train_step
  predict()    the network's relaxed state, resampled back to each channel's lattice
  steps_to_steady() time-to-steady-state of a flow-rate history
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import inputs, lbnci, unet

TAU, A_S, BETA = 1.0, 0.01, 0.7
NU = (TAU - 0.5) / 3.0


@dataclass
class Channel:
    nx: int
    ny: int
    force: float
    A_h: float
    area_fraction: float
    u_p: float            # Poiseuille centre-line velocity G ny^2 / (8 rho nu)
    fields: inputs.Fields


def channels(n: int, seed: int, nx_range=(512, 1024), ny_range=(64, 96), af_range=(0.7, 0.9),
             ah_range=(0.0, 0.1), up_range=(2e-3, 2e-2)) -> list:
    """n seeded channels. The forcing is drawn as a log-uniform Poiseuille velocity scale
    u_P in up_range and set to G = 8 rho nu u_P / ny^2, which keeps the flow at low Mach
    number whatever the width (the body force of the ensemble study, log-uniform)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.integers(nx_range[0] // 32, nx_range[1] // 32 + 1)) * 32
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        af = float(rng.uniform(*af_range))
        ah = float(rng.uniform(*ah_range))
        up = float(math.exp(rng.uniform(math.log(up_range[0]), math.log(up_range[1]))))
        g = 8.0 * NU * up / ny ** 2
        fl = inputs.channel_emulsion_2d(nx, ny, seed=int(rng.integers(1 << 30)), area_fraction=af)
        out.append(Channel(nx, ny, g, ah, fl.meta["area_fraction"], up, fl))
    return out


def _config(c: Channel, stream=None, precision=lbnci.LB_FP32):
    return lbnci.lb_config_make(nx=c.nx, ny=c.ny, wall_y=1, tau=TAU, A_s=A_S, beta=BETA, A_h=c.A_h,
                                force=(c.force, 0.0, 0.0), precision=precision, stream=stream)


def run(chs, steps: int, every: int, u0=None, snap_from=None, snap_every=None, stream=None):
    """Advance all channels together (one batched launch per step) for `steps` steps.

    u0: optional list of initial velocity fields [3][N] (None = at rest).
    Returns (t [K], Q [n][K] flow rates, snapshots: list per channel of (psi, u) arrays
    taken at steps snap_from, snap_from + snap_every, ...)."""
    cfgs = [_config(c, stream) for c in chs]
    ens = lbnci.Ensemble(cfgs)
    try:
        for k, (mv, c) in enumerate(zip(ens.members, chs)):
            u = None if u0 is None or u0[k] is None else np.ascontiguousarray(u0[k], dtype=np.float64)
            mv.init_fields(c.fields.rho1, c.fields.rho2, u)
        ens.tune()
        ts, qs = [], []
        snaps = [[] for _ in chs]
        t = 0
        while True:
            if t % every == 0:
                ts.append(t)
                qs.append([mv.observables(allow_numeric=True)["flow_rate"] for mv in ens.members])
            if snap_from is not None and t >= snap_from and (t - snap_from) % snap_every == 0:
                for k, (mv, c) in enumerate(zip(ens.members, chs)):
                    psi = np.empty(c.nx * c.ny)
                    u = np.empty(3 * c.nx * c.ny)
                    mv.observables(psi_out=psi, u_out=u, allow_numeric=True)
                    snaps[k].append((psi.reshape(c.ny, c.nx), u.reshape(3, c.ny, c.nx)[:2]))
            if t >= steps:
                break
            n = min(every if snap_every is None else math.gcd(every, snap_every), steps - t)
            ens.step(n)
            t += n
        return np.asarray(ts), np.asarray(qs).T, snaps
    finally:
        ens.close()


# ------------------------------------------------------------------ resampling (host)
def _coords(n_src: int, n_dst: int) -> tuple:
    """Cell-centred linear interpolation weights from n_src cells to n_dst cells."""
    x = (np.arange(n_dst) + 0.5) * n_src / n_dst - 0.5
    i0 = np.floor(x).astype(np.int64)
    return i0, x - i0


def resample(img: np.ndarray, H: int, W: int) -> np.ndarray:
    """[ny, nx] -> [H, W]: linear in cell-centred coordinates, periodic in x, clamped in y."""
    ny, nx = img.shape
    j0, fy = _coords(ny, H)
    i0, fx = _coords(nx, W)
    j0c, j1c = np.clip(j0, 0, ny - 1), np.clip(j0 + 1, 0, ny - 1)
    i0w, i1w = i0 % nx, (i0 + 1) % nx
    rows = img[j0c] * (1 - fy)[:, None] + img[j1c] * fy[:, None]
    return rows[:, i0w] * (1 - fx)[None, :] + rows[:, i1w] * fx[None, :]


def features(c: Channel, H: int = 64, W: int = 256) -> np.ndarray:
    """Network input [H][W][5]: fluid mask, initial psi, forcing log10(u_P/0.01), A_h/0.1,
    area fraction. Every channel is resampled to fill the image, so the mask is 1."""
    psi0 = ((c.fields.rho1 - c.fields.rho2) / (c.fields.rho1 + c.fields.rho2)).reshape(c.ny, c.nx)
    x = np.empty((H, W, 5), dtype=np.float32)
    x[..., 0] = 1.0
    x[..., 1] = resample(psi0, H, W)
    x[..., 2] = math.log10(c.u_p / 0.01)
    x[..., 3] = c.A_h / 0.1
    x[..., 4] = c.area_fraction
    return x


def targets(c: Channel, psi: np.ndarray, u: np.ndarray, H: int = 64, W: int = 256) -> np.ndarray:
    t = np.empty((H, W, 3), dtype=np.float32)
    t[..., 0] = resample(psi, H, W)
    t[..., 1] = resample(u[0], H, W) / c.u_p
    t[..., 2] = resample(u[1], H, W) / c.u_p
    return t


# ------------------------------------------------------------------ the surrogate
def train(net: unet.Net, X, T, epochs: int, batch: int, lr: float, seed: int = 0, lam=None, log=None):
    """Adam over shuffled mini-batches of the device arrays X [n][H][W][5], T [n][H][W][3]
    (CUDA tensors); the shuffling indices are the only host work. Returns loss history."""
    import torch
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    steps_per_epoch = max(1, n // batch)
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n).astype(np.int32), device=X.device)
        torch.cuda.synchronize()  # the indices are read by kernels on the network's stream
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))  # cosine schedule
        last = None
        for s in range(steps_per_epoch):
            want = s == steps_per_epoch - 1
            last = net.train_step(X, T, idx=perm[s * batch:(s + 1) * batch], batch=batch, lam=lam, lr=lr_ep,
                                  want_loss=want)
        hist.append(last)
        if log:
            log(f"epoch {ep}: loss {last:.5f} lr {lr_ep:.2e}")
    return hist


def predict(net: unet.Net, chs, H: int = 64, W: int = 256):
    """Predicted relaxed (psi, u_x, u_y) of each channel on its own lattice."""
    out = []
    B = net.cfg.max_batch
    feats = np.stack([features(c, H, W) for c in chs])
    ys = np.concatenate([net.forward(feats[i:i + B]) for i in range(0, len(chs), B)])
    for c, y in zip(chs, ys):
        psi = resample(y[..., 0].astype(np.float64), c.ny, c.nx)
        ux = resample(y[..., 1].astype(np.float64), c.ny, c.nx) * c.u_p
        uy = resample(y[..., 2].astype(np.float64), c.ny, c.nx) * c.u_p
        out.append((psi, ux, uy))
    return out


def windowed(q: np.ndarray, w: int) -> np.ndarray:
    """Trailing mean of a flow-rate history over w records (shorter at the start)."""
    c = np.cumsum(np.insert(np.asarray(q, dtype=np.float64), 0, 0.0))
    i = np.arange(1, len(q) + 1)
    lo = np.maximum(i - w, 0)
    return (c[i] - c[lo]) / (i - lo)


def steps_to_steady(t: np.ndarray, q: np.ndarray, q_ss: float, tol: float = 0.01) -> float:
    """First recorded step after which |Q - q_ss| <= tol |q_ss| holds for every later record
    (inf if the last record is outside the band)."""
    ok = np.abs(q - q_ss) <= tol * abs(q_ss)
    if not ok[-1]:
        return math.inf
    bad = np.nonzero(~ok)[0]
    return float(t[0] if len(bad) == 0 else t[min(bad[-1] + 1, len(t) - 1)])


def convergence(t: np.ndarray, q: np.ndarray, tol: float, window: int) -> dict:
    """A run judged on its own: plateau = mean flow rate over the last quarter of the
    history; time to steady state = the first step after which the windowed flow rate
    stays within tol of the plateau; the run is steady when that happens before the last
    quarter begins."""
    K = len(q)
    plateau = float(np.mean(q[int(0.75 * K):]))
    if not np.all(np.isfinite(q)):
        return {"plateau": plateau, "steady": False, "t_ss": math.inf}
    t_ss = steps_to_steady(t, windowed(q, window), plateau, tol)
    return {"plateau": plateau, "steady": bool(t_ss <= t[int(0.75 * K)]), "t_ss": t_ss}


def _param_shapes(cfg):
    return [("", (co, kh, kw, ci) if kh == 3 else (co, ci)) for co, kh, kw, ci in unet.layer_shapes(cfg)]


def experiment(train_chs, test_chs, steps=60000, every=200, snap_from=44000, snap_every=2000, epochs=30,
               batch=32, lr=1e-3, tol=0.01, window=10, lam=(0.2, 1.0, 1.0), seed=0, stream=None, log=print,
               ensemble_size=96):
    """Generate snapshots with the lattice Boltzmann ensemble, train the surrogate on the
    GPU, then run the held-out channels three times to the same horizon: cold (droplets at
    rest), cold with a velocity perturbation of 1e-4 u_P (a control: packed emulsions are
    path dependent, so two cold starts may settle on plateaus that differ), and warm (the
    predicted velocity field).

    Returns a dict of per-channel and summary results (steps to steady state, plateaus,
    prediction errors, training history and times)."""
    import time

    import torch
    res = {"train_channels": len(train_chs), "test_channels": len(test_chs), "steps": steps, "tol": tol,
           "window_steps": window * every}
    t0 = time.time()
    X, T, dropped = [], [], 0
    for i in range(0, len(train_chs), ensemble_size):
        chunk = train_chs[i:i + ensemble_size]
        _, Q, snaps = run(chunk, steps, every, snap_from=snap_from, snap_every=snap_every, stream=stream)
        for c, q, sn in zip(chunk, Q, snaps):
            if not np.all(np.isfinite(q)) or not sn:
                dropped += 1
                continue
            f = features(c)
            for psi, u in sn:
                X.append(f)
                T.append(targets(c, psi, u))
        log(f"data: {len(X)} snapshots after {i + len(chunk)} channels ({time.time() - t0:.1f} s)")
    res.update(snapshots=len(X), dropped_unstable=dropped, data_seconds=time.time() - t0)
    Xd = torch.tensor(np.stack(X), device="cuda")
    Td = torch.tensor(np.stack(T), device="cuda")
    del X, T
    cfg = unet.make_config(max_batch=batch, stream=stream)
    net = unet.Net(cfg)
    try:
        net.set_params(unet.flatten(inputs.unet_params(_param_shapes(cfg), seed)))
        torch.cuda.synchronize()
        t1 = time.time()
        hist = train(net, Xd, Td, epochs, batch, lr, seed=seed, lam=list(lam), log=log)
        torch.cuda.synchronize()
        res.update(train_seconds=time.time() - t1, loss_history=hist,
                   train_steps=epochs * max(1, Xd.shape[0] // batch), train_launches=net.launches())
        del Xd, Td
        pred = predict(net, test_chs)
    finally:
        net.close()
    t2 = time.time()
    rng = np.random.default_rng(seed + 7)
    tc, Qc, sc = run(test_chs, steps, every, snap_from=steps, snap_every=every, stream=stream)
    u_pert = [np.stack([1e-4 * c.u_p * rng.standard_normal(c.nx * c.ny), np.zeros(c.nx * c.ny),
                        np.zeros(c.nx * c.ny)]) for c in test_chs]
    tp, Qp, _ = run(test_chs, steps, every, u0=u_pert, stream=stream)
    u0 = [np.stack([ux.ravel(), uy.ravel(), np.zeros(ux.size)]) for _, ux, uy in pred]
    tw, Qw, _ = run(test_chs, steps, every, u0=u0, stream=stream)
    res["lb_seconds_test"] = time.time() - t2
    rows = []
    for k, c in enumerate(test_chs):
        cc, cp, cw = (convergence(tc, Qc[k], tol, window), convergence(tp, Qp[k], tol, window),
                      convergence(tw, Qw[k], tol, window))
        psi_f, u_f = sc[k][-1]
        psi_p, ux_p, _ = pred[k]
        q_pred = float(ux_p.sum() / c.nx)  # flow rate of the predicted field (rho = 1)
        ref = cc["plateau"]
        rows.append({
            "channel": k, "nx": c.nx, "ny": c.ny, "A_h": c.A_h, "u_p": c.u_p, "af": c.area_fraction,
            "cold": cc, "cold_perturbed": cp, "warm": cw,
            "spread_cold_perturbed": abs(cp["plateau"] - ref) / abs(ref),
            "spread_warm": abs(cw["plateau"] - ref) / abs(ref),
            "pred_q_rel_err": abs(q_pred - ref) / abs(ref),
            "pred_psi_l2": float(np.linalg.norm(psi_p - psi_f) / np.linalg.norm(psi_f)),
            "pred_u_l2": float(np.linalg.norm(ux_p - u_f[0]) / np.linalg.norm(u_f[0]))})
    res["channels"] = rows
    steady = [r for r in rows if r["cold"]["steady"] and r["warm"]["steady"] and r["cold_perturbed"]["steady"]]
    sp = [r["cold"]["t_ss"] / max(r["warm"]["t_ss"], every) for r in steady]
    spc = [r["cold"]["t_ss"] / max(r["cold_perturbed"]["t_ss"], every) for r in steady]
    med = lambda v: float(np.median(v)) if len(v) else None  # noqa: E731
    res["summary"] = {
        "steady_channels": len(steady), "steady_cold": sum(r["cold"]["steady"] for r in rows),
        "steady_warm": sum(r["warm"]["steady"] for r in rows),
        "median_speedup_warm": med(sp), "median_speedup_control": med(spc),
        "mean_t_cold": med([r["cold"]["t_ss"] for r in steady]) and float(np.mean([r["cold"]["t_ss"] for r in steady])),
        "mean_t_warm": med([r["warm"]["t_ss"] for r in steady]) and float(np.mean([r["warm"]["t_ss"] for r in steady])),
        "median_spread_warm": med([r["spread_warm"] for r in steady]),
        "median_spread_control": med([r["spread_cold_perturbed"] for r in steady]),
        "frac_warm_within_tol": (float(np.mean([r["spread_warm"] <= tol for r in steady])) if steady else None),
        "frac_control_within_tol": (float(np.mean([r["spread_cold_perturbed"] <= tol for r in steady]))
                                    if steady else None),
        "median_pred_q_rel_err": med([r["pred_q_rel_err"] for r in rows]),
    }
    return res
