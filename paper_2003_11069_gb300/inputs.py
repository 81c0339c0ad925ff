"""Seeded synthetic input fields for the colour-gradient NCI lattice Boltzmann runs.

This module builds initial component-density fields (rho1, rho2) only. It holds none
of the method's arithmetic (no equilibria, no streaming, no collision): the same arrays
are handed to the CUDA library and to the CPU oracle, each of which builds its own
populations from them.

Fields are flat float64 arrays in site order idx = x + nx*(y + ny*z). The order
parameter of the initial state is a tanh profile psi0 = tanh((R - r)/w) around each
droplet (psi0 = +1 inside, -1 outside); rho1 = rho0 (1 + psi0)/2, rho2 = rho0 (1 - psi0)/2.
Where droplets overlap, the larger psi0 wins.

Workload shapes follow the paper's soft-flowing-crystal studies: packed droplets of
the dispersed phase (component 1) in a channel or square duct bounded by walls,
with thin films of the continuous phase between neighbours (arXiv:2003.11069,
Results, Figs. 2-3; the geometry of the paper's device is not given, so these are
synthetic stand-ins).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Fields:
    nx: int
    ny: int
    nz: int
    rho1: np.ndarray
    rho2: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def _to_rho(psi0: np.ndarray, rho0: float = 1.0):
    psi0 = np.clip(psi0, -1.0, 1.0)
    return (rho0 * 0.5 * (1.0 + psi0)).ravel().copy(), (rho0 * 0.5 * (1.0 - psi0)).ravel().copy()


def _paint(psi: np.ndarray, centers, radii, width: float, periodic_axes, pad: float = 5.0):
    """psi = max(psi, tanh((R - r)/w)) in a box around each droplet.

    psi has shape (nz, ny, nx) (nz = 1 in 2D); centers are (x, y, z)."""
    nz, ny, nx = psi.shape
    dims = (nx, ny, nz)
    for c, R in zip(centers, radii):
        ext = R + pad * width
        rng_ax = []
        for a in range(3):
            if dims[a] == 1:
                rng_ax.append((np.zeros(1, dtype=np.int64), np.zeros(1)))
                continue
            lo = int(math.floor(c[a] - ext))
            hi = int(math.ceil(c[a] + ext))
            idx = np.arange(lo, hi + 1)
            d = idx - c[a]
            if periodic_axes[a]:
                idx = np.mod(idx, dims[a])
            else:
                keep = (idx >= 0) & (idx < dims[a])
                idx, d = idx[keep], d[keep]
            rng_ax.append((idx, d))
        (ix, dx), (iy, dy), (iz, dz) = rng_ax
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        val = np.tanh((R - r) / width)
        sub = psi[np.ix_(iz, iy, ix)]
        psi[np.ix_(iz, iy, ix)] = np.maximum(sub, val)
    return psi


def droplet(nx: int, ny: int, nz: int = 1, radius: float = 30.0, width: float = 2.0,
            center=None, rho0: float = 1.0) -> Fields:
    """One droplet of the dispersed phase in a periodic box (2D when nz == 1)."""
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0 if nz > 1 else 0.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    psi = np.tanh((radius - r) / width)
    r1, r2 = _to_rho(psi, rho0)
    return Fields(nx, ny, nz, r1, r2, {"kind": "droplet", "radius": radius, "width": width})


def uniform(nx: int, ny: int, nz: int = 1, psi0: float = -1.0, rho0: float = 1.0) -> Fields:
    """Uniform state (psi0 = -1: pure continuous phase, single-phase flow)."""
    psi = np.full((nz, ny, nx), psi0)
    r1, r2 = _to_rho(psi, rho0)
    return Fields(nx, ny, nz, r1, r2, {"kind": "uniform", "psi0": psi0})


def slabs(nx: int, ny: int, bands, width: float = 2.0, nz: int = 1, rho0: float = 1.0) -> Fields:
    """Planar films of the dispersed phase: psi0 = +1 for y in each [y_lo, y_hi] band,
    with tanh edges of the given width (y periodic)."""
    y = np.arange(ny, dtype=np.float64)
    prof = -np.ones(ny)
    for lo, hi in bands:
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        for shift in (-ny, 0, ny):
            d = np.abs(y - mid - shift)
            prof = np.maximum(prof, np.tanh((half - d) / width))
    psi = np.broadcast_to(prof[None, :, None], (nz, ny, nx)).copy()
    r1, r2 = _to_rho(psi, rho0)
    return Fields(nx, ny, nz, r1, r2, {"kind": "slabs", "bands": list(bands)})


def _pair_distances(centers: np.ndarray, dims, periodic) -> np.ndarray:
    """Distances between all pairs of centres (minimum image along periodic axes)."""
    d = centers[:, None, :] - centers[None, :, :]
    for ax in range(len(dims)):
        if periodic[ax] and dims[ax] > 1:
            d[:, :, ax] -= dims[ax] * np.round(d[:, :, ax] / dims[ax])
    dist = np.sqrt((d ** 2).sum(axis=-1))
    np.fill_diagonal(dist, np.inf)
    return dist


def _clip_radii(centers: np.ndarray, radii: np.ndarray, dims, periodic, film: float,
                iters: int = 60) -> np.ndarray:
    """Shrink radii until every pair of droplets keeps a film of at least `film`:
    r_a + r_b + film <= |c_a - c_b|. A violating pair is scaled down together (their
    ratio kept), so a small droplet may sit next to a large one."""
    out = radii.astype(np.float64).copy()
    # only pairs that can ever touch matter: neighbours within twice the largest radius
    dist = _pair_distances(centers, dims, periodic)
    near = dist < 2.0 * out.max() + film + 1e-9
    ia, ib = np.nonzero(np.triu(near, 1))
    dab = dist[ia, ib]
    for _ in range(iters):
        s = out[ia] + out[ib] + film
        viol = s > dab
        if not viol.any():
            break
        scale = (dab[viol] - film) / (out[ia[viol]] + out[ib[viol]])
        f = np.ones(len(out))
        np.minimum.at(f, ia[viol], scale)
        np.minimum.at(f, ib[viol], scale)
        out *= f
    assert np.all(out[ia] + out[ib] + film <= dab + 1e-9), "film constraint not met"
    return out


def channel_emulsion_2d(nx: int, ny: int, seed: int, r_lo: float = 12.0, r_hi: float = 16.0,
                        area_fraction: float = 0.8, jitter: float = 1.0, width: float = 2.0,
                        film: float = 1.0, rho0: float = 1.0, spacing_factor: float = 0.97) -> Fields:
    """Packed 2D emulsion in a channel with walls below y=0 and above y=ny-1, periodic in x.

    Droplet radii are uniform in [r_lo, r_hi]; centres sit on a hexagonal lattice whose
    spacing holds the requested area fraction at the mean squared radius (times
    spacing_factor), with uniform +-jitter. Rows fill the channel height. Every pair of
    droplets keeps a film >= `film` (a violating pair is shrunk together) and every
    droplet stays `film` from the walls, so the near-contact force, not merging,
    separates them. With radii in 12-16, +-1 jitter and a film of 1 the hexagonal rows
    reach an area fraction of about 0.73 (spacing_factor 0.97 is where it peaks): 0.8
    needs equal radii of about 13.6 at this spacing."""
    rng = np.random.default_rng(seed)
    r2 = (r_lo * r_lo + r_lo * r_hi + r_hi * r_hi) / 3.0  # mean of r^2 over U[r_lo, r_hi]
    a = math.sqrt(2.0 * math.pi * r2 / (math.sqrt(3.0) * area_fraction)) * spacing_factor
    ncol = max(1, int(round(nx / a)))
    ax = nx / ncol
    dy = ax * math.sqrt(3.0) / 2.0
    y0 = r_lo + 0.5
    nrow = max(1, int(math.floor((ny - 1 - 2 * y0) / dy)) + 1)
    ytop = y0 + (nrow - 1) * dy
    yshift = 0.5 * ((ny - 1) - ytop - y0)
    centers = []
    for r in range(nrow):
        for c in range(ncol):
            centers.append([(c + 0.5 * (r % 2)) * ax, y0 + yshift + r * dy, 0.0])
    centers = np.asarray(centers, dtype=np.float64)
    centers[:, :2] += rng.uniform(-jitter, jitter, size=(len(centers), 2))
    radii = rng.uniform(r_lo, r_hi, size=len(centers))
    # keep each droplet a film away from the walls (wall planes at y = -1/2, ny - 1/2)
    radii = np.minimum(radii, np.minimum(centers[:, 1] + 0.5, ny - 0.5 - centers[:, 1]) - film)
    radii = _clip_radii(centers[:, :2], radii, (nx, ny), (True, False), film)
    psi = -np.ones((1, ny, nx))
    _paint(psi, centers, radii, width, (True, False, True))
    r1, r2_ = _to_rho(psi, rho0)
    frac = float(np.pi * (radii ** 2).sum() / (nx * ny))
    return Fields(nx, ny, 1, r1, r2_, {
        "kind": "channel_emulsion_2d", "seed": seed, "droplets": len(radii), "rows": nrow,
        "area_fraction": frac, "r_mean": float(radii.mean()), "spacing": ax})


def duct_emulsion_3d(nx: int, ny: int, nz: int, seed: int, radius: float = 10.0,
                     volume_fraction: float = 0.7, jitter: float = 0.2, width: float = 2.0,
                     film: float = 1.0, rho0: float = 1.0) -> Fields:
    """Packed 3D emulsion in a square duct (walls in y and z, periodic in x).

    Centres sit on a face-centred-cubic lattice fitted to the duct: along each walled
    axis as many layers (half a cell apart) as fit between the two droplets that keep a
    film from the walls, along x an even number of half-cells close to the spacing of the
    requested volume fraction (never closer than the film allows); then a uniform
    +-jitter. Every pair keeps a film >= `film` (violating pairs are shrunk together).
    A film of 1 between spheres of radius 10 bounds the nearest-neighbour distance below
    by 21, so in a 128 x 128 duct 8 layers fit across each walled axis and the volume
    fraction is about 0.54 (0.62 for this film in unbounded FCC, 0.74 for touching
    spheres): a requested 0.7 is capped there."""
    rng = np.random.default_rng(seed)
    dnn = 2.0 * radius + film  # smallest allowed centre distance
    hmin = dnn / math.sqrt(2.0)  # half-cell of an FCC lattice whose neighbours are dnn apart

    def layers(n):
        # centres from radius + film - 1/2 to n - 1/2 - radius - film, half-cells >= hmin apart
        lo, hi = radius + film - 0.5, n - 0.5 - radius - film
        if hi <= lo:
            return np.array([0.5 * (n - 1)]), hmin
        k = int(math.floor((hi - lo) / hmin)) + 1
        if k == 1:
            return np.array([0.5 * (lo + hi)]), hmin
        step = (hi - lo) / (k - 1)
        return lo + step * np.arange(k), step

    ys, hy = layers(ny)
    zs, hz = layers(nz)
    # x half-cell: the spacing of the requested fraction, but no closer than the film allows
    # with the y and z half-cells chosen above; an even count keeps the lattice periodic
    cell = (16.0 * math.pi * radius ** 3 / (3.0 * volume_fraction)) ** (1.0 / 3.0)
    hx_need = math.sqrt(max(dnn * dnn - min(hy, hz) ** 2, 0.0))
    hx = max(0.5 * cell, hx_need, 1e-9)
    nhx = max(2, int(math.floor(nx / hx)) // 2 * 2)
    hx = nx / nhx
    pts = []
    for i in range(nhx):
        for j, y in enumerate(ys):
            for k, z in enumerate(zs):
                if (i + j + k) % 2 == 0:
                    pts.append([i * hx, y, z])
    centers = np.asarray(pts, dtype=np.float64)
    centers += rng.uniform(-jitter, jitter, size=centers.shape)
    radii = np.full(len(centers), float(radius))
    wall_gap = np.minimum.reduce([centers[:, 1] + 0.5, ny - 0.5 - centers[:, 1],
                                  centers[:, 2] + 0.5, nz - 0.5 - centers[:, 2]]) - film
    radii = np.minimum(radii, wall_gap)
    radii = _clip_radii(centers, radii, (nx, ny, nz), (True, False, False), film)
    psi = -np.ones((nz, ny, nx))
    _paint(psi, centers, radii, width, (True, False, False))
    r1, r2 = _to_rho(psi, rho0)
    frac = float(4.0 / 3.0 * np.pi * (radii ** 3).sum() / (nx * ny * nz))
    return Fields(nx, ny, nz, r1, r2, {
        "kind": "duct_emulsion_3d", "seed": seed, "droplets": len(radii),
        "volume_fraction": frac, "r_mean": float(radii.mean())})


@dataclass
class Member:
    """One channel of an ensemble: its size, its physical parameters and its fields."""
    nx: int
    ny: int
    force: float
    A_h: float
    fields: Fields


def ensemble_channels(n: int, seed: int, nx_range=(512, 2048), ny_range=(64, 256), af_range=(0.7, 0.9),
                      force_range=(1e-6, 1e-4), ah_range=(0.0, 0.1), r_lo: float = 12.0,
                      r_hi: float = 16.0) -> list:
    """n independent packed-emulsion channels for a parameter sweep: lengths and widths
    uniform in the given ranges (lengths rounded to multiples of 32), target area
    fractions uniform, body force log-uniform, NCI strength uniform, droplet radii as in
    channel_emulsion_2d. The flow-rate-versus-forcing study of the paper's soft flowing
    crystals (Results, Fig. 3) sweeps the same two controls."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n):
        nx = int(rng.integers(nx_range[0] // 32, nx_range[1] // 32 + 1)) * 32
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        af = float(rng.uniform(*af_range))
        g = float(np.exp(rng.uniform(np.log(force_range[0]), np.log(force_range[1]))))
        ah = float(rng.uniform(*ah_range))
        fl = channel_emulsion_2d(nx, ny, seed=int(rng.integers(1 << 30)), r_lo=r_lo, r_hi=r_hi,
                                 area_fraction=af)
        fl.meta["target_area_fraction"] = af
        out.append(Member(nx, ny, g, ah, fl))
    return out


def unet_params(shapes, seed: int, bias_scale: float = 0.0) -> list:
    """Seeded initial parameters of a convolutional network: for each weight shape
    [C_out, ..., C_in] a He-normal weight (standard deviation sqrt(2 / fan_in), fan_in =
    the product of all but the first dimension) and a bias drawn from N(0, bias_scale^2).
    Values are rounded to FP32 so that both sides start from the same numbers."""
    rng = np.random.default_rng(seed)
    out = []
    for _, shape in shapes:
        fan_in = int(np.prod(shape[1:]))
        w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=shape).astype(np.float32).astype(np.float64)
        b = (rng.normal(0.0, 1.0, size=shape[0]) * bias_scale).astype(np.float32).astype(np.float64)
        out.append((w, b))
    return out
