"""An independent NumPy restatement of one step of the method, checked against the C oracle.

The restatement is written from the paper's "Materials and Methods" (Eq. (CGLBE) for the
two population sets, the collision Omega = Omega^(3)[Omega^(1) + Omega^(2)], psi, n and
delta_I after Eq. (stjump), the near-contact force of Eq. (near_c) with its A_h(h)
profile) and the readings the oracle states where the paper is silent (Guo forcing,
B_i = w_i/3, recolouring with cos(theta_i) = c_i.m/|c_i|, halfway bounce-back, the wall
mirror of the gradient, the ray rule of the near-contact distance). It is vectorised
over sites with array shifts, the oracle is nested C loops over sites: the two share no
code, so an error in either (a dropped term, a sign, a transposed index, a wrong probe
rule) shows up as a disagreement. One step on 8 x 8 D2Q9 and 6 x 6 x 6 D3Q27 lattices
with walls and the near-contact force active, compared to 1e-14 on the population scale.
"""
import itertools

import numpy as np
import pytest

import oracle


def _velocities(D):
    """Direction i has components {0,+1,-1}[digit] of the base-3 digits of i (x lowest)."""
    Q = 3 ** D
    c = np.zeros((Q, 3), dtype=np.int64)
    for i in range(Q):
        for a in range(D):
            c[i, a] = (0, 1, -1)[(i // 3 ** a) % 3]
    c2 = (c ** 2).sum(axis=1)
    if D == 2:
        w = np.array([4 / 9, 1 / 9, 1 / 36])[c2]
    else:
        w = np.array([8 / 27, 2 / 27, 1 / 54, 1 / 216])[c2]
    opp = np.array([int(np.flatnonzero((c == -c[i]).all(axis=1))[0]) for i in range(Q)])
    return c, w, opp


class Restated:
    def __init__(self, D, shape, walls, tau, A_s, beta, A_h, h_min, h_max, g_th, G):
        self.D = D
        self.shape = shape  # (nz, ny, nx)
        self.walls = walls  # (wall_y, wall_z)
        self.tau, self.A_s, self.beta = tau, A_s, beta
        self.A_h, self.h_min, self.h_max, self.g_th = A_h, h_min, h_max, g_th
        self.G = np.array(G, dtype=float)
        self.c, self.w, self.opp = _velocities(D)
        self.Q = len(self.w)
        nz, ny, nx = shape
        self.z, self.y, self.x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def _beyond(self, dy, dz):
        """Sites whose neighbour at offset (., dy, dz) lies beyond a wall."""
        nz, ny, _ = self.shape
        out = np.zeros(self.shape, dtype=bool)
        if self.walls[0]:
            out |= (self.y + dy < 0) | (self.y + dy >= ny)
        if self.walls[1]:
            out |= (self.z + dz < 0) | (self.z + dz >= nz)
        return out

    @staticmethod
    def _shift(a, d):
        """b[x] = a[x - d] with periodic wrap on every axis (d in x, y, z order)."""
        return np.roll(a, shift=(d[2], d[1], d[0]), axis=(0, 1, 2))

    def stream(self, f):
        """Pull f_i^k(x) = f*_i^k(x - c_i); halfway bounce-back where x - c_i is a wall."""
        g = np.empty_like(f)
        for i in range(self.Q):
            ci = self.c[i]
            bounce = self._beyond(-ci[1], -ci[2])
            for k in range(2):
                g[k, i] = np.where(bounce, f[k, self.opp[i]], self._shift(f[k, i], ci))
        return g

    def gradient(self, psi):
        """(1/c_s^2) sum_i w_i c_i psi(x + c_i); a neighbour beyond a wall is replaced by its
        mirror image (the wall-crossing components of c_i dropped)."""
        grad = np.zeros((3,) + self.shape)
        nz, ny, nx = self.shape
        for i in range(1, self.Q):
            d = self.c[i].copy()
            yy = self.y + d[1]
            zz = self.z + d[2]
            if self.walls[0]:
                yy = np.where((yy < 0) | (yy >= ny), self.y, yy)
            if self.walls[1]:
                zz = np.where((zz < 0) | (zz >= nz), self.z, zz)
            v = psi[zz % nz, yy % ny, (self.x + d[0]) % nx]
            for a in range(self.D):
                grad[a] += self.w[i] * d[a] * v
        return 3.0 * grad

    def nci(self, grad):
        """h(x): the first probe x + round(s n), s = 1..floor(h_max), that is an interface site
        facing x (n(y).n(x) < 0); a probe beyond a wall ends the search. F_rep = -A_h(h) n delta_I."""
        nz, ny, nx = self.shape
        g = np.sqrt((grad ** 2).sum(axis=0))
        hit = np.zeros(self.shape, dtype=int)
        frep = np.zeros((3,) + self.shape)
        smax = int(np.floor(self.h_max))
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            if not g[z, y, x] > self.g_th:
                continue
            n = -grad[:, z, y, x] / g[z, y, x]
            for s in range(1, smax + 1):
                d = [int(np.sign(v) * np.floor(abs(v) + 0.5)) for v in s * n]  # half away from 0
                if self.D == 2:
                    d[2] = 0
                py, pz = y + d[1], z + d[2]
                if (self.walls[0] and not 0 <= py < ny) or (self.walls[1] and not 0 <= pz < nz):
                    break
                py, pz, px = py % ny, pz % nz, (x + d[0]) % nx
                gp = g[pz, py, px]
                if gp > self.g_th and (-grad[:, pz, py, px] / gp) @ n < 0:
                    hit[z, y, x] = s
                    break
            h = hit[z, y, x]
            if h:
                A = self.A_h if h <= self.h_min else (self.A_h * (self.h_min / h) ** 3 if h <= self.h_max else 0.0)
                frep[:, z, y, x] = -A * n * (0.5 * g[z, y, x])
        return frep, hit

    def step(self, f):
        fp = self.stream(f)
        rho1, rho2 = fp[0].sum(axis=0), fp[1].sum(axis=0)
        rho = rho1 + rho2
        psi = (rho1 - rho2) / rho
        grad = self.gradient(psi)
        frep, hit = self.nci(grad)
        F = self.G[:, None, None, None] + frep
        tot = fp[0] + fp[1]
        j = np.einsum("ia,i...->a...", self.c.astype(float), tot)
        u = (j + 0.5 * F) / rho
        g = np.sqrt((grad ** 2).sum(axis=0))
        m = np.where(g > 0, grad / np.where(g > 0, g, 1.0), 0.0)
        om = 1.0 / self.tau
        uu = (u ** 2).sum(axis=0)
        uF = (u * F).sum(axis=0)
        out = np.empty_like(fp)
        for i in range(self.Q):
            ci = self.c[i].astype(float)
            cu = np.einsum("a,a...->...", ci, u)
            cF = np.einsum("a,a...->...", ci, F)
            cm = np.einsum("a,a...->...", ci, m)
            feq = self.w[i] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)
            guo = (1 - 0.5 * om) * self.w[i] * (3 * (cF - uF) + 9 * cu * cF)
            pert = self.A_s * g * (self.w[i] * cm ** 2 - self.w[i] / 3)  # two components, A_s/2 each
            fs = tot[i] - om * (tot[i] - feq) + guo + pert
            norm = np.sqrt((ci ** 2).sum())
            cos = cm / norm if norm > 0 else 0.0
            rc = self.beta * rho1 * rho2 / rho * self.w[i] * cos
            out[0, i] = rho1 / rho * fs + rc
            out[1, i] = rho2 / rho * fs - rc
        return out, hit


def _case(D):
    rng = np.random.default_rng(17 + D)
    if D == 2:
        shape, walls = (1, 8, 8), (1, 0)
    else:
        shape, walls = (6, 6, 6), (1, 1)
    nz, ny, nx = shape
    # a short-wavelength colour pattern plus noise: many interface sites whose normals face
    # each other within h_max, rays stopped by the walls, several distances h
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    psi0 = 0.9 * np.sin(4 * np.pi * xx / nx + 0.3) * np.cos(2 * np.pi * yy / ny + 0.7)
    if D == 3:
        psi0 = psi0 * np.cos(2 * np.pi * zz / nz + 0.2)
    psi0 = psi0 + 0.05 * rng.uniform(-1, 1, size=shape)
    rho1 = 0.5 * (1 + psi0)
    rho2 = 0.5 * (1 - psi0)
    prm = dict(tau=0.9, A_s=0.02, beta=0.7, A_h=0.05, h_min=2.0, h_max=4.0, g_th=0.05,
               G=(2e-5, -1e-5, 1e-5 if D == 3 else 0.0))
    return shape, walls, rho1.ravel(), rho2.ravel(), prm, rng


@pytest.mark.parametrize("D", [2, 3])
def test_numpy_restatement_matches_oracle(D):
    shape, walls, rho1, rho2, prm, rng = _case(D)
    nz, ny, nx = shape
    lat = oracle.D2Q9 if D == 2 else oracle.D3Q27
    p = oracle.make_params(lattice=lat, nx=nx, ny=ny, nz=nz, wall_y=walls[0], wall_z=walls[1], tau=prm["tau"],
                           A_s=prm["A_s"], beta=prm["beta"], A_h=prm["A_h"], h_min=prm["h_min"],
                           h_max=prm["h_max"], g_th=prm["g_th"], force=prm["G"])
    f0 = oracle.init(p, rho1, rho2)
    Q = 9 if D == 2 else 27
    # a non-equilibrium part as well, so that every term of the collision matters
    f0 = f0 * (1 + 0.05 * rng.uniform(-1, 1, size=f0.size))
    R = Restated(D, shape, walls, **prm)
    fr, hit = R.step(f0.reshape(2, Q, nz, ny, nx))
    ref = oracle.step(p, f0, 1)
    of = oracle.fields(p, f0)
    assert np.array_equal(hit.ravel(), of["hit"])
    assert (hit > 0).sum() >= 3 and len(np.unique(hit)) >= 3  # several distances occur
    _, w, _ = oracle.lattice(lat)
    scale = np.maximum(np.abs(ref), np.tile(np.repeat(w, nx * ny * nz), 2))
    err = np.max(np.abs(fr.ravel() - ref) / scale)
    assert err <= 1e-14, err
