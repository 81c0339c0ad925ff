"""Pins of the FP64 CPU oracle against what the paper and lattice Boltzmann theory fix.

Each test checks the oracle against something other than itself: a defining property
of the lattice, a closed form, a conservation law of Eq. (CGLBE)'s continuum limit
(Eqs. (cont), (Nav_stok)), the augmented Young-Laplace law, or a hand-derived case.
They are chosen so that a dropped term, a wrong sign or index, or a transposed
operand in any stage of the step fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2003_11069_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- lattices
@pytest.mark.parametrize("lat,D,Q", [(oracle.D2Q9, 2, 9), (oracle.D3Q27, 3, 27)])
def test_lattice_isotropy(lat, D, Q):
    """The D2Q9/D3Q27 velocity sets and weights are fixed by their moment
    isotropy up to fourth order with c_s^2 = 1/3 (the lattices the paper names)."""
    c, w, opp = oracle.lattice(lat)
    assert c.shape == (Q, 3)
    assert len({tuple(v) for v in c}) == Q
    assert np.all(np.abs(c) <= 1) and np.all(c[:, D:] == 0)
    assert np.all(c[opp] == -c)
    cf = c[:, :D].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, cf), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cf, cf), np.eye(D) / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf), 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    d = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)
    # the documented ordering: base-3 digits of i, digit d -> {0,+1,-1}[d]
    for i in range(Q):
        dig = [i % 3, (i // 3) % 3, i // 9]
        assert list(c[i]) == [[0, 1, -1][x] for x in dig]


# --------------------------------------------------------------------------- gradient
@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_gradient_closed_form_sine(lat):
    """Isotropic gradient of psi = sin(k x) on a periodic lattice is exactly
    sin(k) cos(k x) (the stencil's Fourier symbol), not k cos(k x)."""
    nx, ny, nz = 16, 6, (1 if lat == oracle.D2Q9 else 5)
    p = oracle.make_params(lattice=lat, nx=nx, ny=ny, nz=nz)
    x = np.arange(nx)
    k = 2 * math.pi / nx
    for axis in range(2 if lat == oracle.D2Q9 else 3):
        dims = (nx, ny, nz)
        L = dims[axis]
        k = 2 * math.pi / L
        coord = np.indices((nz, ny, nx))[[2, 1, 0][axis]]
        psi = np.sin(k * coord).ravel()
        g = oracle.gradient(p, psi)
        expect = np.zeros_like(g)
        expect[axis] = math.sin(k) * np.cos(k * coord).ravel()
        assert np.max(np.abs(g - expect)) < 2e-15


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_gradient_exact_on_quadratics(lat):
    """Second-order isotropic gradient is exact for polynomials of degree <= 2
    (away from the periodic seam)."""
    nx, ny, nz = 10, 9, (1 if lat == oracle.D2Q9 else 8)
    p = oracle.make_params(lattice=lat, nx=nx, ny=ny, nz=nz)
    z, y, x = np.indices((nz, ny, nx)).astype(float)
    a = [0.3, -0.7, 0.45, 0.02, -0.015, 0.01, 0.005, -0.008, 0.004]
    psi = (a[0] * x + a[1] * y + a[2] * z + a[3] * x * x + a[4] * y * y + a[5] * z * z
           + a[6] * x * y + a[7] * y * z + a[8] * x * z)
    g = oracle.gradient(p, psi.ravel())
    ex = a[0] + 2 * a[3] * x + a[6] * y + a[8] * z
    ey = a[1] + 2 * a[4] * y + a[6] * x + a[7] * z
    ez = a[2] + 2 * a[5] * z + a[7] * y + a[8] * x
    if lat == oracle.D2Q9:
        ez = np.zeros_like(ez)
    inner = (x > 0) & (x < nx - 1) & (y > 0) & (y < ny - 1)
    if lat == oracle.D3Q27:
        inner &= (z > 0) & (z < nz - 1)
    for gg, ee in zip(g, (ex, ey, ez)):
        assert np.max(np.abs(gg.reshape(nz, ny, nx)[inner] - ee[inner])) < 1e-13


def test_gradient_wall_mirror():
    """Beyond a wall the stencil sees the mirror image of the solid neighbour across
    the wall plane: a field that varies only along the wall keeps exactly its interior
    gradient sin(k) cos(k x) on the wall rows and zero normal component."""
    for lat, nz, wz in ((oracle.D2Q9, 1, 0), (oracle.D3Q27, 4, 1)):
        p = oracle.make_params(lattice=lat, nx=12, ny=5, nz=nz, wall_y=1, wall_z=wz)
        x = np.indices((nz, 5, 12))[2]
        k = 2 * math.pi / 12
        psi = np.sin(k * x).ravel()
        g = oracle.gradient(p, psi)
        assert np.max(np.abs(g[1])) < 1e-15 and np.max(np.abs(g[2])) < 1e-15
        assert np.allclose(g[0], math.sin(k) * np.cos(k * x).ravel(), atol=2e-15)
    # a field normal to the wall: at y = 0 the mirror makes psi(-1) = psi(0), so the
    # gradient is the one-sided difference (psi(1) - psi(0))/2 times the stencil's 1/2*2
    p = oracle.make_params(nx=4, ny=6, wall_y=1)
    y = np.indices((6, 4))[0]
    psi = (0.1 * y * y).ravel()
    g = oracle.gradient(p, psi).reshape(3, 6, 4)
    assert np.allclose(g[1][0], (0.1 - 0.0) / 2, atol=1e-16)
    assert np.allclose(g[1][5], (0.1 * 25 - 0.1 * 16) / 2, atol=1e-15)


# --------------------------------------------------------------------------- collision
def _moments(c, w, f):
    return f.sum(), c.T @ f, np.einsum("ia,ib,i->ab", c, c, f)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_equilibrium_moments(lat):
    """f_eq has density rho, momentum rho u and second moment rho/3 I + rho u u
    (the moments the Navier-Stokes limit of Eq. (CGLBE) needs)."""
    c, w, _ = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    p = oracle.make_params(lattice=lat, nx=1, ny=1, nz=1)
    u = np.array([0.031, -0.017, 0.011])[:D]
    uu = np.zeros(3)
    uu[:D] = u
    f = oracle.init(p, [0.8], [0.3], uu.reshape(3, 1))
    for k, rk in enumerate((0.8, 0.3)):
        fk = f[k * len(w):(k + 1) * len(w)]
        m0, m1, m2 = _moments(c[:, :D].astype(float), w, fk)
        assert abs(m0 - rk) < 1e-15
        assert np.allclose(m1, rk * u, atol=1e-16)
        assert np.allclose(m2, rk / 3 * np.eye(D) + rk * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_collision_site_invariants(lat):
    """One site's collision: per-component mass kept; momentum gains exactly F (Guo);
    the perturbation's second moment is (2/9) A_s |grad psi| m m; recolouring leaves
    the total population unchanged."""
    rng = np.random.default_rng(3)
    c, w, _ = oracle.lattice(lat)
    Q = len(w)
    D = 2 if lat == oracle.D2Q9 else 3
    cf = c[:, :D].astype(float)
    fin = rng.uniform(0.02, 0.1, size=2 * Q) * np.concatenate([w, w]) * 9
    grad = np.zeros(3)
    grad[:D] = rng.normal(size=D) * 0.3
    F = np.zeros(3)
    F[:D] = rng.normal(size=D) * 1e-3
    base = dict(lattice=lat, nx=1, ny=1, nz=1, tau=0.8)
    p = oracle.make_params(A_s=0.01, beta=0.7, **base)
    out = oracle.collide_site(p, fin, grad, F)
    r1, r2 = fin[:Q].sum(), fin[Q:].sum()
    assert abs(out[:Q].sum() - r1) < 1e-15 * 10
    assert abs(out[Q:].sum() - r2) < 1e-15 * 10
    j_in = cf.T @ (fin[:Q] + fin[Q:])
    j_out = cf.T @ (out[:Q] + out[Q:])
    assert np.allclose(j_out - j_in, F[:D], atol=1e-16 * 20)
    # total population does not depend on beta (recolouring only redistributes colour)
    p0 = oracle.make_params(A_s=0.01, beta=0.0, **base)
    out0 = oracle.collide_site(p0, fin, grad, F)
    assert np.allclose(out[:Q] + out[Q:], out0[:Q] + out0[Q:], atol=1e-16 * 10)
    # beta = 0: colour follows the density ratio
    assert np.allclose(out0[:Q] * (r1 + r2), (out0[:Q] + out0[Q:]) * r1, atol=1e-15)
    # perturbation moments: difference between A_s and A_s = 0 at equal everything else
    pz = oracle.make_params(A_s=0.0, beta=0.0, **base)
    pert = (out0[:Q] + out0[Q:]) - sum(np.split(oracle.collide_site(pz, fin, grad, F), 2))
    g = np.linalg.norm(grad)
    m = grad[:D] / g
    assert abs(pert.sum()) < 1e-16 * 10
    assert np.allclose(cf.T @ pert, 0.0, atol=1e-17 * 10)
    assert np.allclose(np.einsum("ia,ib,i->ab", cf, cf, pert), 2 / 9 * 0.01 * g * np.outer(m, m),
                       atol=1e-16 * 10)
    # recolouring flux of colour: beta rho1 rho2/rho * sum_i w_i c_i (c_i.m)/|c_i|
    inv = np.array([0.0 if not v.any() else 1 / np.linalg.norm(v) for v in cf])
    rc = out[:Q] - out0[:Q]
    expect = 0.7 * r1 * r2 / (r1 + r2) * (w * (cf @ m) * inv)
    assert np.allclose(rc, expect, atol=1e-16 * 10)


# --------------------------------------------------------------------------- conservation
def _two_droplets(nx=48, ny=40):
    f1 = inputs.droplet(nx, ny, radius=9, center=(13.0, 19.5, 0.0))
    f2 = inputs.droplet(nx, ny, radius=9, center=(33.5, 19.5, 0.0))
    rho1 = np.maximum(f1.rho1, f2.rho1)
    return rho1, 1.0 - rho1


def test_mass_conservation_with_nci_and_walls():
    """Each component's mass is conserved to rounding (continuity, Eq. (cont); the
    recolouring keeps rho_k per site) with walls, forcing and active NCI."""
    nx, ny = 48, 40
    rho1, rho2 = _two_droplets(nx, ny)
    p = oracle.make_params(nx=nx, ny=ny, wall_y=1, tau=1.0, A_s=0.01, beta=0.7, A_h=0.05,
                           force=(1e-5, 0, 0))
    f = oracle.init(p, rho1, rho2)
    m0 = oracle.observables(p, f)["mass"]
    fd = oracle.fields(p, oracle.step(p, f, 5))
    assert (fd["hit"] > 0).sum() > 10  # NCI is really active between the droplets
    f = oracle.step(p, f, 300)
    m1 = oracle.observables(p, f)["mass"]
    assert np.all(np.abs(m1 - m0) / m0 < 1e-13)


def test_momentum_conservation_and_forcing():
    """Periodic box, A_h = 0: total momentum is conserved with G = 0 and grows by exactly
    N G per step with G != 0 (Guo source; perturbation and recolouring carry none)."""
    nx, ny = 48, 40
    rho1, rho2 = _two_droplets(nx, ny)
    for G in (0.0, 2e-5):
        p = oracle.make_params(nx=nx, ny=ny, tau=0.9, A_s=0.01, beta=0.7, force=(G, -0.5 * G, 0))
        f = oracle.init(p, rho1, rho2)
        P0 = oracle.observables(p, f)["momentum"]
        f = oracle.step(p, f, 100)
        P1 = oracle.observables(p, f)["momentum"]
        N = nx * ny
        assert np.allclose(P1 - P0, [100 * N * G, -50 * N * G, 0.0], atol=1e-11, rtol=1e-12)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_uniform_flow_is_fixed_point(lat):
    """A uniform single-phase flow f = f_eq(rho, u) with no force in a periodic box is a
    fixed point of stream + BGK (Galilean-invariant steady state)."""
    nz = 1 if lat == oracle.D2Q9 else 3
    N = 5 * 4 * nz
    p = oracle.make_params(lattice=lat, nx=5, ny=4, nz=nz, tau=0.7, A_s=0.01, beta=0.7, A_h=0.05)
    u = np.zeros((3, N))
    u[0], u[1] = 0.04, -0.03
    if nz > 1:
        u[2] = 0.02
    f = oracle.init(p, np.zeros(N), np.full(N, 1.3), u)
    g = oracle.step(p, f, 7)
    assert np.max(np.abs(g - f)) < 1e-16 * 8


# --------------------------------------------------------------------------- Poiseuille
def _poiseuille(lat, H, tau, G=1e-6, walls="y"):
    nz = 1 if lat == oracle.D2Q9 else (H if walls == "z" else 2)
    ny = H if walls == "y" else 2
    p = oracle.make_params(lattice=lat, nx=2, ny=ny, nz=nz, wall_y=int(walls == "y"),
                           wall_z=int(walls == "z"), tau=tau, force=(G, 0, 0))
    fl = inputs.uniform(2, ny, nz, psi0=-1.0)
    f = oracle.init(p, fl.rho1, fl.rho2)
    nu = (tau - 0.5) / 3
    f = oracle.step(p, f, int(12 * H * H / nu))
    u = oracle.fields(p, f)["u"][0].reshape(nz, ny, 2)
    prof = u[0, :, 0] if walls == "y" else u[:, 0, 0]
    y = np.arange(H)
    ua = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return np.sqrt(((prof - ua) ** 2).sum() / (ua ** 2).sum()), f, p


@pytest.mark.parametrize("lat,walls", [(oracle.D2Q9, "y"), (oracle.D3Q27, "y"), (oracle.D3Q27, "z")])
def test_poiseuille_exact_at_magic_tau(lat, walls):
    """Force-driven channel with halfway bounce-back: BGK reproduces the parabolic
    profile u = G/(2 rho nu) (y+1/2)(H-1/2-y) exactly when tau = 1/2 + sqrt(3/16)."""
    err, _, _ = _poiseuille(lat, 10, 0.5 + math.sqrt(3.0 / 16.0), walls=walls)
    assert err < 1e-10


def test_poiseuille_second_order():
    """At tau = 1 the wall-slip error of halfway bounce-back falls as 1/H^2."""
    e8, _, _ = _poiseuille(oracle.D2Q9, 8, 1.0)
    e16, f, p = _poiseuille(oracle.D2Q9, 16, 1.0)
    assert e16 < 2e-3
    assert 3.8 < e8 / e16 < 4.2
    # the flow-rate observable is the cross-section flux sum_y rho u_x (per unit length)
    obs = oracle.observables(p, f)
    u = oracle.fields(p, f)["u"][0]
    assert abs(obs["flow_rate"] - u.sum() / p.nx) < 1e-15
    assert obs["flow_rate_disp"] == 0.0


# --------------------------------------------------------------------------- Laplace
@pytest.mark.slow
@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_laplace_law(lat):
    """Static droplets: pressure jump c_s^2 (rho_in - rho_out) is linear in 1/R with slope
    sigma = (2/9)(A_1 + A_2) tau = 4 A_s tau / 9 (augmented Young-Laplace law with pi = 0).
    D3Q27 runs the 2D geometry extruded along z (nz = 1): a cylinder, dp = sigma/R."""
    n, A_s, tau = 80, 0.01, 1.0
    radii = np.array([10.0, 13.0, 16.0, 19.0])
    dps = []
    for R in radii:
        p = oracle.make_params(lattice=lat, nx=n, ny=n, nz=1, tau=tau, A_s=A_s, beta=0.7)
        fl = inputs.droplet(n, n, radius=R)
        f = oracle.init(p, fl.rho1, fl.rho2)
        f = oracle.step(p, f, 2000)
        fd = oracle.fields(p, f)
        rho = (fd["rho1"] + fd["rho2"]).reshape(n, n)
        dps.append((rho[n // 2, n // 2] - rho[0, 0]) / 3.0)
        assert np.max(np.abs(fd["u"])) < 5e-4  # spurious currents stay small
    dps = np.array(dps)
    A = np.vstack([1.0 / radii, np.ones_like(radii)]).T
    (slope, icept), *_ = np.linalg.lstsq(A, dps, rcond=None)
    fit = A @ np.array([slope, icept])
    r2 = 1 - ((dps - fit) ** 2).sum() / ((dps - dps.mean()) ** 2).sum()
    sigma = 4 * A_s * tau / 9
    assert r2 > 0.999
    assert abs(slope / sigma - 1) < 0.10
    assert abs(icept) < 0.1 * sigma / radii.max()


def test_planar_interface_is_static():
    """A flat interface has zero curvature: no flow and equal bulk pressures
    (Young-Laplace with nabla.n = 0)."""
    p = oracle.make_params(nx=4, ny=64, tau=1.0, A_s=0.01, beta=0.7)
    fl = inputs.slabs(4, 64, [(16, 47)])
    f = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 10000)
    fd = oracle.fields(p, f)
    rho = (fd["rho1"] + fd["rho2"]).reshape(64, 4)[:, 0]
    assert np.max(np.abs(fd["u"])) < 1e-10
    assert abs(rho[32] - rho[0]) < 1e-9
    psi = fd["psi"].reshape(64, 4)[:, 0]
    assert psi[32] > 0.99 and psi[0] < -0.99  # the colours stay segregated


# --------------------------------------------------------------------------- NCI
def _golden_planar():
    rows = np.loadtxt(os.path.join(GOLDEN, "nci_planar_y16.txt"), comments="#")
    return rows


def test_nci_planar_golden():
    """Hand-derived NCI distances and forces on a planar profile (golden fixture)."""
    rows = _golden_planar()
    nx, ny, A = 4, 16, 0.05
    psi = np.repeat(rows[:, 1], nx)  # idx = x + nx*y
    p = oracle.make_params(nx=nx, ny=ny, A_h=A, h_min=2.0, h_max=4.0, g_th=0.05)
    g = oracle.gradient(p, psi)
    assert np.allclose(g[1].reshape(ny, nx), rows[:, 2][:, None], atol=1e-15)
    assert np.max(np.abs(g[0])) < 1e-16
    fr, hit = oracle.nci(p, psi)
    assert np.array_equal(hit.reshape(ny, nx), np.repeat(rows[:, 3].astype(int)[:, None], nx, 1))
    assert np.allclose(fr[1].reshape(ny, nx), A * rows[:, 4][:, None], atol=1e-15, rtol=1e-14)
    assert np.max(np.abs(fr[0])) < 1e-16
    # h_max = 3: the h = 4 pairs fall beyond the cutoff and feel nothing
    p3 = oracle.make_params(nx=nx, ny=ny, A_h=A, h_min=2.0, h_max=3.0, g_th=0.05)
    fr3, hit3 = oracle.nci(p3, psi)
    exp3 = rows[:, 3].astype(int)
    exp3[exp3 > 3] = 0
    assert np.array_equal(hit3.reshape(ny, nx)[:, 0], exp3)


def test_nci_probe_threshold_golden():
    """The probe-side interface test of the ray (golden fixture): a facing probe with
    0 < |grad psi| <= g_th is passed over, one just above g_th is a hit."""
    rows = np.loadtxt(os.path.join(GOLDEN, "nci_probe_threshold_y16.txt"), comments="#")
    nx, ny, A = 4, 16, 0.05
    psi = np.repeat(rows[:, 1], nx)
    p = oracle.make_params(nx=nx, ny=ny, A_h=A, h_min=2.0, h_max=4.0, g_th=0.05)
    g = oracle.gradient(p, psi)
    gy = rows[:, 2]
    assert np.allclose(g[1].reshape(ny, nx), gy[:, None], atol=1e-15)
    assert np.max(np.abs(g[0])) < 1e-16
    # the fixture's premise: one weak facing row (0 < |g| <= g_th), one just above g_th
    assert 0 < abs(gy[3]) <= 0.05 and 0.05 < abs(gy[12]) < 0.07
    fr, hit = oracle.nci(p, psi)
    assert np.array_equal(hit.reshape(ny, nx), np.repeat(rows[:, 3].astype(int)[:, None], nx, 1))
    assert np.allclose(fr[1].reshape(ny, nx), A * rows[:, 4][:, None], atol=1e-15, rtol=1e-14)
    assert np.max(np.abs(fr[0])) < 1e-16


def _diag_expected(prof, g_th, smax):
    """Brute force for psi(x, y) = prof[(x + y) mod L] on an L x L periodic D2Q9 lattice.
    For such fields the isotropic gradient has equal x and y components
    (psi(q+1) - psi(q-1))/3 + (psi(q+2) - psi(q-2))/12, so n = -sign(g) (1,1)/sqrt(2);
    the probe at step s is (d, d) with d = sign * round(s/sqrt(2)), i.e. q + 2d."""
    L = len(prof)
    gq = np.array([(prof[(q + 1) % L] - prof[(q - 1) % L]) / 3 + (prof[(q + 2) % L] - prof[(q - 2) % L]) / 12
                   for q in range(L)])
    hit = np.zeros(L, dtype=int)
    for q in range(L):
        g = abs(gq[q]) * math.sqrt(2)
        if not g > g_th:
            continue
        sgn = -1 if gq[q] > 0 else 1
        for s in range(1, smax + 1):
            d = sgn * int(math.floor(s / math.sqrt(2) + 0.5))
            qq = (q + 2 * d) % L
            if abs(gq[qq]) * math.sqrt(2) > g_th and np.sign(gq[qq]) != np.sign(gq[q]):
                hit[q] = s
                break
    return gq, hit


def test_nci_diagonal_brute_force():
    """Rays along the lattice diagonal: rounding of s n and periodic wrap of the probe."""
    L = 16
    prof = np.array([1, 1, 1, 1, 0.6, -0.2, -0.9, -1, -0.9, -0.2, 0.6, 1, 1, 1, 1, 1], dtype=float)
    x, y = np.meshgrid(np.arange(L), np.arange(L))
    psi = prof[(x + y) % L].ravel()
    p = oracle.make_params(nx=L, ny=L, A_h=0.05, g_th=0.05)
    g = oracle.gradient(p, psi)
    gq, hq = _diag_expected(prof, 0.05, 4)
    q = ((x + y) % L).ravel()
    assert np.allclose(g[0], gq[q], atol=1e-15) and np.allclose(g[1], gq[q], atol=1e-15)
    fr, hit = oracle.nci(p, psi)
    assert np.array_equal(hit, hq[q])
    assert (hq > 0).sum() >= 4


def test_nci_zero_beyond_cutoff_is_bitwise():
    """One isolated droplet has no facing interface within h_max, so A_h = 0.05 gives a
    state bitwise identical to A_h = 0 (the force vanishes beyond h_max)."""
    n = 64
    fl = inputs.droplet(n, n, radius=20)
    states = []
    for A_h in (0.0, 0.05):
        p = oracle.make_params(nx=n, ny=n, tau=1.0, A_s=0.01, beta=0.7, A_h=A_h)
        f = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), 150)
        states.append(f)
        assert (oracle.fields(p, f)["hit"] == 0).all()
    assert np.array_equal(states[0], states[1])


def test_nci_films_far_and_near():
    """Two planar films: no site feels a force when the continuous gap is much wider than
    h_max; a narrow gap gives a nonzero force that is antisymmetric across it."""
    nx, ny = 4, 64
    p = oracle.make_params(nx=nx, ny=ny, A_h=0.05, g_th=0.05)
    far = inputs.slabs(nx, ny, [(10, 22), (42, 54)])
    fr, hit = oracle.nci(p, (far.rho1 - far.rho2))
    assert (hit == 0).all() and np.max(np.abs(fr)) == 0.0
    near = inputs.slabs(nx, ny, [(4, 29), (35, 60)])
    psi = near.rho1 - near.rho2
    fr, hit = oracle.nci(p, psi)
    fy = fr[1].reshape(ny, nx)[:, 0]
    assert (hit > 0).sum() > 0
    mid = 32.0  # the gap centre: psi is symmetric about y = 32
    for yy in range(ny):
        mirror = int(round(2 * mid - yy)) % ny
        assert abs(fy[yy] + fy[mirror]) < 1e-15
    # the force on the lower film's upper face points down (away from the other film)
    assert fy[27:31].min() < 0 and fy[27:31].max() <= 0.0


# --------------------------------------------------------------------------- EDM forcing
@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_edm_site_invariants(lat):
    """Exact difference method (the paper's insertion of the near-contact force): each
    component's mass is kept, the mixture gains exactly F = G + F_rep of momentum, and the
    continuous phase (component 2) is untouched by F_rep: it feels only its mass share
    of the body force."""
    rng = np.random.default_rng(5)
    c, w, _ = oracle.lattice(lat)
    Q = len(w)
    D = 2 if lat == oracle.D2Q9 else 3
    cf = c[:, :D].astype(float)
    fin = rng.uniform(0.02, 0.1, size=2 * Q) * np.concatenate([w, w]) * 9
    grad = np.zeros(3)
    grad[:D] = rng.normal(size=D) * 0.3
    G = np.zeros(3)
    G[:D] = rng.normal(size=D) * 1e-4
    Frep = np.zeros(3)
    Frep[:D] = rng.normal(size=D) * 1e-3
    p = oracle.make_params(lattice=lat, nx=1, ny=1, nz=1, tau=0.8, A_s=0.01, beta=0.7, force=tuple(G), forcing=1)
    out = oracle.collide_site(p, fin, grad, G + Frep)
    r1, r2 = fin[:Q].sum(), fin[Q:].sum()
    assert abs(out[:Q].sum() - r1) < 1e-14 and abs(out[Q:].sum() - r2) < 1e-14
    j_in = cf.T @ (fin[:Q] + fin[Q:])
    assert np.allclose(cf.T @ (out[:Q] + out[Q:]) - j_in, (G + Frep)[:D], atol=1e-16 * 50)
    # component 2 does not see F_rep
    out0 = oracle.collide_site(p, fin, grad, G)
    assert np.allclose(out[Q:], out0[Q:], atol=1e-16 * 10)
    assert not np.allclose(out[:Q], out0[:Q], atol=1e-9)
    # the added populations are f_eq(rho_k, u + dU_k) - f_eq(rho_k, u): zero without force
    pz = oracle.make_params(lattice=lat, nx=1, ny=1, nz=1, tau=0.8, A_s=0.01, beta=0.7, forcing=1)
    pg = oracle.make_params(lattice=lat, nx=1, ny=1, nz=1, tau=0.8, A_s=0.01, beta=0.7, forcing=0)
    assert np.allclose(oracle.collide_site(pz, fin, grad, np.zeros(3))[Q:],
                       oracle.collide_site(pg, fin, grad, np.zeros(3))[Q:], atol=1e-16)


def test_edm_poiseuille_second_order():
    """Single-phase channel driven by G with the exact difference method: the parabolic
    profile is reached with second-order convergence in H."""
    errs = []
    for H in (8, 16):
        tau = 1.0
        p = oracle.make_params(nx=2, ny=H, wall_y=1, tau=tau, force=(1e-6, 0, 0), forcing=1)
        fl = inputs.uniform(2, H, 1, psi0=-1.0)
        f = oracle.step(p, oracle.init(p, fl.rho1, fl.rho2), int(12 * H * H / ((tau - 0.5) / 3)))
        u = oracle.fields(p, f)["u"][0].reshape(H, 2)[:, 0]
        nu = (tau - 0.5) / 3
        y = np.arange(H)
        ua = 1e-6 / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
        errs.append(np.sqrt(((u - ua) ** 2).sum() / (ua ** 2).sum()))
    assert errs[1] < 2e-3 and 3.5 < errs[0] / errs[1] < 4.5, errs
