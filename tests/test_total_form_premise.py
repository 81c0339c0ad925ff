"""The premise of the total + recolouring form of the state (LB_STATE_TOTAL_RECOLOUR), checked
on the FP64 oracle's collision with no GPU involved.

With Guo forcing the collision (paper, "Materials and Methods": Omega = Omega^(3)[Omega^(1) +
Omega^(2)]) applies BGK, the Guo source and the perturbation to the total population and then
recolours it, so its output at a site is fixed by the totals f*_i = f_i^1 + f_i^2 and four
numbers: for every moving direction
    f_i^1 = phi_1 f*_i + (w_i/|c_i|) c_i.s,   f_i^2 = f*_i - f_i^1,
phi_1 = rho_1/rho, s = beta (rho_1 rho_2/rho) grad psi/|grad psi|; and the rest population of
each component is rho_k minus that component's moving populations (BGK, the Guo source and
the perturbation keep the total mass, and the recolouring terms of opposite directions
cancel). The GPU stores exactly these quantities. With the exact difference method the
collision adds a term per component after the recolouring, so the split does not hold there:
those steps keep the two-population state, and the last test shows the difference."""
import numpy as np
import pytest

import oracle


def _random_site(rng, lat, p):
    c, w, _ = oracle.lattice(lat)
    Q = len(w)
    rho1, rho2 = rng.uniform(0.0, 1.0), rng.uniform(0.0, 1.0)
    if rng.uniform() < 0.2:  # a pure phase
        rho2 = 0.0
    u = rng.normal(0.0, 0.02, 3)
    if lat == oracle.D2Q9:
        u[2] = 0.0
    cu = c @ u
    feq = w * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    fin = np.stack([rho1 * feq, rho2 * feq]) * (1 + rng.normal(0.0, 0.01, (2, Q)))
    grad = rng.normal(0.0, 0.1, 3) if rng.uniform() > 0.2 else np.zeros(3)  # some sites in a bulk
    if lat == oracle.D2Q9:
        grad[2] = 0.0
    F = rng.normal(0.0, 1e-4, 3)
    if lat == oracle.D2Q9:
        F[2] = 0.0
    return c, w, fin, grad, F


def _split(c, w, fin, grad, beta, out):
    rho1, rho2 = fin[0].sum(), fin[1].sum()
    rho = rho1 + rho2
    g = np.linalg.norm(grad)
    m = grad / g if g > 0 else np.zeros(3)
    phi1 = rho1 / rho
    s = beta * rho1 * rho2 / rho * m
    t = out.sum(axis=0)
    length = np.sqrt((c ** 2).sum(axis=1))
    inv_len = np.divide(1.0, length, out=np.zeros_like(length), where=length > 0)
    a = phi1 * t + w * inv_len * (c @ s)
    return rho1, rho2, a, t


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_guo_collision_output_is_the_recolouring_of_its_totals(lat):
    rng = np.random.default_rng(2003 + lat)
    p = oracle.make_params(lattice=lat, tau=0.8, A_s=0.01, beta=0.7, force=(1e-5, 2e-6, 0.0))
    for _ in range(40):
        c, w, fin, grad, F = _random_site(rng, lat, p)
        Q = len(w)
        out = oracle.collide_site(p, fin, grad, F).reshape(2, Q)
        rho1, rho2, a, t = _split(c, w, fin, grad, p.beta, out)
        scale = np.maximum(np.abs(out), w)
        moving = np.arange(Q) != 0
        assert np.all(np.abs(out[0][moving] - a[moving]) <= 1e-14 * scale[0][moving])
        assert np.all(np.abs(out[1][moving] - (t - a)[moving]) <= 1e-14 * scale[1][moving])
        # the rest populations complete each component's mass
        assert abs(out[0][0] - (rho1 - out[0][moving].sum())) <= 1e-14 * max(rho1, w[0])
        assert abs(out[1][0] - (rho2 - out[1][moving].sum())) <= 1e-14 * max(rho2, w[0])


def test_recolouring_terms_of_opposite_directions_cancel():
    """The rest populations rho_k - phi_k S rely on sum_i (w_i/|c_i|) c_i.s = 0: each moving
    direction's term is the negative of its opposite's."""
    c, w, opp = oracle.lattice(oracle.D3Q27)
    length = np.sqrt((c ** 2).sum(axis=1))
    s = np.array([0.3, -0.2, 0.7])
    term = np.where(length > 0, w / np.where(length > 0, length, 1) * (c @ s), 0.0)
    assert np.all(term + term[opp] == 0.0)
    assert np.all(w == w[opp])


def test_exact_difference_forcing_is_not_a_recolouring_of_totals():
    """With the exact difference method (forcing = 1) and a nonzero force the component
    populations differ from the recolouring split of the totals by the per-component
    equilibrium shifts, far beyond rounding: those steps keep two populations per direction."""
    rng = np.random.default_rng(11)
    p = oracle.make_params(lattice=oracle.D3Q27, tau=0.8, A_s=0.01, beta=0.7, force=(1e-4, 0.0, 0.0), forcing=1)
    worst = 0.0
    for _ in range(10):
        c, w, fin, grad, F = _random_site(rng, oracle.D3Q27, p)
        F = np.array([1e-4, 3e-5, 0.0])
        out = oracle.collide_site(p, fin, grad, F).reshape(2, 27)
        if fin[0].sum() == 0.0 or fin[1].sum() == 0.0:
            continue
        _, _, a, _ = _split(c, w, fin, grad, p.beta, out)
        worst = max(worst, float(np.max(np.abs(out[0][1:] - a[1:]) / np.maximum(np.abs(out[0][1:]), w[1:]))))
    assert worst > 1e-8


@pytest.mark.parametrize("rho0", [0.97, 1.0, 1.013, 1.2])
def test_fp16_totals_on_the_2_24_grid_sum_exactly(rho0):
    """The FP16 form holds its reference as (216 w_i) r with r = rho_0/216 rounded to a
    multiple of 2^-24, so a decoded total (216 w_i) r + d_i (d_i an FP16 value, itself a
    multiple of 2^-24) is a multiple of 2^-24 below 1: exact in FP32. A running FP32 sum of
    a site's 26 totals is then exact too, and equals 152 r + the sum of the deviations
    (152 = 216 (1 - w_0)), which is how the collision forms it: the rest populations complete
    the stored mass with no rounding (measured: no drift; with the reference rounded to
    nearest instead, a plain sum rounded the same way at every site)."""
    from fractions import Fraction

    _, w, _ = oracle.lattice(oracle.D3Q27)
    k = np.rint(216.0 * w).astype(np.int64)
    assert np.all(np.abs(216.0 * w - k) < 1e-12) and sorted(set(k.tolist())) == [1, 4, 16, 64]
    assert int(k[1:].sum()) == 152
    r = np.float32(np.rint(rho0 / 216.0 * 2.0 ** 24) / 2.0 ** 24)
    rng = np.random.default_rng(int(rho0 * 1000))
    for _ in range(100):
        d = (rng.normal(0.0, 3e-3, 26) * w[1:]).astype(np.float16).astype(np.float32)
        base = np.float32(k[1:].astype(np.float32) * r)  # exact: (216 w_i) r on the grid
        t = base + d
        for ti, ki, di in zip(t, k[1:], d):
            assert Fraction(float(ti)) == int(ki) * Fraction(float(r)) + Fraction(float(di))
        S = np.float32(0.0)
        Sd = np.float32(0.0)
        for ti, di in zip(t, d):
            S = np.float32(S + ti)
            Sd = np.float32(Sd + di)
        exact = sum(Fraction(float(x)) for x in t)
        assert Fraction(float(S)) == exact
        St = np.float32(np.float32(152.0) * r) + Sd
        assert Fraction(float(np.float32(St))) == exact


def test_collision_on_deviations_equals_collision_on_totals():
    """A step that reads the FP16 form collides on the deviations d_i = f*_i - (216 w_i) r: the
    references carry no momentum (sum_i c_i w_i = 0), so j is the deviations' momentum, and
    BGK with the Guo source and the perturbation, f*_i' = (1 - omega) f*_i + w_i (E_i +/- O_i),
    with E_i containing K0 = omega rho (1 - 1.5 u.u) - 3 (1 - omega/2) u.F - pamp/3, gives
    f*_i' - (216 w_i) r = (1 - omega) d_i + w_i (E_i +/- O_i - 216 omega r): the formula of the
    deviations' collision, checked here in FP64 against the collision on the totals."""
    rng = np.random.default_rng(77)
    c, w, _ = oracle.lattice(oracle.D3Q27)
    k = 216.0 * w
    for _ in range(50):
        omega = rng.uniform(0.6, 1.8)
        guo = 1.0 - 0.5 * omega
        r = np.rint(rng.uniform(0.97, 1.03) / 216.0 * 2.0 ** 24) / 2.0 ** 24
        d = rng.normal(0.0, 3e-3, 27) * w
        t = k * r + d
        rho = rng.uniform(0.97, 1.03)
        F = rng.normal(0.0, 1e-4, 3)
        m = rng.normal(0.0, 1.0, 3)
        m /= np.linalg.norm(m)
        pamp = 0.01 * rng.uniform(0.0, 0.2)
        j_t = c[1:].T @ t[1:]
        j_d = c[1:].T @ d[1:]
        assert np.allclose(j_t, j_d, rtol=0, atol=1e-15)  # the references' momentum is zero
        u = (j_d + 0.5 * F) / rho
        uu, uF = u @ u, u @ F
        cu, cF, cm = c @ u, c @ F, c @ m
        E_core = 4.5 * omega * rho * cu ** 2 + 9 * guo * cu * cF + pamp * cm ** 2
        O = 3 * omega * rho * cu + 3 * guo * cF
        K0 = omega * rho * (1 - 1.5 * uu) - 3 * guo * uF - pamp / 3
        K0d = omega * ((rho - 216 * r) - 1.5 * rho * uu) - 3 * guo * uF - pamp / 3
        fs = (1 - omega) * t + w * (K0 + E_core + O)  # the collision on the totals
        dout = (1 - omega) * d + w * (K0d + E_core + O)  # on the deviations
        assert np.allclose(fs[1:] - k[1:] * r, dout[1:], rtol=0, atol=1e-15)
