"""Pins of the FP64 oracle's per-site operators against closed forms.

Each test fixes a part of the method by something other than the oracle itself:
the textbook lattice sets, lattice isotropy, the moment identities implied by
Eqs. 6-8 (equilibrium), Eq. 9 (perturbation), Eq. 10 (recolouring) and Eq. 11
(regularization), and the values the paper prints (tests/golden)."""
import itertools

import numpy as np
import pytest

import oracle

D2Q9, D3Q19 = 0, 1
RNG = np.random.default_rng(12345)


def expected_set(lattice):
    if lattice == D2Q9:
        return {(a, b, 0) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    return {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2}


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_lattice_sets_weights_opposites(lattice):
    c, w, opp, B = oracle.tables(lattice)
    assert {tuple(v) for v in c} == expected_set(lattice)
    assert tuple(c[0]) == (0, 0, 0)
    for i in range(len(c)):
        assert tuple(c[opp[i]]) == tuple(-c[i])
    # textbook weights by speed class (Qian, d'Humieres, Lallemand 1992)
    c2 = (c * c).sum(1)
    ref = {D2Q9: {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}, D3Q19: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}}[lattice]
    for i in range(len(c)):
        assert w[i] == pytest.approx(ref[c2[i]], abs=1e-16)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_lattice_isotropy(lattice):
    c, w, _, _ = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    c = c[:, :d].astype(float)
    I = np.eye(d)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), I / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    c4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(c4, iso, atol=1e-15)


def test_phi_eq7_and_unit_ratio(golden):
    # Eq. 7: rest alpha, axis (1-alpha)/5, diagonal (1-alpha)/20
    alpha = 0.3
    c, w, _, _ = oracle.tables(D2Q9)
    ph = oracle.phi(D2Q9, alpha)
    c2 = (c * c).sum(1)
    for i in range(9):
        exp = {0: alpha, 1: (1 - alpha) / 5, 2: (1 - alpha) / 20}[c2[i]]
        assert ph[i] == pytest.approx(exp, abs=1e-16)
    assert ph.sum() == pytest.approx(1.0, abs=1e-15)
    # alpha = w_0 gives phi = w (density ratio 1)
    assert np.allclose(oracle.phi(D2Q9, 4 / 9), w, atol=1e-16)
    assert np.allclose(oracle.phi(D3Q19, 1 / 3), oracle.tables(D3Q19)[1], atol=1e-16)
    for a in (0.2, 0.5, 0.8):
        assert oracle.phi(D3Q19, a).sum() == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_equilibrium_moments(lattice):
    """Eq. 6 moments: sum f = rho^k; sum f c = rho^k u; sum f c c = p^k I + rho^k u u,
    with p^k from Eq. 8 (D2Q9: 3 rho (1-alpha)/5) or rho (1-alpha)/2 (D3Q19 reading)."""
    c, _, _, _ = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    cf = c[:, :d].astype(float)
    for _ in range(20):
        alpha = RNG.uniform(0.1, 0.9)
        rho = RNG.uniform(0.1, 2.0)
        u = RNG.uniform(-0.1, 0.1, d)
        f = oracle.feq(lattice, alpha, rho, u)
        p = 3 * rho * (1 - alpha) / 5 if lattice == D2Q9 else rho * (1 - alpha) / 2
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(f @ cf, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", f, cf, cf), p * np.eye(d) + rho * np.outer(u, u),
                           atol=1e-14)


def test_equilibrium_pressure_eq8_golden(golden):
    assert golden["pressure_d2q9"]["cite"] == "Eq. 8"
    rho, alpha = 0.7, 0.25
    f = oracle.feq(D2Q9, alpha, rho, [0.0, 0.0])
    c, _, _, _ = oracle.tables(D2Q9)
    pxx = (f * c[:, 0] ** 2).sum()
    assert pxx == pytest.approx(3 * rho * (1 - alpha) / 5, rel=1e-14)


def _hermite2(lattice, Pi):
    c, w, _, _ = oracle.tables(lattice)
    d = Pi.shape[0]
    cf = c[:, :d].astype(float)
    Q = np.einsum("ia,ib->iab", cf, cf) - np.eye(d)[None] / 3.0
    return 4.5 * w * np.einsum("iab,ab->i", Q, Pi)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_reg_equals_bgk_for_second_order_nonequilibrium(lattice):
    """Eq. 11: if f - f^eq lies in the second-order Hermite space, REG == BGK."""
    d = 2 if lattice == D2Q9 else 3
    for _ in range(10):
        rho, u = RNG.uniform(0.5, 1.5), RNG.uniform(-0.05, 0.05, d)
        fe = oracle.feq(lattice, 4 / 9 if lattice == D2Q9 else 1 / 3, rho, u)
        M = RNG.normal(size=(d, d)) * 1e-3
        Pi = M + M.T
        f = fe + _hermite2(lattice, Pi)
        omega = RNG.uniform(0.2, 1.9)
        reg = oracle.relax(lattice, 0, omega, f, fe)
        bgk = oracle.relax(lattice, 1, omega, f, fe)
        assert np.allclose(reg, bgk, atol=1e-15)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_reg_keeps_hydrodynamic_moments_and_filters_ghosts(lattice):
    """REG and BGK outputs share rho, j and Pi; for a generic f they differ (ghost modes filtered)."""
    c, _, _, _ = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    cf = c[:, :d].astype(float)
    a = 4 / 9 if lattice == D2Q9 else 1 / 3
    f = oracle.feq(lattice, a, 1.0, RNG.uniform(-0.05, 0.05, d)) + RNG.normal(size=len(c)) * 1e-3
    rho = f.sum()
    fe = oracle.feq(lattice, a, rho, (f @ cf) / rho)   # equilibrium of f's own moments
    omega = 1 / 5.0
    reg = oracle.relax(lattice, 0, omega, f, fe)
    bgk = oracle.relax(lattice, 1, omega, f, fe)
    assert reg.sum() == pytest.approx(bgk.sum(), abs=1e-15)
    assert np.allclose(reg @ cf, bgk @ cf, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", reg, cf, cf), np.einsum("i,ia,ib->ab", bgk, cf, cf),
                       atol=1e-15)
    assert np.abs(reg - bgk).max() > 1e-5
    # the regularized non-equilibrium is exactly second-order Hermite
    Pi = np.einsum("i,ia,ib->ab", f - fe, cf, cf)
    assert np.allclose(reg - fe, (1 - omega) * _hermite2(lattice, Pi), atol=1e-16)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_perturbation_moments(lattice, golden):
    """Eq. 9: sum Delta = 0, sum Delta c = 0, sum Delta c c = (A/9)|F| (n n - I)."""
    c, _, _, B = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    cf = c[:, :d].astype(float)
    for _ in range(10):
        F = RNG.normal(size=d)
        A = RNG.uniform(0.001, 0.1)
        delta = oracle.perturbation(lattice, A, F)
        fn = np.linalg.norm(F)
        n = F / fn
        assert abs(delta.sum()) < 1e-16
        assert np.allclose(delta @ cf, 0.0, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", delta, cf, cf), A / 9 * fn * (np.outer(n, n) - np.eye(d)),
                           atol=1e-15)
    # below the threshold: no perturbation
    assert np.all(oracle.perturbation(lattice, 0.1, np.full(d, 1e-12)) == 0.0)
    # B_i against the cited colour-gradient values
    key = "B_d2q9" if lattice == D2Q9 else "B_d3q19"
    c2 = (c * c).sum(1)
    names = ["rest", "axis", "diagonal"] if lattice == D2Q9 else ["rest", "face", "edge"]
    for i in range(len(B)):
        assert B[i] == pytest.approx(golden[key][names[c2[i]]], abs=1e-16)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_recolour_invariants_and_direction(lattice):
    """Eq. 10: per-site component masses kept, R + B = f, identity for one component,
    and red is pushed along +F (towards larger psi)."""
    c, w, _, _ = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    a = 4 / 9 if lattice == D2Q9 else 1 / 3
    for _ in range(10):
        rr, rb = RNG.uniform(0.05, 1.0, 2)
        f = oracle.feq(lattice, a, rr + rb, RNG.uniform(-0.05, 0.05, d)) + RNG.normal(size=len(w)) * 1e-3
        F = RNG.normal(size=d)
        beta = RNG.uniform(0.1, 1.0)
        R, Bo = oracle.recolour(lattice, beta, a, a, rr, rb, F, f)
        # sum_i f differs from rr + rb by the noise; masses follow rho^k / rho * sum f
        assert R.sum() == pytest.approx(rr / (rr + rb) * f.sum(), rel=1e-14)
        assert Bo.sum() == pytest.approx(rb / (rr + rb) * f.sum(), rel=1e-14)
        assert np.allclose(R + Bo, f, atol=1e-16)
    R, Bo = oracle.recolour(lattice, 0.7, a, a, 1.0, 0.0, np.ones(d), f)
    assert np.array_equal(R, f) and np.all(Bo == 0.0)
    R, Bo = oracle.recolour(lattice, 0.0, a, a, 0.3, 0.7, np.ones(d), f)
    assert np.allclose(R, 0.3 * f, atol=1e-16)
    F = np.zeros(d)
    F[0] = 1.0
    f0 = oracle.feq(lattice, a, 1.0, np.zeros(d))
    R, _ = oracle.recolour(lattice, 0.7, a, a, 0.5, 0.5, F, f0)
    iplus = [i for i in range(len(w)) if tuple(c[i]) == (1, 0, 0)][0]
    iminus = [i for i in range(len(w)) if tuple(c[i]) == (-1, 0, 0)][0]
    assert R[iplus] > 0.5 * f0[iplus] > R[iminus]
    # segregation term for an axis direction with F along it: beta rho_R rho_B / rho^2 * w_i rho
    assert R[iplus] - 0.5 * f0[iplus] == pytest.approx(0.7 * 0.25 * w[iplus], rel=1e-14)


def test_mixture_relaxation():
    class P:
        lattice, nx, ny, nz, periodic, collision = 0, 1, 1, 1, (1, 1, 1), 0
        tau_r, tau_b, alpha_r, alpha_b, A, beta, rho0, psi_wall = 5.0, 1.0, 4 / 9, 4 / 9, 0.0, 0.7, 1.0, -1.0
    assert oracle.mixture_omega(P, 1.0) == pytest.approx(1 / 5.0, rel=1e-15)
    assert oracle.mixture_omega(P, -1.0) == pytest.approx(1.0, rel=1e-15)
    nu_r, nu_b = 1.5, 1 / 6
    nu = 1.0 / (0.5 / nu_r + 0.5 / nu_b)
    assert oracle.mixture_omega(P, 0.0) == pytest.approx(1.0 / (3 * nu + 0.5), rel=1e-14)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_collision_conserves_component_mass_and_momentum(lattice):
    c, w, _, _ = oracle.tables(lattice)
    d = 2 if lattice == D2Q9 else 3
    a = 4 / 9 if lattice == D2Q9 else 1 / 3

    class P:
        nx = ny = nz = 1
        periodic = (1, 1, 1)
        tau_r, tau_b, alpha_r, alpha_b, A, beta, rho0, psi_wall = 1.3, 0.8, a, a, 0.02, 0.7, 1.0, -1.0
    P.lattice = lattice
    cf = c[:, :d].astype(float)
    for coll in (0, 1):
        P.collision = coll
        for _ in range(10):
            fr = oracle.feq(lattice, a, RNG.uniform(0.1, 1), RNG.uniform(-.05, .05, d)) + RNG.normal(size=len(w)) * 1e-3
            fb = oracle.feq(lattice, a, RNG.uniform(0.1, 1), RNG.uniform(-.05, .05, d)) + RNG.normal(size=len(w)) * 1e-3
            F = RNG.normal(size=d) * 0.1
            R, Bo = oracle.collide(P, fr, fb, F)
            assert R.sum() == pytest.approx(fr.sum(), rel=1e-14)
            assert Bo.sum() == pytest.approx(fb.sum(), rel=1e-14)
            assert np.allclose((R + Bo) @ cf, (fr + fb) @ cf, atol=1e-15)
