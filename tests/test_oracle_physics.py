"""Whole-step pins of the FP64 oracle: conservation, symmetry, the paper's printed
viscosities, the Poiseuille profile, the Laplace law, interface width and the
regularized-vs-BGK spurious-current reduction (Fig. 1)."""
import numpy as np
import pytest

import oracle
from paper_1711_02003_gb300 import workloads as W


def _psi(rr, rb):
    return (rr - rb) / (rr + rb)


def test_mass_conservation_periodic_2d():
    s = oracle.Sim(W.static_droplet(W.D2Q9, 64, 16))
    o0 = s.observables((32, 32))
    s.step(2000)
    o1 = s.observables((32, 32))
    assert abs(o1["mass_r"] / o0["mass_r"] - 1) < 1e-12
    assert abs(o1["mass_b"] / o0["mass_b"] - 1) < 1e-12
    assert np.abs(o1["mom"]).max() < 1e-11


def test_mass_conservation_walls_3d():
    pb = W.static_droplet(W.D3Q19, 16, 5, tau_r=1.4, tau_b=0.8)
    m = np.zeros(pb.shape, np.uint8)
    m[0, :, :] = m[-1, :, :] = m[:, 0, :] = m[:, -1, :] = m[:, :, 0] = m[:, :, -1] = W.WALL
    fl = m.ravel() == W.FLUID
    pb = pb.replace(mask=m.ravel(), periodic=(0, 0, 0), rho_r=pb.rho_r * fl, rho_b=pb.rho_b * fl)
    s = oracle.Sim(pb)
    o0 = s.observables((8, 8, 8))
    s.step(300)
    o1 = s.observables((8, 8, 8))
    assert abs(o1["mass_r"] / o0["mass_r"] - 1) < 1e-12
    assert abs(o1["mass_b"] / o0["mass_b"] - 1) < 1e-12


def test_reflection_and_transpose_symmetry_2d():
    n = 64
    s = oracle.Sim(W.static_droplet(W.D2Q9, n, 13, tau_r=1.3, tau_b=0.9))
    s.step(300)
    rr, rb, u = s.fields()
    rr = rr.reshape(n, n)
    ref = np.roll(rr[:, ::-1], 1, axis=1)       # x -> n - x (mod n)
    assert np.abs(rr - ref).max() < 1e-13
    ref = np.roll(rr[::-1, :], 1, axis=0)       # y -> n - y
    assert np.abs(rr - ref).max() < 1e-13
    assert np.abs(rr - rr.T).max() < 1e-13      # x <-> y
    ux = u[0].reshape(n, n)
    assert np.abs(ux + np.roll(ux[:, ::-1], 1, axis=1)).max() < 1e-15


def test_permutation_symmetry_3d():
    n = 20
    s = oracle.Sim(W.static_droplet(W.D3Q19, n, 6))
    s.step(60)
    rr, _, _ = s.fields()
    rr = rr.reshape(n, n, n)
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.abs(rr - rr.transpose(perm)).max() < 1e-13


def test_periodic_shift_is_exact():
    pb = W.static_droplet(W.D2Q9, 48, 11, centre=(20, 23, 0), tau_r=1.2, tau_b=0.9)
    sh = (5, -7)

    def roll(a):
        return np.roll(a.reshape(48, 48), sh, axis=(0, 1)).ravel()
    a = oracle.Sim(pb)
    b = oracle.Sim(pb.replace(rho_r=roll(pb.rho_r), rho_b=roll(pb.rho_b)))
    a.step(80)
    b.step(80)
    fa, fb = a.populations(), b.populations()
    for k in range(2):
        for i in range(9):
            assert np.array_equal(roll(fa[k, i]), fb[k, i])


def _shear_nu(lattice, tau, n, collision=W.REG):
    pb = W.shear_wave(lattice, n, 1e-3, tau).replace(collision=collision)
    s = oracle.Sim(pb)
    k = 2 * np.pi / n
    steps = max(10, int(0.5 / ((tau - 0.5) / 3 * k * k)))
    y = np.broadcast_to(np.arange(pb.ny)[None, :, None], (pb.nz, pb.ny, pb.nx)).ravel()
    sn = np.sin(k * y)

    def amp():
        return (s.fields()[2][0] * sn).sum() / (sn * sn).sum()
    s.step(20)
    a0 = amp()
    s.step(steps)
    return -np.log(amp() / a0) / (k * k * steps)


@pytest.mark.parametrize("key,n", [("nu_tau1", 32), ("nu_flow_focuser_dispersed", 64), ("nu_tau5", 128)])
def test_viscosity_matches_paper(golden, key, n):
    """nu = (tau - 1/2)/3 gives the paper's printed 0.167 (tau 1), 0.5 (tau 2), 1.5 (tau 5)."""
    g = golden[key]
    nu = _shear_nu(W.D2Q9, g["tau"], n)
    assert abs(nu - g["nu"]) <= max(g["tol"], 0.02 * g["nu"])


def test_viscosity_3d():
    nu = _shear_nu(W.D3Q19, 1.0, 32)
    assert abs(nu - 1 / 6) < 1e-4


def test_poiseuille_profile_second_order():
    """Flat inlet -> developed parabola (mean U) between halfway walls; shape error
    converges at second order in W; mass flux is the same along the channel."""
    errs = []
    for Wd, steps in ((16, 6000), (32, 16000)):
        pb = W.channel(W.D2Q9, 96, Wd, U=0.01, outlet=W.PRESSURE_OUTLET)
        s = oracle.Sim(pb)
        s.step(steps)
        rr, rb, u = s.fields()
        ux = u[0].reshape(pb.shape)
        rho = (rr + rb).reshape(pb.shape)
        prof = ux[1:Wd + 1, 72]
        sc = np.arange(Wd) + 0.5
        par = sc * (Wd - sc)
        errs.append(np.abs(prof / prof.mean() - par / par.mean()).max() / (par.max() / par.mean()))
        f24 = (rho[1:Wd + 1, 24] * ux[1:Wd + 1, 24]).sum()
        f72 = (rho[1:Wd + 1, 72] * prof).sum()
        assert abs(f24 / f72 - 1) < 5e-3
        assert abs(f72 / (0.01 * Wd) - 1) < 0.03
    assert errs[0] < 5e-3 and errs[1] < 1.5e-3
    assert errs[0] / errs[1] > 3.0


def test_pressure_outlet_sets_density():
    pb = W.channel(W.D2Q9, 64, 16, U=0.005, outlet=W.PRESSURE_OUTLET)
    s = oracle.Sim(pb)
    s.step(3000)
    rr, rb, _ = s.fields()
    rho = (rr + rb).reshape(pb.shape)
    assert np.abs(rho[1:17, pb.nx - 2] - 1.0).max() < 2e-3
    assert rho[8, 2] > rho[8, pb.nx - 2]      # pressure falls along the flow


def test_laplace_law_2d():
    """Delta p = sigma / R with sigma = 2 A tau / 9: the perturbation adds the stress
    (A/9)|F|(n n - I) each step (Eq. 9), relaxation keeps it for tau steps on
    average, and the integral of |grad psi| across the interface is 2."""
    A, tau = 0.01, 2.0
    sigma = 2 * A * tau / 9
    errs = []
    for R in (8, 12, 16):
        s = oracle.Sim(W.static_droplet(W.D2Q9, 64, R, tau_r=tau, tau_b=tau, A=A))
        s.step(3000)
        o = s.observables((32, 32))
        assert o["dp"] > 0
        errs.append(abs(o["dp"] * o["r_eff"] / sigma - 1))
    assert max(errs) < 0.06
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("ratio", [2.0, 5.0])
def test_laplace_law_density_ratio(ratio):
    """Density ratio gamma != 1 through alpha_k (Eqs. 7-8): the droplet holds gamma times the
    surrounding density with alpha_R chosen for equal bulk pressures.  The surface stress of
    Eq. 9 depends on psi alone (+-1 in both bulks whatever the densities), so the same
    sigma = 2 A tau / 9 must give Delta p = sigma / R; component masses stay conserved."""
    A, tau = 0.01, 1.0
    sigma = 2 * A * tau / 9
    pb = W.static_droplet(W.D2Q9, 48, 12, A=A, tau_r=tau, tau_b=tau, density_ratio=ratio)
    assert pb.alpha_r > pb.alpha_b
    s = oracle.Sim(pb)
    o0 = s.observables((24, 24))
    s.step(3000)
    o = s.observables((24, 24))
    assert o["dp"] > 0
    assert abs(o["dp"] * o["r_eff"] / sigma - 1) < 0.06
    assert abs(o["mass_r"] / o0["mass_r"] - 1) < 1e-12
    assert abs(o["mass_b"] / o0["mass_b"] - 1) < 1e-12


def test_laplace_law_3d():
    A, tau = 0.01, 2.0
    sigma = 2 * A * tau / 9
    s = oracle.Sim(W.static_droplet(W.D3Q19, 32, 8, tau_r=tau, tau_b=tau, A=A))
    s.step(500)
    o = s.observables((16, 16, 16))
    assert abs(o["dp"] * o["r_eff"] / 2 / sigma - 1) < 0.08


def test_interface_width_and_segregation(golden):
    s = oracle.Sim(W.static_droplet(W.D2Q9, 64, 16))
    s.step(2000)
    rr, rb, _ = s.fields()
    psi = _psi(rr, rb).reshape(64, 64)
    width = np.sum(np.abs(psi[32]) < 0.9) / 2
    g = golden["interface_width_lu"]
    assert g["lo"] <= width <= g["hi"]
    assert psi[32, 32] > 0.99 and psi[0, 0] < -0.99


def test_regularization_reduces_spurious_currents(golden):
    """Fig. 1: resting droplet, tau 1 (continuous) and 5 (droplet): REG max|u| well below BGK."""
    g = golden["spurious_current_reduction"]
    umax = {}
    for coll in (W.REG, W.BGK):
        s = oracle.Sim(W.static_droplet(W.D2Q9, 64, 16, tau_r=g["tau_droplet"], tau_b=g["tau_continuous"],
                                        collision=coll))
        s.step(3000)
        umax[coll] = s.observables((32, 32))["umax"]
    assert umax[W.BGK] / umax[W.REG] >= g["soft_min"]


def test_threads_do_not_change_results():
    pb = W.cross_junction(nx=96, channel_w=16, side_x=32, side_len=12, fill_x=20)
    n0 = oracle.threads()
    try:
        oracle.set_threads(1)
        a = oracle.Sim(pb)
        a.step(50)
        oracle.set_threads(max(2, n0))
        b = oracle.Sim(pb)
        b.step(50)
        assert np.array_equal(a.populations(), b.populations())
    finally:
        oracle.set_threads(n0)
