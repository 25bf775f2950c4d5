"""Pins of the oracle's boundary rules and droplet statistics (CPU).

The paper prints no boundary conditions (reading R11 of the library: halfway bounce-back,
ports as ghost sites refilled from their inward neighbour x' before every step).  Each rule
is pinned here by what it must produce, so that a plausible slip (a transverse width off by
one, a missing half-site offset, copying from the wrong neighbour, a ghost seen as a wall)
fails a test:

  * velocity inlet: every ghost carries exactly the imposed profile u_max 4s(W-s)/W^2 per
    transverse axis (s = j + 1/2 from the port edge, W = number of port sites), and a
    parabolic inlet into a walled channel is the developed Poiseuille flow at once: the first
    fluid column and every later one carry that profile, with its exact discrete flux;
  * zero-gradient outlet: a ghost is a bit-exact copy of its inward neighbour, and the
    velocity has no outlet-normal gradient at the last column (the pressure outlet, unlike
    the copy, also keeps the flux the same through every column);
  * the psi a ghost feeds into the colour gradient is the psi of its own populations: a red
    inlet into a red box leaves F = 0 everywhere (results independent of A, whatever psi the
    walls carry), and a blue inlet into a red box gives F = (1, 0) at the first column, whose
    perturbation (Eq. 9) is then known in closed form;
  * the per-droplet site counts and volumes of the labelling equal a brute-force count and a
    sequential sum of (1 + psi)/2 over each component, on fields with droplets across
    periodic edges.
"""
import numpy as np
import pytest

import oracle
from paper_1711_02003_gb300 import workloads as W

from test_oracle_label import brute_labels


def _ghosts(pb, port):
    """(ghost sites, inward neighbours) of port `port`."""
    mask = np.asarray(pb.mask).ravel()
    g = np.nonzero(mask == W.PORT0 + port)[0]
    pt = pb.ports[port]
    dims = (pb.nx, pb.ny, pb.nz)
    xyz = np.stack([g % pb.nx, (g // pb.nx) % pb.ny, g // (pb.nx * pb.ny)])
    xyz[pt.normal_axis] += pt.normal_sign
    assert np.all((xyz[pt.normal_axis] >= 0) & (xyz[pt.normal_axis] < dims[pt.normal_axis]))
    return g, xyz[0] + pb.nx * (xyz[1] + pb.ny * xyz[2])


def _moments(f, lattice, sites):
    c, _, _, _ = oracle.tables(lattice)
    tot = f[0][:, sites] + f[1][:, sites]
    rho = tot.sum(axis=0)
    return rho, (c.T.astype(float) @ tot) / rho


def _parabola(W_, j):
    s = j + 0.5
    return 4.0 * s * (W_ - s) / (W_ * W_)


# ----------------------------------------------------------------- velocity inlet profile

@pytest.mark.parametrize("lattice", [W.D2Q9, W.D3Q19])
def test_inlet_ghosts_carry_the_exact_profile(lattice):
    Wd, D, U = 12, 6, 0.02
    pb = W.channel(lattice, 24, Wd, D=D, U=U, profile=W.PARABOLIC, outlet=W.PRESSURE_OUTLET)
    s = oracle.Sim(pb)
    s.step(5)  # every ghost of the returned state has been refilled
    rho, u = _moments(s.populations(), lattice, _ghosts(pb, 0)[0])
    g = _ghosts(pb, 0)[0]
    y = (g // pb.nx) % pb.ny - 1          # port sites start at y = 1 (z = 1)
    z = g // (pb.nx * pb.ny) - 1
    want = U * _parabola(Wd, y) * (_parabola(D, z) if lattice == W.D3Q19 else 1.0)
    assert np.abs(u[0] - want).max() <= 1e-14
    assert np.abs(u[1:]).max() <= 1e-15
    assert np.all(rho > 0.99)


def test_parabolic_inlet_is_developed_poiseuille():
    """Between halfway walls the parabola is the exact steady solution, so a parabolic inlet
    delivers it at the first fluid column and keeps it along the channel; the flux through
    every column equals the discrete sum of the imposed profile."""
    Wd, U = 16, 0.01
    pb = W.channel(W.D2Q9, 64, Wd, U=U, profile=W.PARABOLIC, outlet=W.PRESSURE_OUTLET)
    s = oracle.Sim(pb)
    s.step(6000)
    rr, rb, u = s.fields()
    ux = u[0].reshape(pb.shape)[1:Wd + 1]
    rho = (rr + rb).reshape(pb.shape)[1:Wd + 1]
    prof = U * _parabola(Wd, np.arange(Wd))
    flux = prof.sum()
    for x in (1, 2, 32, pb.nx - 2):
        assert np.abs(ux[:, x] - prof).max() <= 0.01 * U, x
        assert abs((rho[:, x] * ux[:, x]).sum() / flux - 1) <= 5e-3, x


# ------------------------------------------------------------------- zero-gradient outlet

def test_zero_gradient_ghost_copies_inward_neighbour():
    pb = W.channel(W.D3Q19, 20, 8, D=5, U=0.02, profile=W.PARABOLIC, outlet=W.ZERO_GRADIENT_OUTLET)
    x = np.arange(pb.nsites) % pb.nx
    pb = pb.replace(rho_r=pb.rho_r * (1.0 + 0.01 * np.sin(0.7 * x)))  # a state that varies along x
    s = oracle.Sim(pb)
    s.step(7)
    p1 = s.populations()
    s.step(2)
    p2 = s.populations()
    g, xp = _ghosts(pb, 1)
    # the state after step n holds the refill made at step n - 1 from the state after n - 2
    assert np.array_equal(p2[:, :, g], p1[:, :, xp])
    assert not np.array_equal(p2[:, :, g], p1[:, :, xp - 1])


def test_outlet_flux_and_normal_gradient():
    """Developed Poiseuille flow from a parabolic inlet.  Pressure outlet: the flux is the same
    through every column.  Zero-gradient outlet (the ghost copies x', a first-order Neumann
    condition): the velocity has no outlet-normal gradient at the last column, but the copy
    also removes the pressure gradient the flow needs there, so the outlet passes only part
    of the inflow (0.69 at W = 16, 0.94 at W = 64) and mass accumulates in the box."""
    Wd, U = 16, 0.01
    out = {}
    for outlet in (W.PRESSURE_OUTLET, W.ZERO_GRADIENT_OUTLET):
        pb = W.channel(W.D2Q9, 64, Wd, U=U, profile=W.PARABOLIC, outlet=outlet)
        s = oracle.Sim(pb)
        m0 = s.observables((32, 8))["mass_r"]
        s.step(6000)
        rr, rb, u = s.fields()
        ux = u[0].reshape(pb.shape)[1:Wd + 1]
        rho = (rr + rb).reshape(pb.shape)[1:Wd + 1]
        flux = (rho * ux).sum(axis=0)[1:pb.nx - 1]        # every fluid column
        last = pb.nx - 2
        out[outlet] = (flux, ux[:, last] - ux[:, last - 1], s.observables((32, 8))["mass_r"] / m0)
    flux, du, growth = out[W.PRESSURE_OUTLET]
    assert np.abs(flux / flux[0] - 1).max() <= 5e-3
    assert abs(growth - 1) <= 1e-2
    flux, du, growth = out[W.ZERO_GRADIENT_OUTLET]
    assert np.abs(du).max() <= 5e-3 * U
    assert np.all(np.diff(flux) < 0) and 0.6 < flux[-1] / flux[0] < 0.8
    assert growth > 1.1


# --------------------------------------------------------------------- psi at a ghost site

def _open_box(nx=24, ny=10, psi_in=1.0, A=0.02, psi_wall=-1.0, u_in=0.0):
    """Box periodic in y, closed in x by a velocity inlet (x = 0) and a zero-gradient outlet
    (x = nx - 1): no wall site anywhere, red fluid at rest."""
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, :, 0] = W.PORT0
    mask[0, :, nx - 1] = W.PORT0 + 1
    mask = mask.ravel()
    fluid = mask == W.FLUID
    ports = [W.Port(kind=W.VELOCITY_INLET, normal_axis=0, normal_sign=1, profile=W.FLAT, u_max=u_in, psi=psi_in),
             W.Port(kind=W.ZERO_GRADIENT_OUTLET, normal_axis=0, normal_sign=-1, psi=1.0)]
    return W.Problem(lattice=W.D2Q9, nx=nx, ny=ny, nz=1, periodic=(0, 1, 1), A=A, beta=0.7, psi_wall=psi_wall,
                     mask=mask, ports=ports, rho_r=fluid * 1.0, rho_b=fluid * 0.0, name="open box")


@pytest.mark.parametrize("psi_wall", [-1.0, 1.0])
def test_red_inlet_into_red_box_has_no_colour_gradient(psi_wall):
    a = oracle.Sim(_open_box(A=0.05, psi_wall=psi_wall, u_in=0.01))
    b = oracle.Sim(_open_box(A=0.0, psi_wall=psi_wall, u_in=0.01))
    a.step(40)
    b.step(40)
    assert np.array_equal(a.populations(), b.populations())


def test_blue_inlet_gradient_and_perturbation_at_first_column():
    """Step 1: the ghosts (x = 0) hold blue fluid (psi = -1), every site with x >= 2 is still
    red (psi = +1), and the box is uniform in y, so the first column sees
    F = 3 sum_i w_i psi(x + c_i) c_i = (1/2)(psi(2) - psi(0)) x^ = (1, 0).  The perturbation
    (Eq. 9) is the only difference between runs with and without A, and acts on the total
    populations: Delta_i = (A/2)|F| [w_i (F.c_i)^2/|F|^2 - B_i] = (A/2)(w_i c_ix^2 - B_i)."""
    A = 0.02
    a = oracle.Sim(_open_box(psi_in=-1.0, A=A))
    b = oracle.Sim(_open_box(psi_in=-1.0, A=0.0))
    a.step(1)
    b.step(1)
    fa, fb = a.populations(), b.populations()
    first = np.arange(10) * 24 + 1             # x = 1 of every row of the 24 x 10 box
    d = (fa[0] + fa[1])[:, first] - (fb[0] + fb[1])[:, first]
    c, w, _, B = oracle.tables(W.D2Q9)
    want = 0.5 * A * (w * c[:, 0] ** 2 - B)
    assert np.abs(d - want[:, None]).max() <= 1e-15
    assert np.abs(want).max() > 1e-3


# ------------------------------------------------------------ droplet counts and volumes

def _drops_field(shape, centres, radii, seed):
    """psi = +1 inside any of the balls (minimum image), -1 outside, plus small noise."""
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    inside = np.zeros(shape, bool)
    for cen, r in zip(centres, radii):
        d2 = np.zeros(shape)
        for a, n in enumerate(shape):
            dd = np.abs(grids[a] - cen[a])
            dd = np.minimum(dd, n - dd)
            d2 = d2 + dd * dd
        inside |= d2 < r * r
    rng = np.random.default_rng(seed)
    return np.where(inside, 1.0, -1.0) * (1.0 - 0.05 * rng.random(shape))


@pytest.mark.parametrize("lattice", [W.D2Q9, W.D3Q19])
def test_label_counts_and_volumes_brute_force(lattice):
    if lattice == W.D2Q9:
        shape = (48, 64)                       # (y, x)
        centres = [(0, 5), (24, 63), (10, 30), (40, 40), (30, 12), (20, 50)]
        radii = [4, 5, 3.5, 6, 3, 2.5]
        dims = (64, 48)
    else:
        shape = (24, 32, 36)                   # (z, y, x)
        centres = [(0, 0, 0), (12, 16, 34), (6, 24, 12), (18, 8, 20), (12, 26, 26), (5, 8, 22)]
        radii = [4.5, 4, 4, 4.2, 3.8, 4]
        dims = (36, 32, 24)
    psi = _drops_field(shape, centres, radii, 3).ravel()
    pb = W.static_droplet(lattice, dims[0], 2, ny=dims[1], **({"nz": dims[2]} if lattice == W.D3Q19 else {}))
    pb = pb.replace(rho_r=(1 + psi) / 2, rho_b=(1 - psi) / 2)
    s = oracle.Sim(pb)
    s.step(10)                                # diffuse interfaces: (1 + psi)/2 takes many values
    labels, counts, vols, nd = s.label()
    rr, rb, _ = s.fields()
    drop = (rr > rb).astype(np.uint8)
    per = (1,) * len(dims)
    want = brute_labels(dims, per, drop)
    assert np.array_equal(labels, want)
    roots = sorted(set(want[want >= 0].tolist()))
    assert nd == len(roots) >= 5
    half = (1.0 + (rr - rb) / (rr + rb)) / 2.0
    for k, r in enumerate(roots):
        sites = np.nonzero(want == r)[0]        # ascending index order
        assert counts[k] == sites.size
        v = 0.0
        for x in sites:
            v += half[x]
        assert vols[k] == v
    # some droplets wrap a periodic edge and are still one component each
    xs = np.arange(labels.size) % dims[0]
    wrapped = [r for r in roots if {0, dims[0] - 1} <= set(xs[want == r].tolist())]
    assert wrapped
