"""Seeded synthetic inputs: problem parameters, integer geometry masks and initial fields.

This module holds no arithmetic of the lattice Boltzmann method itself.  It
describes *what* is simulated -- lattice, box, relaxation times, surface-tension
parameter A, recolouring beta, the integer wall/port mask and the initial
densities and velocity -- and both the CUDA library and the FP64 oracle take
these objects as input.  Every generator is deterministic (integer geometry,
seeded splitmix64 where randomness is involved).

Mask codes: 0 fluid, 1 wall, 2 + m ghost site of port m (inlet or outlet).

The workloads mirror the paper's cases:
  * static droplet (Fig. 1 resting droplet; Laplace-law checks),
  * 2D flow-focusing cross junction (Sec. IV A, Figs. 2-3),
  * 3D step emulsifier ("volcano" nozzle, Sec. IV B, Fig. 5),
  * walled channels (Poiseuille) and the shear wave (viscosity check).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

D2Q9 = 0
D3Q19 = 1
REG = 0
BGK = 1

FLUID = 0
WALL = 1
PORT0 = 2

VELOCITY_INLET = 0
PRESSURE_OUTLET = 1
ZERO_GRADIENT_OUTLET = 2

PARABOLIC = 0
FLAT = 1

#: rest weight of each lattice; alpha_k equal to it gives density ratio 1 (Eq. 7)
ALPHA_UNIT_RATIO = {D2Q9: 4.0 / 9.0, D3Q19: 1.0 / 3.0}


@dataclass
class Port:
    """One inlet or outlet.  Its ghost sites carry mask code 2 + index."""

    kind: int = VELOCITY_INLET
    normal_axis: int = 0          # inward normal axis
    normal_sign: int = 1          # inward normal sign
    profile: int = PARABOLIC
    u_max: float = 0.0
    rho: float = 1.0              # inlet density or imposed outlet density
    psi: float = 1.0              # inlet colour: +1 red (dispersed), -1 blue (continuous)


@dataclass
class Problem:
    """A complete simulation input: parameters, geometry and initial fields."""

    lattice: int = D2Q9
    nx: int = 64
    ny: int = 64
    nz: int = 1
    periodic: tuple = (1, 1, 1)
    tau_r: float = 1.0
    tau_b: float = 1.0
    alpha_r: float = 4.0 / 9.0
    alpha_b: float = 4.0 / 9.0
    A: float = 0.01
    beta: float = 0.7
    rho0: float = 1.0
    psi_wall: float = -1.0
    collision: int = REG
    mask: np.ndarray = None       # uint8, shape (nz, ny, nx) flattened x-fastest
    ports: list = field(default_factory=list)
    rho_r: np.ndarray = None      # float64 per site
    rho_b: np.ndarray = None
    u: np.ndarray = None          # float64 (dim, nsites) or None for rest
    name: str = ""

    @property
    def dim(self) -> int:
        return 2 if self.lattice == D2Q9 else 3

    @property
    def q(self) -> int:
        return 9 if self.lattice == D2Q9 else 19

    @property
    def nsites(self) -> int:
        return self.nx * self.ny * (self.nz if self.lattice == D3Q19 else 1)

    @property
    def shape(self) -> tuple:
        """numpy shape of a per-site field (z, y, x) or (y, x)."""
        if self.lattice == D2Q9:
            return (self.ny, self.nx)
        return (self.nz, self.ny, self.nx)

    def fluid_sites(self) -> int:
        return int(np.count_nonzero(self.mask == FLUID))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------- rng

def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of the splitmix64 generator started at `seed` (uint64)."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & 0xFFFFFFFFFFFFFFFF
    m = 0xFFFFFFFFFFFFFFFF
    for k in range(n):
        s = (s + 0x9E3779B97F4A7C15) & m
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out[k] = z ^ (z >> 31)
    return out


def _uniform(seed: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) / float(1 << 53)


# ------------------------------------------------------------------- fields

def _two_phase_fields(psi: np.ndarray, rho0: float, mask: np.ndarray):
    """Sharp initial colour field psi = +-1 -> component densities at rest."""
    psi = psi.astype(np.float64).ravel()
    fluid = mask.ravel() == FLUID
    rho_r = np.where(fluid, rho0 * (1.0 + psi) / 2.0, 0.0)
    rho_b = np.where(fluid, rho0 * (1.0 - psi) / 2.0, 0.0)
    return rho_r, rho_b


def static_droplet(lattice: int = D2Q9, n: int = 64, R: float = 16, *, nz: int | None = None,
                   tau_r: float = 1.0, tau_b: float = 1.0, A: float = 0.01, beta: float = 0.7,
                   rho0: float = 1.0, collision: int = REG, ny: int | None = None,
                   centre=None, density_ratio: float = 1.0) -> Problem:
    """Centred resting droplet in a fully periodic box (Fig. 1 setting).

    psi = +1 strictly inside (integer test (x-xc)^2 + (y-yc)^2 [+ (z-zc)^2] < R^2,
    default centre n/2), -1 outside; rho_R = rho0 (1+psi)/2, rho_B = rho0 (1-psi)/2,
    fluid at rest.  density_ratio = gamma != 1: the droplet (red) holds gamma * rho0, the
    surrounding fluid rho0, and alpha_R = 1 - (1 - alpha_B) / gamma with alpha_B the unit-
    ratio value, so that the two bulk pressures of Eq. 8 (proportional to rho^k (1 - alpha_k))
    are equal."""
    nx = n
    ny = n if ny is None else ny
    if lattice == D2Q9:
        nzz = 1
    else:
        nzz = n if nz is None else nz
    cx, cy, cz = (nx // 2, ny // 2, nzz // 2) if centre is None else centre
    z, y, x = np.meshgrid(np.arange(nzz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    if lattice == D3Q19:
        r2 = r2 + (z - cz) ** 2
    psi = np.where(r2 < R * R, 1.0, -1.0)
    mask = np.zeros(nx * ny * nzz, dtype=np.uint8)
    rho_r, rho_b = _two_phase_fields(psi, rho0, mask)
    alpha = ALPHA_UNIT_RATIO[lattice]
    alpha_r = alpha
    if density_ratio != 1.0:
        rho_r = rho_r * density_ratio
        alpha_r = 1.0 - (1.0 - alpha) / density_ratio
    tag = "" if density_ratio == 1.0 else f" ratio={density_ratio:g}"
    return Problem(lattice=lattice, nx=nx, ny=ny, nz=nzz, periodic=(1, 1, 1), tau_r=tau_r, tau_b=tau_b,
                   alpha_r=alpha_r, alpha_b=alpha, A=A, beta=beta, rho0=rho0, collision=collision,
                   mask=mask, ports=[], rho_r=rho_r, rho_b=rho_b, u=None,
                   name=f"static droplet {'D2Q9' if lattice == D2Q9 else 'D3Q19'} n={n} R={R}{tag}")


def shear_wave(lattice: int = D2Q9, n: int = 32, U: float = 1e-3, tau: float = 1.0) -> Problem:
    """Single-phase (rho_B = 0, psi = 1) periodic shear wave u_x = U sin(2 pi y / n)."""
    nx = ny = n
    nzz = 1 if lattice == D2Q9 else 4
    nsite = nx * ny * nzz
    mask = np.zeros(nsite, dtype=np.uint8)
    y = np.broadcast_to(np.arange(ny)[None, :, None], (nzz, ny, nx)).ravel()
    u = np.zeros((2 if lattice == D2Q9 else 3, nsite))
    u[0] = U * np.sin(2.0 * np.pi * y / ny)
    alpha = ALPHA_UNIT_RATIO[lattice]
    return Problem(lattice=lattice, nx=nx, ny=ny, nz=nzz, periodic=(1, 1, 1), tau_r=tau, tau_b=tau,
                   alpha_r=alpha, alpha_b=alpha, A=0.0, beta=0.7, mask=mask,
                   rho_r=np.ones(nsite), rho_b=np.zeros(nsite), u=u, name=f"shear wave n={n} tau={tau}")


def channel(lattice: int = D2Q9, nx: int = 64, W: int = 16, *, D: int = 8, U: float = 0.01,
            profile: int = FLAT, tau: float = 1.0, outlet: int = ZERO_GRADIENT_OUTLET,
            two_phase: bool = False, A: float = 0.0, beta: float = 0.7) -> Problem:
    """Walled channel along x: velocity inlet at x = 0, outlet at x = nx-1.

    2D: fluid y in [1, W], walls at y = 0 and y = W+1.  3D: fluid y in [1, W],
    z in [1, D], walls around.  Single phase (psi = +1) unless two_phase, in which
    case the inlet injects red into a blue-filled channel."""
    if lattice == D2Q9:
        ny, nzz = W + 2, 1
    else:
        ny, nzz = W + 2, D + 2
    mask = np.full((nzz, ny, nx), WALL, dtype=np.uint8)
    if lattice == D2Q9:
        mask[0, 1:W + 1, 1:nx - 1] = FLUID
        mask[0, 1:W + 1, 0] = PORT0 + 0
        mask[0, 1:W + 1, nx - 1] = PORT0 + 1
    else:
        mask[1:D + 1, 1:W + 1, 1:nx - 1] = FLUID
        mask[1:D + 1, 1:W + 1, 0] = PORT0 + 0
        mask[1:D + 1, 1:W + 1, nx - 1] = PORT0 + 1
    mask = mask.ravel()
    psi_in = 1.0
    ports = [Port(kind=VELOCITY_INLET, normal_axis=0, normal_sign=1, profile=profile, u_max=U, rho=1.0,
                  psi=psi_in),
             Port(kind=outlet, normal_axis=0, normal_sign=-1, rho=1.0, psi=-1.0)]
    if two_phase:
        psi0 = np.full(mask.shape, -1.0)
    else:
        psi0 = np.full(mask.shape, 1.0)
    rho_r, rho_b = _two_phase_fields(psi0, 1.0, mask)
    alpha = ALPHA_UNIT_RATIO[lattice]
    return Problem(lattice=lattice, nx=nx, ny=ny, nz=nzz, periodic=(0, 0, 0), tau_r=tau, tau_b=tau,
                   alpha_r=alpha, alpha_b=alpha, A=A, beta=beta, psi_wall=-1.0 if two_phase else 1.0,
                   mask=mask, ports=ports, rho_r=rho_r, rho_b=rho_b, u=None,
                   name=f"channel nx={nx} W={W}")


def cross_junction(nx: int = 1024, channel_w: int = 64, side_x: int = 256, side_len: int = 64, *,
                   u_disp: float = 0.005, u_cont: float = 0.005, tau_cont: float = 1.0,
                   tau_disp: float = 1.0, A: float = 0.01, beta: float = 0.7,
                   outlet: int = ZERO_GRADIENT_OUTLET, fill_x: int = 200) -> Problem:
    """2D flow-focusing cross junction (Sec. IV A).

    Box nx x (2*side_len + channel_w).  Main channel y in [side_len, side_len+channel_w),
    x in [1, nx-1); two side channels x in [side_x, side_x+channel_w) running to the box
    edges.  Ports: 0 dispersed (red) inlet at x = 0, 1 and 2 continuous (blue) inlets at
    y = 0 and y = ny-1, 3 outlet at x = nx-1.  Initially blue everywhere except red in
    the main channel for x < fill_x.  Red is the dispersed phase (tau_r = tau_disp)."""
    ny = 2 * side_len + channel_w
    y0, y1 = side_len, side_len + channel_w
    sx0, sx1 = side_x, side_x + channel_w
    m = np.full((ny, nx), WALL, dtype=np.uint8)
    m[y0:y1, 1:nx - 1] = FLUID
    m[1:y0, sx0:sx1] = FLUID
    m[y1:ny - 1, sx0:sx1] = FLUID
    m[y0:y1, 0] = PORT0 + 0
    m[0, sx0:sx1] = PORT0 + 1
    m[ny - 1, sx0:sx1] = PORT0 + 2
    m[y0:y1, nx - 1] = PORT0 + 3
    ports = [Port(VELOCITY_INLET, 0, +1, PARABOLIC, u_disp, 1.0, 1.0),
             Port(VELOCITY_INLET, 1, +1, PARABOLIC, u_cont, 1.0, -1.0),
             Port(VELOCITY_INLET, 1, -1, PARABOLIC, u_cont, 1.0, -1.0),
             Port(outlet, 0, -1, PARABOLIC, 0.0, 1.0, -1.0)]
    psi = -np.ones((ny, nx))
    psi[y0:y1, :fill_x] = 1.0
    mask = m.ravel()
    rho_r, rho_b = _two_phase_fields(psi, 1.0, mask)
    a = ALPHA_UNIT_RATIO[D2Q9]
    return Problem(lattice=D2Q9, nx=nx, ny=ny, nz=1, periodic=(0, 0, 0), tau_r=tau_disp, tau_b=tau_cont,
                   alpha_r=a, alpha_b=a, A=A, beta=beta, psi_wall=-1.0, mask=mask, ports=ports,
                   rho_r=rho_r, rho_b=rho_b, u=None, name=f"cross junction {nx}x{ny}")


def step_emulsifier(nx: int = 768, ny: int = 128, nz: int = 32, *, terrace_len: int = 256,
                    terrace_h: int = 8, u_in: float = 0.002, tau_cont: float = 1.0,
                    tau_disp: float = 1.0, A: float = 0.01, beta: float = 0.7,
                    outlet: int = PRESSURE_OUTLET, fill_x: int | None = None, seed: int = 0,
                    roughness: int = 0, nozzle_w: int | None = None) -> Problem:
    """3D step emulsifier ("volcano" nozzle, Sec. IV B, Fig. 5).

    Box nx x ny x nz.  Walls at y = 0, y = ny-1, z = 0 and z = nz-1.  Terrace for
    x < terrace_len: fluid z in [1, 1+terrace_h), solid above.  Reservoir for
    x >= terrace_len: full height.  Port 0: red (dispersed) velocity inlet at x = 0
    over the terrace cross-section; port 1: outlet at x = nx-1 over the reservoir.
    `roughness` seeded single-site bumps are placed on the reservoir floor.  `nozzle_w`: the
    terrace (and the inlet) only `nozzle_w` sites wide, centred in y (a single nozzle);
    default the full channel width."""
    m = np.full((nz, ny, nx), WALL, dtype=np.uint8)
    zt = 1 + terrace_h
    ya, yb = 1, ny - 1
    if nozzle_w is not None:
        ya = max(1, (ny - nozzle_w) // 2)
        yb = min(ny - 1, ya + nozzle_w)
    m[1:zt, ya:yb, 1:terrace_len] = FLUID
    m[1:nz - 1, 1:ny - 1, terrace_len:nx - 1] = FLUID
    m[1:zt, ya:yb, 0] = PORT0 + 0
    m[1:nz - 1, 1:ny - 1, nx - 1] = PORT0 + 1
    if roughness:
        r = splitmix64(seed, 2 * roughness)
        for k in range(roughness):
            x = terrace_len + 4 + int(r[2 * k] % np.uint64(max(1, nx - terrace_len - 8)))
            y = 2 + int(r[2 * k + 1] % np.uint64(max(1, ny - 4)))
            m[1, y, x] = WALL
    ports = [Port(VELOCITY_INLET, 0, +1, PARABOLIC, u_in, 1.0, 1.0),
             Port(outlet, 0, -1, PARABOLIC, 0.0, 1.0, -1.0)]
    psi = -np.ones((nz, ny, nx))
    fx = terrace_len // 2 if fill_x is None else fill_x
    psi[:, :, :fx] = 1.0
    mask = m.ravel()
    rho_r, rho_b = _two_phase_fields(psi, 1.0, mask)
    a = ALPHA_UNIT_RATIO[D3Q19]
    return Problem(lattice=D3Q19, nx=nx, ny=ny, nz=nz, periodic=(0, 0, 0), tau_r=tau_disp, tau_b=tau_cont,
                   alpha_r=a, alpha_b=a, A=A, beta=beta, psi_wall=-1.0, mask=mask, ports=ports,
                   rho_r=rho_r, rho_b=rho_b, u=None, name=f"step emulsifier {nx}x{ny}x{nz}")


def random_request(seed: int) -> dict:
    """One serving request of the mixed workload: lattice, size, geometry kind,
    Capillary number (log-uniform 1e-3..1e-1), viscosity ratio (1..10) and step
    count (log-uniform 2e3..2e4), all drawn from splitmix64(seed)."""
    r = _uniform(seed, 8)
    is3d = r[0] >= 0.5
    if not is3d:
        nx = [128, 256, 512, 1024][int(r[1] * 4)]
        ny = [32, 64, 128][int(r[2] * 3)]
        nz = 1
    else:
        nx = [64, 128, 256][int(r[1] * 3)]
        ny = [32, 64][int(r[2] * 2)]
        nz = [16, 32][int(r[3] * 2)]
    geom = "junction" if r[4] < 0.5 else "step"
    ca = 10.0 ** (-3.0 + 2.0 * r[5])
    visc_ratio = 1.0 + 9.0 * r[6]
    steps = int(round(10.0 ** (np.log10(2e3) + r[7] * (np.log10(2e4) - np.log10(2e3)))))
    return dict(lattice=D3Q19 if is3d else D2Q9, nx=nx, ny=ny, nz=nz, geom=geom, ca=ca,
                visc_ratio=visc_ratio, steps=steps, seed=seed)


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of n requests with exponential gaps of mean 1/rate."""
    u = _uniform(seed ^ 0x5DEECE66D, n)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)


def step_channel_2d(nx: int = 256, ny: int = 64, *, terrace_frac: float = 1 / 3, terrace_h: int | None = None,
                    u_in: float = 0.002, tau_cont: float = 1.0, tau_disp: float = 1.0, A: float = 0.01,
                    beta: float = 0.7) -> Problem:
    """2D step emulsifier: a shallow terrace (height ny/4) opening into a full-height reservoir;
    red velocity inlet over the terrace at x = 0, pressure outlet at x = nx-1."""
    th = max(2, ny // 4) if terrace_h is None else terrace_h
    tl = max(4, int(nx * terrace_frac))
    m = np.full((ny, nx), WALL, dtype=np.uint8)
    m[1:1 + th, 1:tl] = FLUID
    m[1:ny - 1, tl:nx - 1] = FLUID
    m[1:1 + th, 0] = PORT0 + 0
    m[1:ny - 1, nx - 1] = PORT0 + 1
    ports = [Port(VELOCITY_INLET, 0, +1, PARABOLIC, u_in, 1.0, 1.0), Port(PRESSURE_OUTLET, 0, -1, PARABOLIC, 0.0, 1.0, -1.0)]
    psi = -np.ones((ny, nx))
    psi[:, :tl // 2] = 1.0
    mask = m.ravel()
    rho_r, rho_b = _two_phase_fields(psi, 1.0, mask)
    a = ALPHA_UNIT_RATIO[D2Q9]
    return Problem(lattice=D2Q9, nx=nx, ny=ny, nz=1, periodic=(0, 0, 0), tau_r=tau_disp, tau_b=tau_cont, alpha_r=a,
                   alpha_b=a, A=A, beta=beta, psi_wall=-1.0, mask=mask, ports=ports, rho_r=rho_r, rho_b=rho_b,
                   u=None, name=f"2D step channel {nx}x{ny}")


def cross_junction_3d(nx: int = 128, ny: int = 64, nz: int = 16, *, u_disp: float = 0.002, u_cont: float = 0.002,
                      tau_cont: float = 1.0, tau_disp: float = 1.0, A: float = 0.01, beta: float = 0.7) -> Problem:
    """The 2D cross junction extruded in z between walls at z = 0 and z = nz-1 (channel depth nz-2)."""
    cw = max(4, ny // 3)
    sl = max(2, (ny - cw) // 2)
    nyy = 2 * sl + cw
    base = cross_junction(nx=nx, channel_w=cw, side_x=max(2, nx // 4), side_len=sl, u_disp=u_disp, u_cont=u_cont,
                          tau_cont=tau_cont, tau_disp=tau_disp, A=A, beta=beta, fill_x=max(2, nx // 5))
    m2 = base.mask.reshape(nyy, nx)
    m = np.full((nz, nyy, nx), WALL, dtype=np.uint8)
    m[1:nz - 1] = m2[None]
    psi2 = np.where(base.rho_r.reshape(nyy, nx) > 0.5, 1.0, -1.0)
    psi = np.broadcast_to(psi2[None], (nz, nyy, nx))
    mask = m.ravel()
    rho_r, rho_b = _two_phase_fields(psi, 1.0, mask)
    a = ALPHA_UNIT_RATIO[D3Q19]
    return Problem(lattice=D3Q19, nx=nx, ny=nyy, nz=nz, periodic=(0, 0, 0), tau_r=tau_disp, tau_b=tau_cont,
                   alpha_r=a, alpha_b=a, A=A, beta=beta, psi_wall=-1.0, mask=mask, ports=list(base.ports),
                   rho_r=rho_r, rho_b=rho_b, u=None, name=f"3D cross junction {nx}x{nyy}x{nz}")


def serving_problem(spec: dict, A: float = 0.01, tau_cont: float = 1.0) -> Problem:
    """The Problem of one serving request (random_request).  Continuous phase tau = tau_cont;
    dispersed viscosity = visc_ratio x continuous; inlet speed U from Ca = rho nu U / sigma with
    sigma = 2 A tau_cont / 9 (the Laplace-law closed form), clipped to [1e-4, 0.02]."""
    nu_c = (tau_cont - 0.5) / 3.0
    tau_d = 0.5 + 3.0 * nu_c * spec["visc_ratio"]
    sigma = 2.0 * A * tau_cont / 9.0
    U = float(np.clip(spec["ca"] * sigma / nu_c, 1e-4, 0.02))
    nx, ny, nz = spec["nx"], spec["ny"], spec["nz"]
    if spec["lattice"] == D2Q9:
        if spec["geom"] == "junction":
            cw = max(4, ny // 3)
            sl = max(2, (ny - cw) // 2)
            pb = cross_junction(nx=nx, channel_w=cw, side_x=max(2, nx // 4), side_len=sl, u_disp=U, u_cont=U,
                                tau_cont=tau_cont, tau_disp=tau_d, A=A, fill_x=max(2, nx // 5))
        else:
            pb = step_channel_2d(nx, ny, u_in=U, tau_cont=tau_cont, tau_disp=tau_d, A=A)
    else:
        if spec["geom"] == "junction":
            pb = cross_junction_3d(nx, ny, nz, u_disp=U, u_cont=U, tau_cont=tau_cont, tau_disp=tau_d, A=A)
        else:
            pb = step_emulsifier(nx, ny, nz, terrace_len=max(4, nx // 3), terrace_h=max(2, nz // 4), u_in=U,
                                 tau_cont=tau_cont, tau_disp=tau_d, A=A, fill_x=max(2, nx // 6), seed=spec["seed"])
    return pb.replace(name=f"request {spec['seed']}: {pb.name}, Ca {spec['ca']:.2e}, ratio {spec['visc_ratio']:.2f}")


# Named single-instance workloads (benchmark and profiling runs): name -> (problem,
# description, a site inside the dispersed phase for the observables)
NAMED = ("step_emulsifier", "flow_focuser", "droplet2d", "droplet3d")


def named(name: str):
    if name == "step_emulsifier":
        return (step_emulsifier(), "3D step emulsifier D3Q19 768x128x32 (terrace 256x126x8, reservoir 512x126x30)",
                (384, 64, 16))
    if name == "flow_focuser":
        return (cross_junction(), "2D flow-focusing cross junction D2Q9 1024x192 (main channel 64, side inlets 64 "
                "at x=256)", (512, 96))
    if name == "droplet2d":
        return static_droplet(D2Q9, 4096, 512), "2D static droplet D2Q9 4096x4096 periodic, R=512", (2048, 2048)
    if name == "droplet3d":
        c = (127.5, 127.5, 127.5)
        return (static_droplet(D3Q19, 256, 64, centre=c), "3D static droplet D3Q19 256^3 periodic, R=64 (off-site "
                "centre)", c)
    raise ValueError(f"unknown workload {name}; known: {', '.join(NAMED)}")
