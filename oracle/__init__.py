"""Python access to the FP64 CPU oracle (rcg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it to check and time the CUDA library.  It never imports
the CUDA library, and the CUDA library never imports it.  Inputs are plain
numpy arrays plus any object carrying the problem attributes (lattice, nx, ny,
nz, periodic, tau_r, tau_b, alpha_r, alpha_b, A, beta, rho0, psi_wall,
collision, mask, ports, rho_r, rho_b, u).

Parity pins: every function here is checked by tests/test_oracle_*.py against
closed forms, invariants and the paper's printed values (see the test files);
no function is "parity unpinned" except the absolute surface tension sigma(A),
which the paper does not print (it is calibrated from the Laplace fit).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile rcg_oracle.c into liboracle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3), ("collision", C.c_int),
                ("tau_r", C.c_double), ("tau_b", C.c_double), ("alpha_r", C.c_double),
                ("alpha_b", C.c_double), ("A", C.c_double), ("beta", C.c_double),
                ("rho0", C.c_double), ("psi_wall", C.c_double)]


class _Port(C.Structure):
    _fields_ = [("kind", C.c_int), ("normal_axis", C.c_int), ("normal_sign", C.c_int),
                ("profile", C.c_int), ("u_max", C.c_double), ("rho", C.c_double), ("psi", C.c_double)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_lattice_tables.argtypes = [C.c_int, _ip, _dp, _ip, _dp]
            L.orc_phi.argtypes = [C.c_int, C.c_double, _dp]
            L.orc_feq.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp]
            L.orc_relax.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
            L.orc_perturbation.argtypes = [C.c_int, C.c_double, _dp, _dp]
            L.orc_recolour.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _dp, _dp, _dp, _dp]
            L.orc_mixture_omega.argtypes = [C.POINTER(_Params), C.c_double]
            L.orc_mixture_omega.restype = C.c_double
            L.orc_collide.argtypes = [C.POINTER(_Params), _dp, _dp, _dp, _dp, _dp]
            L.orc_sim_create.argtypes = [C.POINTER(_Params), _u8p, C.POINTER(_Port), C.c_int]
            L.orc_sim_create.restype = C.c_void_p
            L.orc_sim_destroy.argtypes = [C.c_void_p]
            L.orc_sim_init_fields.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p]
            L.orc_sim_set_populations.argtypes = [C.c_void_p, _dp]
            L.orc_sim_get_populations.argtypes = [C.c_void_p, _dp]
            L.orc_sim_step.argtypes = [C.c_void_p, C.c_longlong]
            L.orc_sim_step_count.argtypes = [C.c_void_p]
            L.orc_sim_step_count.restype = C.c_longlong
            L.orc_sim_fields.argtypes = [C.c_void_p, _dp, _dp, _dp]
            L.orc_sim_observables.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp]
            L.orc_sim_label.argtypes = [C.c_void_p, _ip, _i64p, _dp, C.c_int]
            L.orc_label_field.argtypes = [C.c_int, _ip, _ip, _u8p, _ip]
            L.orc_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _q(lattice: int) -> int:
    return 9 if lattice == 0 else 19


def tables(lattice: int):
    """(c[q,3] int, w[q], opp[q], B[q]) of the oracle's lattice."""
    q = _q(lattice)
    c = np.zeros(3 * q, np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, np.int32)
    B = np.zeros(q)
    lib().orc_lattice_tables(lattice, c, w, opp, B)
    return c.reshape(q, 3), w, opp, B


def phi(lattice: int, alpha: float) -> np.ndarray:
    out = np.zeros(_q(lattice))
    lib().orc_phi(lattice, alpha, out)
    return out


def feq(lattice: int, alpha: float, rho_k: float, u) -> np.ndarray:
    out = np.zeros(_q(lattice))
    uu = np.zeros(3)
    uu[: len(u)] = u
    lib().orc_feq(lattice, alpha, rho_k, uu, out)
    return out


def relax(lattice: int, collision: int, omega: float, f, f_eq) -> np.ndarray:
    out = np.zeros(_q(lattice))
    lib().orc_relax(lattice, collision, omega, np.ascontiguousarray(f, np.float64),
                    np.ascontiguousarray(f_eq, np.float64), out)
    return out


def perturbation(lattice: int, A: float, F) -> np.ndarray:
    out = np.zeros(_q(lattice))
    FF = np.zeros(3)
    FF[: len(F)] = F
    lib().orc_perturbation(lattice, A, FF, out)
    return out


def recolour(lattice: int, beta: float, alpha_r: float, alpha_b: float, rho_r: float, rho_b: float, F, f):
    q = _q(lattice)
    outr, outb = np.zeros(q), np.zeros(q)
    FF = np.zeros(3)
    FF[: len(F)] = F
    lib().orc_recolour(lattice, beta, alpha_r, alpha_b, rho_r, rho_b, FF,
                       np.ascontiguousarray(f, np.float64), outr, outb)
    return outr, outb


def _params(pb) -> _Params:
    p = _Params()
    p.lattice = int(pb.lattice)
    p.nx, p.ny, p.nz = int(pb.nx), int(pb.ny), int(pb.nz)
    for a in range(3):
        p.periodic[a] = int(pb.periodic[a])
    p.collision = int(pb.collision)
    p.tau_r, p.tau_b = float(pb.tau_r), float(pb.tau_b)
    p.alpha_r, p.alpha_b = float(pb.alpha_r), float(pb.alpha_b)
    p.A, p.beta, p.rho0, p.psi_wall = float(pb.A), float(pb.beta), float(pb.rho0), float(pb.psi_wall)
    return p


def mixture_omega(pb, psi: float) -> float:
    p = _params(pb)
    return lib().orc_mixture_omega(C.byref(p), psi)


def collide(pb, fr, fb, F):
    q = _q(pb.lattice)
    p = _params(pb)
    outr, outb = np.zeros(q), np.zeros(q)
    FF = np.zeros(3)
    FF[: len(F)] = F
    lib().orc_collide(C.byref(p), np.ascontiguousarray(fr, np.float64), np.ascontiguousarray(fb, np.float64),
                      FF, outr, outb)
    return outr, outb


def label_field(dims, periodic, field) -> np.ndarray:
    """Face-connected components of a boolean field; label = smallest linear index."""
    d = len(dims)
    dd = np.array(list(dims) + [1] * (3 - d), np.int32)
    pp = np.array(list(periodic) + [1] * (3 - d), np.int32)
    f = np.ascontiguousarray(np.asarray(field, dtype=np.uint8).ravel())
    out = np.zeros(f.size, np.int32)
    lib().orc_label_field(d, dd, pp, f, out)
    return out


def threads() -> int:
    return lib().orc_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(n)


class Sim:
    """FP64 oracle simulation of one Problem."""

    def __init__(self, pb):
        L = lib()
        self.pb = pb
        self.q = _q(pb.lattice)
        self.dim = 2 if pb.lattice == 0 else 3
        nz = pb.nz if pb.lattice == 1 else 1
        self.n = pb.nx * pb.ny * nz
        self._p = _params(pb)
        ports = list(pb.ports)
        arr = (_Port * max(1, len(ports)))()
        for m, pt in enumerate(ports):
            arr[m].kind, arr[m].normal_axis = int(pt.kind), int(pt.normal_axis)
            arr[m].normal_sign, arr[m].profile = int(pt.normal_sign), int(pt.profile)
            arr[m].u_max, arr[m].rho, arr[m].psi = float(pt.u_max), float(pt.rho), float(pt.psi)
        mask = np.ascontiguousarray(np.asarray(pb.mask, np.uint8).ravel())
        assert mask.size == self.n
        self._h = L.orc_sim_create(C.byref(self._p), mask, arr, len(ports))
        if not self._h:
            raise ValueError("oracle: invalid problem (ports / mask)")
        if pb.rho_r is not None:
            self.init_fields(pb.rho_r, pb.rho_b, pb.u)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_sim_destroy(h)
            self._h = None

    def init_fields(self, rho_r, rho_b, u=None):
        rr = np.ascontiguousarray(rho_r, np.float64).ravel()
        rb = np.ascontiguousarray(rho_b, np.float64).ravel()
        if u is None:
            lib().orc_sim_init_fields(self._h, rr, rb, None)
        else:
            uu = np.ascontiguousarray(u, np.float64).reshape(self.dim, self.n)
            lib().orc_sim_init_fields(self._h, rr, rb, uu.ctypes.data_as(C.c_void_p))

    def step(self, n: int = 1):
        lib().orc_sim_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return lib().orc_sim_step_count(self._h)

    def populations(self) -> np.ndarray:
        out = np.zeros(2 * self.q * self.n)
        lib().orc_sim_get_populations(self._h, out)
        return out.reshape(2, self.q, self.n)

    def set_populations(self, f):
        lib().orc_sim_set_populations(self._h, np.ascontiguousarray(f, np.float64).ravel())

    def fields(self):
        rr, rb = np.zeros(self.n), np.zeros(self.n)
        u = np.zeros(self.dim * self.n)
        lib().orc_sim_fields(self._h, rr, rb, u)
        return rr, rb, u.reshape(self.dim, self.n)

    def observables(self, centre, r_in: float = -1.0, r_out: float = -1.0) -> dict:
        out = np.zeros(13)
        c = np.zeros(3)
        c[: len(centre)] = centre
        lib().orc_sim_observables(self._h, c, r_in, r_out, out)
        return dict(mass_r=out[0], mass_b=out[1], mom=out[2:5].copy(), p_in=out[5], p_out=out[6],
                    dp=out[7], r_eff=out[8], umax=out[9], amount=out[10], n_in=out[11], n_out=out[12])

    def label(self, cap: int = 4096):
        labels = np.zeros(self.n, np.int32)
        counts = np.zeros(cap, np.int64)
        vols = np.zeros(cap)
        nd = lib().orc_sim_label(self._h, labels, counts, vols, cap)
        k = min(nd, cap)
        return labels, counts[:k].copy(), vols[:k].copy(), nd
