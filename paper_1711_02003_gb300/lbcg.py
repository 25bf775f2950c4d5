"""Thin Python binding of liblbcg.so (include/lbcg.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The functions keep the C names (``lbcg_create``, ``lbcg_step`` ...); the
:class:`Simulation` helper allocates the two population buffers with torch on
the current CUDA device, binds them, and wraps the calls for one problem.

There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbcg.so")

LBCG_OK = 0
LBCG_D2Q9, LBCG_D3Q19 = 0, 1
LBCG_FP64, LBCG_FP32, LBCG_FP32_DEV, LBCG_FP16_SCALED = 0, 1, 2, 3
LBCG_REG, LBCG_BGK = 0, 1
LBCG_ERR_STATE = -2  # call out of order (or a synchronous call on a capturing stream)
LBCG_ERR_TIMEOUT = -9  # a bounded device-side wait or iteration ran out
LBCG_ERR_BOUNDS = -10  # bounds-checked build: a step kernel met an index outside its array
PRECISION_NAMES = {LBCG_FP64: "f64", LBCG_FP32: "f32", LBCG_FP32_DEV: "f32dev", LBCG_FP16_SCALED: "f16scaled"}
ELEM_BYTES = {LBCG_FP64: 8, LBCG_FP32: 4, LBCG_FP32_DEV: 4, LBCG_FP16_SCALED: 2}


class lbcg_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3), ("collision", C.c_int), ("precision", C.c_int),
                ("tau_r", C.c_double), ("tau_b", C.c_double), ("alpha_r", C.c_double),
                ("alpha_b", C.c_double), ("A", C.c_double), ("beta", C.c_double), ("rho0", C.c_double),
                ("psi_wall", C.c_double)]


class lbcg_port(C.Structure):
    _fields_ = [("kind", C.c_int), ("normal_axis", C.c_int), ("normal_sign", C.c_int), ("profile", C.c_int),
                ("u_max", C.c_double), ("rho", C.c_double), ("psi", C.c_double)]


class lbcg_obs(C.Structure):
    _fields_ = [("mass_r", C.c_double), ("mass_b", C.c_double), ("mom", C.c_double * 3), ("p_in", C.c_double),
                ("p_out", C.c_double), ("dp", C.c_double), ("r_eff", C.c_double), ("umax", C.c_double),
                ("amount", C.c_double), ("n_in", C.c_double), ("n_out", C.c_double), ("step", C.c_longlong),
                ("nonfinite", C.c_int), ("pad_", C.c_int)]


class LbcgError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn} failed with status {status}: {message}")
        self.status = status


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_PROTOS = {
    "lbcg_strerror": (C.c_char_p, [C.c_int]),
    "lbcg_last_error": (C.c_char_p, []),
    "lbcg_abi_version": (C.c_int, []),
    "lbcg_bounds_checked": (C.c_int, []),
    "lbcg_state_bytes": (C.c_size_t, [C.POINTER(lbcg_params)]),
    "lbcg_create": (C.c_int, [C.POINTER(lbcg_params), _vp, C.POINTER(_vp)]),
    "lbcg_destroy": (None, [_vp]),
    "lbcg_bind_state": (C.c_int, [_vp, _vp, _vp, C.c_size_t]),
    "lbcg_set_geometry": (C.c_int, [_vp, _vp, C.POINTER(lbcg_port), C.c_int]),
    "lbcg_init_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbcg_init_fields_device": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbcg_step": (C.c_int, [_vp, C.c_longlong]),
    "lbcg_step_count": (C.c_longlong, [_vp]),
    "lbcg_synchronize": (C.c_int, [_vp]),
    "lbcg_get_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbcg_get_fields_device": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbcg_get_populations": (C.c_int, [_vp, _vp]),
    "lbcg_set_populations": (C.c_int, [_vp, _vp]),
    "lbcg_get_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lbcg_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lbcg_save": (C.c_int, [_vp, C.c_char_p]),
    "lbcg_load": (C.c_int, [_vp, C.c_char_p]),
    "lbcg_observables": (C.c_int, [_vp, _dp, C.c_double, C.c_double, C.POINTER(lbcg_obs)]),
    "lbcg_label": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.POINTER(C.c_int)]),
    "lbcg_observables_noalloc": (C.c_int, [C.POINTER(lbcg_params), _vp, _vp, _dp, C.c_double, C.c_double, _vp,
                                           C.POINTER(lbcg_obs)]),
    "lbcg_set_kernel_timing": (C.c_int, [_vp, C.c_int]),
    "lbcg_kernel_time": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong)]),
    "lbcg_set_launch": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "lbcg_get_launch": (C.c_int, [_vp, _ip, _ip, _ip]),
    "lbcg_get_grid": (C.c_int, [_vp, C.POINTER(C.c_longlong), _ip, _ip]),
    "lbcg_current_state": (_vp, [_vp]),
    "lbcg_fma_peak": (C.c_int, [C.c_int, _vp, _dp]),
    "lbcg_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, C.POINTER(_vp)]),
    "lbcg_batch_destroy": (None, [_vp]),
    "lbcg_batch_add": (C.c_int, [_vp, _vp, C.c_longlong, C.POINTER(C.c_int)]),
    "lbcg_batch_remove": (C.c_int, [_vp, C.c_int]),
    "lbcg_batch_remaining": (C.c_longlong, [_vp, C.c_int]),
    "lbcg_batch_step": (C.c_int, [_vp, C.c_longlong]),
    "lbcg_batch_poll": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_int)]),
    "lbcg_batch_last_error": (C.c_char_p, []),
    "lbcg_batch_set_shape": (C.c_int, [_vp, _vp]),
    "lbcg_batch_get_shape": (C.c_int, [_vp, _vp]),
}


def load(path: str | None = None):
    """Load liblbcg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build it with paper_1711_02003_gb300.build.build() "
                           "(CUDA toolkit required; there is no CPU fallback)")
    L = C.CDLL(p)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(fn: str, status: int) -> int:
    if status != LBCG_OK:
        raise LbcgError(fn, status, _lib.lbcg_last_error().decode())
    return status


def params_of(pb, precision: int) -> lbcg_params:
    p = lbcg_params()
    p.lattice, p.nx, p.ny, p.nz = int(pb.lattice), int(pb.nx), int(pb.ny), int(pb.nz)
    for a in range(3):
        p.periodic[a] = int(pb.periodic[a])
    p.collision, p.precision = int(pb.collision), int(precision)
    p.tau_r, p.tau_b = float(pb.tau_r), float(pb.tau_b)
    p.alpha_r, p.alpha_b = float(pb.alpha_r), float(pb.alpha_b)
    p.A, p.beta, p.rho0, p.psi_wall = float(pb.A), float(pb.beta), float(pb.rho0), float(pb.psi_wall)
    return p


def ports_of(pb):
    arr = (lbcg_port * max(1, len(pb.ports)))()
    for m, pt in enumerate(pb.ports):
        arr[m].kind, arr[m].normal_axis = int(pt.kind), int(pt.normal_axis)
        arr[m].normal_sign, arr[m].profile = int(pt.normal_sign), int(pt.profile)
        arr[m].u_max, arr[m].rho, arr[m].psi = float(pt.u_max), float(pt.rho), float(pt.psi)
    return arr


def fma_peak(precision: int = 0, stream=None) -> float:
    """Measured multiply-add throughput of the current device, GFLOP/s (FP64 or FP32)."""
    load()
    g = C.c_double()
    sp = C.c_void_p(stream.cuda_stream if stream is not None else 0)
    _check("lbcg_fma_peak", _lib.lbcg_fma_peak(int(precision), sp, C.byref(g)))
    return g.value


def state_bytes(pb, precision: int) -> int:
    L = load()
    p = params_of(pb, precision)
    return int(L.lbcg_state_bytes(C.byref(p)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Simulation:
    """One problem on the current CUDA device, state in two torch-allocated buffers.

    Calls are enqueued on ``stream`` (a torch.cuda.Stream; default: the current stream)."""

    def __init__(self, pb, precision: int = LBCG_FP32_DEV, stream=None, init: bool = True, rows: int = 0,
                 block_rows: int = 0, variant: int = 0):
        import torch
        L = load()
        self.pb = pb
        self.precision = precision
        self.q = pb.q
        self.dim = pb.dim
        self.n = pb.nsites
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._p = params_of(pb, precision)
        h = _vp()
        _check("lbcg_create", L.lbcg_create(C.byref(self._p), _vp(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.state_bytes = int(L.lbcg_state_bytes(C.byref(self._p)))
        with torch.cuda.stream(self.stream):
            self._a = torch.empty(self.state_bytes, dtype=torch.uint8, device="cuda")
            self._b = torch.empty(self.state_bytes, dtype=torch.uint8, device="cuda")
        _check("lbcg_bind_state", L.lbcg_bind_state(h, _vp(self._a.data_ptr()), _vp(self._b.data_ptr()),
                                                    self.state_bytes))
        if rows or block_rows or variant:
            self.set_launch(rows, block_rows, variant)
        mask = np.ascontiguousarray(np.asarray(pb.mask, np.uint8).ravel())
        ports = ports_of(pb)
        _check("lbcg_set_geometry", L.lbcg_set_geometry(h, _ptr(mask), ports, len(pb.ports)))
        if init and pb.rho_r is not None:
            self.init_fields(pb.rho_r, pb.rho_b, pb.u)

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- calls
    def set_launch(self, rows: int = 0, block_rows: int = 0, variant: int = 0):
        _check("lbcg_set_launch", _lib.lbcg_set_launch(self._h, int(rows), int(block_rows), int(variant)))

    @property
    def launch(self) -> dict:
        """The launch shape in use after defaults: rows, block_rows, variant."""
        r, b, v = C.c_int(), C.c_int(), C.c_int()
        _check("lbcg_get_launch", _lib.lbcg_get_launch(self._h, C.byref(r), C.byref(b), C.byref(v)))
        return {"rows": r.value, "block_rows": b.value, "variant": v.value}

    @property
    def current_state_ptr(self) -> int:
        """Device address of the buffer holding the current state (valid until the next step)."""
        return int(_lib.lbcg_current_state(self._h) or 0)

    @property
    def grid(self) -> dict:
        """Thread blocks and threads per block of the next step launch, kernels per step."""
        b, t, k = C.c_longlong(), C.c_int(), C.c_int()
        _check("lbcg_get_grid", _lib.lbcg_get_grid(self._h, C.byref(b), C.byref(t), C.byref(k)))
        return {"blocks": b.value, "threads": t.value, "kernels_per_step": k.value}

    def init_fields(self, rho_r, rho_b, u=None):
        rr = np.ascontiguousarray(rho_r, np.float64).ravel()
        rb = np.ascontiguousarray(rho_b, np.float64).ravel()
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(self.dim, self.n)
        _check("lbcg_init_fields", _lib.lbcg_init_fields(self._h, _ptr(rr), _ptr(rb),
                                                         None if uu is None else _ptr(uu)))

    def init_fields_device(self, rho_r, rho_b, u=None):
        """Device tensors (float64, contiguous) on this device."""
        _check("lbcg_init_fields_device", _lib.lbcg_init_fields_device(
            self._h, _vp(rho_r.data_ptr()), _vp(rho_b.data_ptr()), None if u is None else _vp(u.data_ptr())))

    def step(self, n: int = 1):
        _check("lbcg_step", _lib.lbcg_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        return int(_lib.lbcg_step_count(self._h))

    def synchronize(self):
        _check("lbcg_synchronize", _lib.lbcg_synchronize(self._h))

    def fields(self):
        rr, rb = np.zeros(self.n), np.zeros(self.n)
        u = np.zeros(self.dim * self.n)
        _check("lbcg_get_fields", _lib.lbcg_get_fields(self._h, _ptr(rr), _ptr(rb), _ptr(u)))
        return rr, rb, u.reshape(self.dim, self.n)

    def fields_device(self, rr, rb, u):
        _check("lbcg_get_fields_device", _lib.lbcg_get_fields_device(
            self._h, _vp(rr.data_ptr()), _vp(rb.data_ptr()), _vp(u.data_ptr())))

    def populations(self) -> np.ndarray:
        f = np.zeros(2 * self.q * self.n)
        _check("lbcg_get_populations", _lib.lbcg_get_populations(self._h, _ptr(f)))
        return f.reshape(2, self.q, self.n)

    def set_populations(self, f):
        ff = np.ascontiguousarray(f, np.float64).ravel()
        _check("lbcg_set_populations", _lib.lbcg_set_populations(self._h, _ptr(ff)))

    def observables(self, centre, r_in: float = -1.0, r_out: float = -1.0, allow_diverged: bool = False) -> dict:
        c = (C.c_double * 3)(*([float(v) for v in centre] + [0.0] * (3 - len(centre))))
        o = lbcg_obs()
        st = _lib.lbcg_observables(self._h, c, float(r_in), float(r_out), C.byref(o))
        if not (allow_diverged and st == -5):
            _check("lbcg_observables", st)
        return dict(mass_r=o.mass_r, mass_b=o.mass_b, mom=np.array(o.mom[:]), p_in=o.p_in, p_out=o.p_out,
                    dp=o.dp, r_eff=o.r_eff, umax=o.umax, amount=o.amount, n_in=o.n_in, n_out=o.n_out,
                    step=o.step, nonfinite=o.nonfinite)

    def label(self, cap: int = 4096):
        labels = np.zeros(self.n, np.int32)
        counts = np.zeros(cap, np.int64)
        vols = np.zeros(cap)
        nd = C.c_int(0)
        _check("lbcg_label", _lib.lbcg_label(self._h, _ptr(labels), _ptr(counts), _ptr(vols), cap, C.byref(nd)))
        k = min(nd.value, cap)
        return labels, counts[:k].copy(), vols[:k].copy(), nd.value

    # ------------------------------------------------------------ checkpoints
    def get_state(self) -> np.ndarray:
        """The raw stored state (storage format bytes)."""
        buf = np.empty(self.state_bytes, np.uint8)
        _check("lbcg_get_state", _lib.lbcg_get_state(self._h, _ptr(buf), self.state_bytes))
        return buf

    def set_state(self, buf):
        b = np.ascontiguousarray(buf, np.uint8)
        _check("lbcg_set_state", _lib.lbcg_set_state(self._h, _ptr(b), b.size))

    def save(self, path: str):
        """Checkpoint: the raw stored state (lossless in every precision) and the step count."""
        np.savez(path, state=self.get_state(), step=self.total_steps, lattice=self.pb.lattice,
                 precision=self.precision, shape=np.array([self.pb.nx, self.pb.ny, self.pb.nz]))

    @classmethod
    def load(cls, path: str, pb, stream=None, **launch) -> "Simulation":
        """A Simulation of problem `pb` resumed from a checkpoint written by save()."""
        d = np.load(path)
        if int(d["lattice"]) != pb.lattice or list(d["shape"]) != [pb.nx, pb.ny, pb.nz]:
            raise ValueError("checkpoint does not match the problem's lattice or box")
        sim = cls(pb, int(d["precision"]), stream=stream, init=False, **launch)
        sim.set_state(d["state"])
        sim._step_offset = int(d["step"])
        return sim

    def save_file(self, path: str):
        """Checkpoint through the library's own file format (lbcg_save)."""
        _check("lbcg_save", _lib.lbcg_save(self._h, path.encode()))

    def load_file(self, path: str):
        """Restore a lbcg_save checkpoint into this context (same lattice, box, precision)."""
        _check("lbcg_load", _lib.lbcg_load(self._h, path.encode()))

    @property
    def total_steps(self) -> int:
        """Steps since the initial state, across checkpoint/resume."""
        return self.step_count + getattr(self, "_step_offset", 0)

    def set_kernel_timing(self, enable: bool):
        _check("lbcg_set_kernel_timing", _lib.lbcg_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_time(self):
        ms = C.c_double(0.0)
        nl = C.c_longlong(0)
        _check("lbcg_kernel_time", _lib.lbcg_kernel_time(self._h, C.byref(ms), C.byref(nl)))
        return ms.value, nl.value


def header_functions(header_path: str | None = None) -> list:
    """Names of the functions declared in include/lbcg.h."""
    import re
    hp = header_path or os.path.join(_HERE, "..", "include", "lbcg.h")
    text = open(hp).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbcg_[a-z0-9_]+)\s*\(", text)))


class lbcg_batch_shape(C.Structure):
    _fields_ = [("rows", C.c_int), ("block_rows", C.c_int), ("strips_per_item", C.c_int),
                ("blocks_per_sm", C.c_int), ("graph_steps", C.c_int), ("sms", C.c_int)]


class Batch:
    """Many instances of one lattice and storage precision advanced together
    (lbcg_batch_*).  Instances are Simulation objects; they must use the batch's stream.
    ``shape``: a dict of lbcg_batch_shape fields (rows, block_rows, strips_per_item,
    blocks_per_sm, graph_steps; missing or 0 = default)."""

    def __init__(self, lattice: int, precision: int = LBCG_FP32_DEV, max_instances: int = 64, stream=None,
                 shape: dict | None = None):
        import torch
        L = load()
        self.lattice, self.precision = lattice, precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _vp()
        st = L.lbcg_batch_create(int(lattice), int(precision), int(max_instances), _vp(self.stream.cuda_stream),
                                 C.byref(h))
        self._bcheck("lbcg_batch_create", st)
        self._h = h
        self.max_instances = max_instances
        self.sims = {}
        if shape:
            self.set_shape(**shape)

    def set_shape(self, rows: int = 0, block_rows: int = 0, strips_per_item: int = 0, blocks_per_sm: int = 0,
                  graph_steps: int = 0, **_ignored):
        sh = lbcg_batch_shape(int(rows), int(block_rows), int(strips_per_item), int(blocks_per_sm), int(graph_steps), 0)
        self._bcheck("lbcg_batch_set_shape", _lib.lbcg_batch_set_shape(self._h, C.byref(sh)))

    @property
    def shape(self) -> dict:
        """The launch shape after defaults (and the device's SM count)."""
        sh = lbcg_batch_shape()
        self._bcheck("lbcg_batch_get_shape", _lib.lbcg_batch_get_shape(self._h, C.byref(sh)))
        return {f: getattr(sh, f) for f, _ in lbcg_batch_shape._fields_}

    @staticmethod
    def _bcheck(fn, st):
        if st != LBCG_OK:
            raise LbcgError(fn, st, _lib.lbcg_batch_last_error().decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbcg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, sim: "Simulation", steps: int) -> int:
        slot = C.c_int(-1)
        self._bcheck("lbcg_batch_add", _lib.lbcg_batch_add(self._h, sim._h, int(steps), C.byref(slot)))
        self.sims[slot.value] = sim
        return slot.value

    def remove(self, slot: int):
        self._bcheck("lbcg_batch_remove", _lib.lbcg_batch_remove(self._h, int(slot)))
        self.sims.pop(slot, None)

    def remaining(self, slot: int) -> int:
        return int(_lib.lbcg_batch_remaining(self._h, int(slot)))

    def step(self, max_steps: int):
        self._bcheck("lbcg_batch_step", _lib.lbcg_batch_step(self._h, int(max_steps)))

    def poll(self) -> list:
        cap = max(1, self.max_instances)
        out = (C.c_int * cap)()
        n = C.c_int(0)
        self._bcheck("lbcg_batch_poll", _lib.lbcg_batch_poll(self._h, out, cap, C.byref(n)))
        return [out[i] for i in range(n.value)]

    @property
    def active(self) -> int:
        return len(self.sims)
