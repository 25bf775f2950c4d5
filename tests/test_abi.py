"""The C-ABI library loads and exports every function include/lbcg.h declares
(no GPU needed: only host-side entry points are called)."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1711_02003_gb300 import build as B
from paper_1711_02003_gb300 import lbcg
from paper_1711_02003_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbcg.load()


def test_header_declares_the_boundary():
    names = lbcg.header_functions()
    for must in ("lbcg_create", "lbcg_bind_state", "lbcg_set_geometry", "lbcg_init_fields", "lbcg_step",
                 "lbcg_get_fields", "lbcg_get_populations", "lbcg_observables", "lbcg_label", "lbcg_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    names = lbcg.header_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in names:
        assert n in exported, n
        assert getattr(lib, n) is not None
    # the binding marshals exactly the declared functions
    assert sorted(lbcg._PROTOS) == names


def test_host_side_entry_points(lib):
    assert lib.lbcg_abi_version() == 2
    assert lib.lbcg_strerror(0) == b"ok"
    assert lib.lbcg_strerror(-5) == b"non-finite or non-positive density"
    pb = W.static_droplet(W.D2Q9, 64, 16)
    for prec, es in lbcg.ELEM_BYTES.items():
        assert lbcg.state_bytes(pb, prec) == 2 * 9 * 4096 * es
    pb3 = W.static_droplet(W.D3Q19, 10, 3)
    assert lbcg.state_bytes(pb3, lbcg.LBCG_FP32_DEV) == 2 * 19 * 1024 * 4   # 1000 sites padded to 1024


@pytest.mark.parametrize("field,value", [("tau_r", 0.5), ("tau_b", 0.4), ("beta", 1.5), ("A", -1.0),
                                         ("alpha_r", 1.0), ("psi_wall", 2.0), ("rho0", 0.0), ("nx", 0),
                                         ("lattice", 3), ("precision", 7)])
def test_invalid_parameters_rejected(lib, field, value):
    pb = W.static_droplet(W.D2Q9, 16, 4)
    p = lbcg.params_of(pb, lbcg.LBCG_FP32_DEV)
    setattr(p, field, type(getattr(p, field))(value))
    assert lib.lbcg_state_bytes(C.byref(p)) == 0
    h = C.c_void_p()
    assert lib.lbcg_create(C.byref(p), None, C.byref(h)) == -1
    assert lib.lbcg_last_error()


def test_build_uses_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.exists(B.LIB)
