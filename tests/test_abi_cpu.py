"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/lbsq.h declares; argument validation that
needs no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1903_04799_gb300 import lbsq
    return lbsq.load()


def test_header_declares_the_api():
    names = declared_functions()
    for required in ["lb_create", "lb_destroy", "lb_add_squirmer", "lb_add_wall", "lb_step",
                     "lb_get_fields", "lb_get_force_torque"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1903_04799_gb300 import lbsq
    assert declared_functions() <= set(lbsq.SIGNATURES)


def test_params_default_and_invalid_arguments(lib):
    from paper_1903_04799_gb300 import lbsq
    p = lbsq.lb_params_default()
    assert (p.nx, p.ny, p.nz) == (32, 32, 32) and p.lambda_e == 1.0 and abs(p.magic - 0.1875) < 1e-15
    ctx = C.c_void_p()
    assert p.equilibrium == lbsq.LB_EQ_COMPRESSIBLE
    for field, bad in [("nx", 0), ("lambda_e", 2.0), ("lambda_e", 0.0), ("rho0", -1.0),
                       ("storage", 9), ("collision", 5), ("equilibrium", 2), ("equilibrium", -1),
                       ("rounding", 2), ("rounding", -2)]:
        q = lbsq.lb_params_default()
        setattr(q, field, bad)
        assert lib.lb_create(C.byref(q), C.byref(ctx)) == lbsq.LB_ERR_INVALID
    q = lbsq.lb_params_default()
    q.nx = q.ny = q.nz = 1024  # 2^30 cells: beyond the 2^27 cell limit of the link codes
    assert lib.lb_create(C.byref(q), C.byref(ctx)) == lbsq.LB_ERR_INVALID
    assert lib.lb_create(None, C.byref(ctx)) == lbsq.LB_ERR_INVALID
    assert lib.lb_destroy(None) == lbsq.LB_OK
    assert lib.lb_step(None, 1) == lbsq.LB_ERR_INVALID
    assert lib.lb_set_force_average(None, 1) == lbsq.LB_ERR_INVALID
    assert lib.lb_set_link_options(None, 1, 0) == lbsq.LB_ERR_INVALID
    assert lib.lb_set_coupling(None, lbsq.LB_COUPLE_PSM) == lbsq.LB_ERR_INVALID
    assert lib.lb_get_solid_fraction(None, None) == lbsq.LB_ERR_INVALID
    assert lbsq.lb_params_default().rounding == lbsq.LB_ROUND_DEFAULT
    assert lib.lb_last_error(None) == b"null context"
