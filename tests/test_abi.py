"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/u1u1.h; host-only helpers agree with the oracle (CPU)."""
import ctypes
import math
import os
import re

import pytest

import oracle as O
import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(u1u1_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = U.lib()
    decl = declared_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(L, name), name
    assert decl == set(_abi.PROTOTYPES), decl ^ set(_abi.PROTOTYPES)


def test_struct_mirrors_match_header():
    out = (ctypes.c_size_t * 4)()
    U.lib().u1u1_abi_sizes(out)
    assert list(out) == [ctypes.sizeof(_abi.CParams), ctypes.sizeof(_abi.CBuffers),
                         ctypes.sizeof(_abi.CStrings), ctypes.sizeof(_abi.CDiag)]


def test_version_and_defaults():
    assert re.match(r"\d+\.\d+\.\d+", U.version())
    cp = _abi.CParams()
    U.check(U.lib().u1u1_params_default(ctypes.byref(cp)))
    # equal-tension, critical couplings of Sec. IV
    assert (cp.lambda_p, cp.lambda_q, cp.e_p, cp.e_q, cp.sigma_p, cp.kappa) == (2.0, 2.0, 1.0, 1.0, 1.0, 0.9)
    assert (cp.dx, cp.deta, cp.alpha) == (0.5, 0.1, 2.0)


@pytest.mark.parametrize("field,value", [
    ("nx", 6), ("nx", 0), ("ny", 3), ("dx", 0.0), ("deta", -0.1), ("m", 1.0), ("m", -0.1),
    ("eta_ref", 0.0), ("e_p", 0.0), ("precision", 7), ("kappa", float("nan")),
])
def test_invalid_params_rejected(field, value):
    p = U.Params.cube(16)
    setattr(p, field, value)
    rc = U.lib().u1u1_check_params(ctypes.byref(p.c()))
    assert rc == -1
    assert U.lib().u1u1_last_error().decode()


def test_eta0_must_be_positive_when_expanding():
    p = U.Params.cube(16, eta0=0.0, m=0.5)
    with pytest.raises(U.U1U1Error):
        U.check_params(p)
    U.check_params(U.Params.cube(16, eta0=0.0, m=0.0))


@pytest.mark.parametrize("m,beta,eta_ref", [(0.5, 1.0, 65.0), (2.0 / 3.0, 0.0, 1.0), (0.5, -1.0, 1.0),
                                            (0.0, 1.0, 1.0), (2.0 / 3.0, 0.4, 3.0)])
def test_host_coefficients_match_oracle(m, beta, eta_ref):
    p = U.Params.cube(16, m=m, beta=beta, eta_ref=eta_ref)
    q = O.Params(16, 16, 16, m=m, beta=beta, eta_ref=eta_ref)
    for n in (0, 1, 17, 640):
        a = U.coefficients(p, n)
        b = O.coeffs(q, n)
        for k in a:
            assert math.isclose(a[k], b[k], rel_tol=1e-14, abs_tol=0.0), (k, a[k], b[k])


def test_field_bytes():
    p = U.Params(nx=8, ny=12, nz=20)
    assert U.lib().u1u1_field_bytes(ctypes.byref(p.c())) == 8 * 12 * 20 * 4
    p.precision = U.FP64
    assert U.lib().u1u1_field_bytes(ctypes.byref(p.c())) == 8 * 12 * 20 * 8
    assert U.lib().u1u1_field_bytes(None) == 0


def test_null_handles_are_rejected_without_gpu():
    L = U.lib()
    assert L.u1u1_step(None, 1, 0, None) == -1
    assert L.u1u1_current(None, None, None) == -1
    assert L.u1u1_set_overlap_tol(None, 1) == -1
    L.u1u1_destroy(None)


def test_ensemble_and_probe_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks that come before any device work: NULL handles and
    outputs, a negative detection cadence, unknown modes."""
    L = U.lib()
    steps = (ctypes.c_int * 2)(1, 1)
    assert L.u1u1_ensemble_run(None, steps, 0, 0, 0, None) == -1
    assert L.u1u1_ensemble_set_tuning(None, 32, 1, None) == -1
    assert L.u1u1_ensemble_get_tuning(None, None, None) == -1
    assert L.u1u1_ensemble_autotune(None, 4, None, None, None) == -1
    assert L.u1u1_fp64_fma_rate(None, None) == -1
    assert L.u1u1_inject_copy_timeout(1, 10) == -1  # limit below 1000 ns
    L.u1u1_ensemble_destroy(None)


def test_allocation_hook_and_accounting_without_gpu():
    """The allocation-failure hook and the live-allocation count are host
    state: without a GPU no handle can exist, so nothing is held, and a
    negative nth is rejected."""
    import torch
    count, nbytes = U.live_allocations()
    assert count >= 0 and nbytes >= 0
    if not torch.cuda.is_available():
        assert (count, nbytes) == (0, 0)
    U.inject_alloc_failure(3)
    U.inject_alloc_failure(0)
    with pytest.raises(U.U1U1Error) as ei:
        U.inject_alloc_failure(-1)
    assert ei.value.code == -1
    assert U.lib().u1u1_live_allocations(None, None) == -1


def test_guard_zones_detect_writes_and_poison_reads():
    """The guard zones of the debugging aid (host logic, on CPU tensors): a
    write one element past either end of a guarded array is counted, and a
    read past a floating-point array yields NaN."""
    import torch
    from paper_2208_01525_gb300 import _guarded_empty, _guards_damaged
    for dtype in (torch.float32, torch.float64, torch.uint8, torch.int8, torch.int32):
        guarded = []
        t = _guarded_empty(1000, dtype, "cpu", 256, guarded)
        full, g = guarded[0]
        assert t.numel() == 1000 and t.data_ptr() - full.data_ptr() == 256
        t.fill_(1)
        assert _guards_damaged(guarded) == 0
        if dtype.is_floating_point:
            assert torch.isnan(full[g - 1]) and torch.isnan(full[g + 1000])
        full[g + 1000] = 0  # one past the end
        assert _guards_damaged(guarded) == 1
        full[g + 1000] = t[0]
        guarded2 = []
        _guarded_empty(10, dtype, "cpu", 512, guarded2)[0] = 3
        full2, g2 = guarded2[0]
        full2[g2 - 1] = 0  # one before the start
        assert _guards_damaged(guarded2) == 1
    with pytest.raises(ValueError):
        _guarded_empty(10, torch.float32, "cpu", 100, [])
    assert U.lib().u1u1_set_alloc_guard(100) == -1
    assert U.lib().u1u1_set_alloc_guard(-256) == -1
    U.set_alloc_guard(256)
    U.set_alloc_guard(0)
    assert U.lib().u1u1_check_alloc_guards(None) == -1
