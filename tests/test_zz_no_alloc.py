"""The allocation-free detection entry point (u1u1_detect_strings_noalloc).

Some callers cannot allocate device memory while they run (a framework owns
the device pool, the call happens inside an allocator callback, or a policy
forbids allocation after start-up).  For them the library offers one entry
point whose scratch lives in a fixed static device array.  This test calls
it through the C ABI twice in a row on the same state and requires both
results to equal the handle-based u1u1_detect_strings (integer counts bit
exact, derived lengths, separations and fractions equal).  The file sorts
last so that a run stopping at the first failure has run everything else;
it also passes alone in a fresh process.
"""
import ctypes
import math

import pytest

import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import _abi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def noalloc(lat: U.Lattice, tol: int) -> dict:
    fields = (ctypes.c_void_p * 20)(*[t.data_ptr() for t in lat.fields()])
    out = _abi.CStrings()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    U.check(U.lib().u1u1_detect_strings_noalloc(ctypes.byref(lat.params.c()), fields, lat.n, tol,
                                                ctypes.byref(out), stream))
    return _abi.struct_to_dict(out)


def same(a: dict, b: dict) -> bool:
    for k, v in b.items():
        w = a[k]
        if isinstance(v, float) and math.isnan(v):
            if not math.isnan(w):
                return False
        elif w != v:
            return False
    return True


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_noalloc_detection_matches_handle_twice(prec):
    p = U.Params(nx=48, ny=40, nz=36, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=7, precision=prec)
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(25)
    for tol in (1, 0):
        ref = lat.detect_strings(tol=tol)
        first = noalloc(lat, tol)
        # the second call must not touch the device memory pool: neither the
        # driver's free-memory figure nor PyTorch's allocator may move
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        second = noalloc(lat, tol)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0
        assert ref["n_p"] > 0
        assert same(first, ref), (first, ref)
        assert same(second, ref), (second, ref)


def test_noalloc_rejects_oversized_scratch():
    """A lattice under the site limit whose scratch does not fit the static
    array (4 x 2048 x 2048: face bytes plus one cell-mask word per row) is
    refused before any launch, with the byte count in the message."""
    p = U.Params(nx=4, ny=2048, nz=2048)
    assert p.nsites <= 16777216
    dummy = torch.empty(64, device="cuda")
    fields = (ctypes.c_void_p * 20)(*([dummy.data_ptr()] * 20))
    out = _abi.CStrings()
    rc = U.lib().u1u1_detect_strings_noalloc(ctypes.byref(p.c()), fields, 0, 1, ctypes.byref(out), None)
    assert rc == -1  # INVALID_ARG
    msg = U.lib().u1u1_last_error().decode()
    assert "bytes of scratch" in msg and str(48 << 20) in msg, msg


def test_noalloc_rejects_oversized_lattice():
    p = U.Params(nx=512, ny=256, nz=256)
    dummy = torch.empty(1, device="cuda")
    fields = (ctypes.c_void_p * 20)(*([dummy.data_ptr()] * 20))
    out = _abi.CStrings()
    rc = U.lib().u1u1_detect_strings_noalloc(ctypes.byref(p.c()), fields, 0, 1, ctypes.byref(out), None)
    assert rc == -1
    assert "limit" in U.lib().u1u1_last_error().decode()
