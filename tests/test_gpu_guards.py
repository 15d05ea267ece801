"""Out-of-bounds checks in place of a device memory checker, which is not
available here.  With guard zones around every library allocation (0xA5
bytes) and around every field and output array (a NaN pattern for floating
point, 0xA5 bytes otherwise), every entry point runs on ragged boxes, in both
precisions and with both step kernels.  No guard byte may change, and every
result must equal, bit for bit, the same calls on unguarded arrays: a read
past an array would have brought a NaN or a pattern byte into it.
"""
import ctypes
import math

import pytest

import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import _abi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GUARD = 4096

# ragged tiles in every direction; 4^3 (smaller than one tile); nx % 32 == 0
# with a ragged nz (the word-wise cell kernels); rows of 1024 (the 32-word
# overlap rows)
SHAPES = [(36, 20, 12), (4, 4, 4), (64, 8, 40), (32, 32, 33), (1024, 10, 6)]


@pytest.fixture(autouse=True)
def guard_off_afterwards():
    yield
    U.set_alloc_guard(0)


def same(a, b) -> bool:
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(same(a[k], b[k]) for k in a)
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    if isinstance(a, torch.Tensor):  # bit patterns: NaN included
        if a.is_floating_point():
            it = torch.int64 if a.element_size() == 8 else torch.int32
            a, b = a.contiguous().view(it), b.contiguous().view(it)
        return a.shape == b.shape and torch.equal(a.cpu(), b.cpu())
    if isinstance(a, float) and isinstance(b, float) and math.isnan(a) and math.isnan(b):
        return True
    return a == b


def noalloc(lat, tol):
    fields = (ctypes.c_void_p * 20)(*[t.data_ptr() for t in lat.fields()])
    out = _abi.CStrings()
    U.check(U.lib().u1u1_detect_strings_noalloc(ctypes.byref(lat.params.c()), fields, lat.n, tol,
                                                ctypes.byref(out), None))
    return _abi.struct_to_dict(out)


def lattice_calls(p, kernel, guard, tmp_path):
    """Every single-lattice entry point once; returns the results in order and
    the guard counts (library, arrays) taken while the handle is alive."""
    U.set_alloc_guard(guard)
    lat = U.Lattice(p, kernel=kernel, guard=guard)
    out = []
    lat.cool(0.05, 2)
    lat.autotune()  # candidate steps on the handle's own state, which it restores
    lat.set_kernel(kernel)
    lat.step(5)
    lat.step(8, detect_every=4)
    out.append(lat.read_records())
    for tol in (0, 1):
        r = lat.detect_strings(tol=tol, cells=True, windings=True)
        out.append(r)
        out.append(noalloc(lat, tol))
    out.append(lat.diagnostics())
    out.append(lat.pq_segments(labels=True))
    host = [torch.empty(p.nsites, dtype=lat.dtype).pin_memory() for _ in range(20)]
    lat.download(host)
    lat.upload(host)
    path = tmp_path / f"ckpt_{guard}.u1u1"
    lat.save(str(path))
    lat.step(3)
    lat.load(str(path))
    lat.step(2)
    out.append(lat.state().clone())
    assert bool(torch.isfinite(out[-1]).all())
    counts = (U.check_alloc_guards(), lat.check_guards())
    lat.close()
    return out, counts


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kernel", [U.KERNEL_SIMPLE, U.KERNEL_TILED])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_guarded_lattice_calls(shape, kernel, prec, tmp_path):
    p = U.Params(nx=shape[0], ny=shape[1], nz=shape[2], m=0.5, beta=1.0, eta0=1.0, eta_ref=3.0, seed=12,
                 precision=prec, lambda_p=2.0, lambda_q=1.62, e_p=1.0, e_q=0.9, sigma_p=1.0, sigma_q=0.8,
                 kappa=0.5)
    ref, _ = lattice_calls(p, kernel, 0, tmp_path)
    got, (lib_bad, arr_bad) = lattice_calls(p, kernel, GUARD, tmp_path)
    assert lib_bad == 0 and arr_bad == 0
    assert same(got, ref)


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_guarded_ensemble_runs(prec):
    """Every ensemble schedule with detection inside the run, graph replays
    included, on ragged boxes with guards."""
    shapes = [(36, 20, 12), (4, 4, 4), (32, 32, 33)]

    def calls(guard):
        U.set_alloc_guard(guard)
        # a stays between 0.44 and 1.8 over the runs (eta 3 .. 6.1), so every
        # box, the core-growth one included, stays finite
        ps = [U.Params(nx=s[0], ny=s[1], nz=s[2], m=2.0 / 3.0, beta=b, eta0=3.0, eta_ref=4.5, seed=70 + i,
                       precision=prec) for i, (s, b) in enumerate(zip(shapes, (1.0, 0.0, -1.0)))]
        e = U.Ensemble(ps, guard=guard)
        out = []
        for mode, graph in ((U.ENS_PERSISTENT, True), (U.ENS_PER_STEP, True), (U.ENS_UNBATCHED, False)):
            e.run([9, 6, 4], mode=mode, use_graph=graph, detect_every=3)
            out.append([b.read_records() for b in e.boxes])
        e.run([4, 4, 4], mode=U.ENS_PERSISTENT, use_graph=True)
        out.append([b.detect_strings(tol=1, cells=True) for b in e.boxes])
        out.append([b.state().clone() for b in e.boxes])
        counts = (U.check_alloc_guards(), e.check_guards())
        e.close()
        return out, counts

    ref, _ = calls(0)
    got, (lib_bad, arr_bad) = calls(GUARD)
    assert lib_bad == 0 and arr_bad == 0
    assert all(bool(torch.isfinite(st).all()) for st in ref[-1])
    assert same(got, ref)


def test_guard_checks_see_a_write_past_the_end():
    """The checks themselves: a byte changed in the tail guard of a library
    allocation (by the library's test hook, in memory the library owns) and
    an element written one past the end of a guarded field array (into its
    guard zone, which the lattice owns) are each reported once."""
    U.set_alloc_guard(GUARD)
    lat = U.Lattice(U.Params(nx=8, ny=8, nz=8, seed=1), guard=GUARD)
    lat.step(2, detect_every=1)
    lat.read_records()
    assert U.check_alloc_guards() == 0 and lat.check_guards() == 0
    U.check(U.lib().u1u1_inject_guard_damage())
    assert U.check_alloc_guards() == 1
    full, g = lat._guarded[-1]
    full[g + lat.params.nsites] = 0.0
    assert lat.check_guards() == 1
    lat.close()
    U.set_alloc_guard(0)
    assert U.lib().u1u1_inject_guard_damage() == -8  # no guarded allocation is live
