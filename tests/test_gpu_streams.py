"""Streams: every entry point enqueues its work on the stream it is given,
and the calls that fill host structs synchronise that stream only.  Two
lattices are driven at once, from two host threads on two side streams,
through every stream-taking entry point.  An ensemble runs its three
schedules, with detection and graph replays, on a side stream.  Every
result must equal, bit for bit, the same calls made one after another on
the default stream.
"""
import ctypes
import math
import threading

import pytest

import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import _abi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# The allocation-free detection shares one static scratch array between all
# calls, so calls that overlap on the GPU race; each call synchronises its
# stream before it returns, so holding this lock around it keeps them apart.
NOALLOC_LOCK = threading.Lock()


def same(a, b) -> bool:
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(same(a[k], b[k]) for k in a)
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    if isinstance(a, torch.Tensor):  # bit patterns, NaN included
        if a.is_floating_point():
            it = torch.int64 if a.element_size() == 8 else torch.int32
            a, b = a.contiguous().view(it), b.contiguous().view(it)
        return a.shape == b.shape and torch.equal(a.cpu(), b.cpu())
    if isinstance(a, float) and isinstance(b, float) and math.isnan(a) and math.isnan(b):
        return True
    return a == b


def params(shape, seed):
    return U.Params(nx=shape[0], ny=shape[1], nz=shape[2], m=0.5, beta=1.0, eta0=1.0, eta_ref=3.0, seed=seed,
                    precision=U.FP32, sigma_q=0.8, e_q=0.9)


def workload(p, stream):
    """Every stream-taking call on one lattice; returns the results."""
    lat = U.Lattice(p, stream=stream)
    out = []
    lat.step(9, detect_every=3, stream=stream)
    out.append(lat.read_records(stream=stream))
    out.append(lat.detect_strings(tol=1, cells=True, windings=True, stream=stream))
    out.append(lat.diagnostics(stream=stream))
    out.append(lat.pq_segments(labels=True, stream=stream))
    fields = (ctypes.c_void_p * 20)(*[t.data_ptr() for t in lat.fields()])
    res = _abi.CStrings()
    sptr = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    with NOALLOC_LOCK:
        U.check(U.lib().u1u1_detect_strings_noalloc(ctypes.byref(lat.params.c()), fields, lat.n, 1,
                                                    ctypes.byref(res), sptr))
    out.append(_abi.struct_to_dict(res))
    lat.cool(0.05, 2, stream=stream)
    lat.step(5, stream=stream)
    host = [torch.empty(p.nsites).pin_memory() for _ in range(20)]
    lat.download(host, stream=stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    out.append(torch.stack(host))
    out.append(lat.state().clone())
    lat.close()
    return out


def test_two_lattices_on_two_threads_and_streams():
    ps = [params((36, 20, 12), 31), params((32, 32, 16), 32)]
    ref = [workload(p, None) for p in ps]  # also sets every kernel's launch attributes once
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    got = [None, None]
    errors = []

    def run(i):
        try:
            got[i] = workload(ps[i], streams[i])
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(2):
        assert same(got[i], ref[i]), (i, [k for k, (a, b) in enumerate(zip(got[i], ref[i])) if not same(a, b)])


def test_ensemble_on_a_side_stream():
    ps = [U.Params(nx=s[0], ny=s[1], nz=s[2], m=2.0 / 3.0, beta=b, eta0=3.0, eta_ref=4.5, seed=80 + i,
                   precision=U.FP32) for i, (s, b) in enumerate(zip([(36, 20, 12), (16, 16, 16), (32, 8, 24)],
                                                                      (1.0, 0.0, -1.0)))]

    def runs(stream):
        e = U.Ensemble(ps, stream=stream)
        out = []
        for mode, graph in ((U.ENS_PERSISTENT, True), (U.ENS_PER_STEP, True), (U.ENS_UNBATCHED, False)):
            e.run([9, 6, 4], mode=mode, use_graph=graph, detect_every=3, stream=stream)
            out.append([b.read_records(stream=stream) for b in e.boxes])
        out.append(e.status(stream=stream))
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        out.append([b.state().clone() for b in e.boxes])
        e.close()
        return out

    ref = runs(None)
    got = runs(torch.cuda.Stream())
    assert got[3] == 0 and all(bool(torch.isfinite(s).all()) for s in ref[-1])
    assert same(got, ref)
