"""GB300-native U(1)xU(1) lattice strings (arXiv:2208.01525) -- Python binding.

A thin layer over the C ABI of ``libu1u1`` (include/u1u1.h): PyTorch only
allocates the device field arrays and supplies CUDA streams; initial
conditions, leapfrog steps, winding detection, cell overlap and diagnostics
all run in the library's CUDA kernels.  There is no CPU fallback: without the
built library and a CUDA device, every call raises.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, fields

from . import _abi
from ._abi import (ENS_PER_STEP, ENS_PERSISTENT, ENS_UNBATCHED, FP32, FP64, KERNEL_AUTO,  # noqa: F401
                   KERNEL_SIMPLE, KERNEL_TILED, NFIELDS, NMOM, NPOS, U1U1Error, check, lib)

__all__ = ["Params", "Lattice", "Ensemble", "U1U1Error", "FP32", "FP64", "KERNEL_AUTO", "KERNEL_SIMPLE",
           "KERNEL_TILED", "coefficients", "version", "lib"]


@dataclass
class Params:
    """Model and lattice parameters (u1u1_params), named after the paper."""
    nx: int = 64
    ny: int = 64
    nz: int = 64
    dx: float = 0.5
    deta: float = 0.1
    eta0: float = 1.0
    m: float = 0.5
    eta_ref: float = 1.0
    beta: float = 1.0
    alpha: float = 2.0
    lambda_p: float = 2.0
    lambda_q: float = 2.0
    e_p: float = 1.0
    e_q: float = 1.0
    sigma_p: float = 1.0
    sigma_q: float = 1.0
    kappa: float = 0.9
    seed: int = 1
    precision: int = FP32

    @classmethod
    def cube(cls, n: int, **kw) -> "Params":
        return cls(nx=n, ny=n, nz=n, **kw)

    @property
    def nsites(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def c(self) -> _abi.CParams:
        cp = _abi.CParams()
        for f in fields(self):
            v = getattr(self, f.name)
            if f.name == "seed":
                v = int(v) & 0xFFFFFFFFFFFFFFFF
            setattr(cp, f.name, v)
        return cp


def version() -> str:
    return lib().u1u1_version().decode()


def coefficients(p: Params, n: int) -> dict:
    """Host-side step coefficients of step n (Eqs. 12, 19, 22)."""
    out = (ctypes.c_double * 6)()
    check(lib().u1u1_coefficients(ctypes.byref(p.c()), int(n), out))
    return dict(eta=out[0], a=out[1], c=out[2], delta=out[3], omega=out[4], ctilde=out[5])


def host_span_mapped(ptr: int, nbytes: int) -> bool:
    """Whether state transfers through the host span run on the SMs
    (page-locked, mapped, 16-byte aligned, inside one allocation)."""
    v = ctypes.c_int()
    check(lib().u1u1_host_span_mapped(ctypes.c_void_p(ptr), int(nbytes), ctypes.byref(v)))
    return bool(v.value)


def fp64_fma_rate(stream=None) -> float:
    """Measured FP64 fused-multiply-add rate of the current device, TFLOP/s."""
    v = ctypes.c_double()
    check(lib().u1u1_fp64_fma_rate(ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def inject_alloc_failure(nth: int) -> None:
    """Make the nth library allocation from now on fail as out of memory
    (0 disarms the hook)."""
    check(lib().u1u1_inject_alloc_failure(int(nth)))


def live_allocations() -> tuple:
    """(count, bytes) of the library's own allocations held at the moment."""
    c, b = ctypes.c_int64(), ctypes.c_int64()
    check(lib().u1u1_live_allocations(ctypes.byref(c), ctypes.byref(b)))
    return c.value, b.value


def set_alloc_guard(nbytes: int) -> None:
    """Guard zones of nbytes (a multiple of 256) around every library
    allocation made from now on (0: none)."""
    check(lib().u1u1_set_alloc_guard(int(nbytes)))


def check_alloc_guards() -> int:
    """Number of live library allocations whose guard zones were written."""
    v = ctypes.c_int64()
    check(lib().u1u1_check_alloc_guards(ctypes.byref(v)))
    return v.value


def check_params(p: Params) -> None:
    check(lib().u1u1_check_params(ctypes.byref(p.c())))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Lattice:
    """One lattice on one GPU: caller-owned field tensors plus a library handle.

    ``pos[k][f]`` (k = ping-pong buffer, f = U1U1_POS_* order) and ``mom[f]``
    are flat torch tensors of nx*ny*nz elements on the device.
    """

    def __init__(self, params: Params, device="cuda", init: bool = True, stream=None,
                 kernel: int = KERNEL_AUTO, guard: int = 0, _borrow=None):
        """guard > 0 (bytes, a multiple of 256): every field array, and every
        cell, winding and label array a call returns, sits between guard
        zones of a fixed pattern, a debugging aid that check_guards reads."""
        import torch
        check_params(params)
        if not torch.cuda.is_available():
            raise U1U1Error(-4, "no CUDA device: libu1u1 has no CPU path")
        self.params = params
        self.device = torch.device(device)
        self.dtype = torch.float64 if params.precision == FP64 else torch.float32
        self._owner = None
        self._guard = guard
        self._guarded = []     # (full tensor, guard elements) of the guarded field arrays
        self._guard_hits = 0   # output arrays found with a changed guard zone
        if _borrow is not None:  # a box of an Ensemble: tensors and handle belong to it
            self.pos, self.mom, handle, self._owner = _borrow
            self._bufs = None
            self._h = handle
            return
        self.pos, self.mom, self._bufs = _alloc_fields(params, self.dtype, self.device, guard, self._guarded)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if init:
                check(lib().u1u1_init_lattice(ctypes.byref(params.c()), ctypes.byref(self._bufs),
                                              _stream_ptr(stream), ctypes.byref(self._h)))
            else:
                check(lib().u1u1_attach_lattice(ctypes.byref(params.c()), ctypes.byref(self._bufs),
                                                0, 0, ctypes.byref(self._h)))
        if kernel != KERNEL_AUTO:
            self.set_kernel(kernel)

    # -- lifecycle --
    def close(self):
        if self._owner is not None:  # borrowed from an Ensemble
            self._h = ctypes.c_void_p()
            return
        if self._h:
            lib().u1u1_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state --
    def current(self):
        n = ctypes.c_int64()
        cur = ctypes.c_int()
        check(lib().u1u1_current(self._h, ctypes.byref(n), ctypes.byref(cur)))
        return n.value, cur.value

    @property
    def n(self) -> int:
        return self.current()[0]

    def check_guards(self) -> int:
        """Number of guarded arrays of this lattice (fields, and the outputs of
        past calls) whose guard zones were written: 0 unless something wrote
        past the end of an array."""
        return _guards_damaged(self._guarded) + self._guard_hits

    def fields(self):
        """The 20 current field tensors (positions of the current buffer, then momenta)."""
        cur = self.current()[1]
        return list(self.pos[cur]) + list(self.mom)

    def state(self):
        """Copy of the whole state as a (20, nz, ny, nx) tensor on the device."""
        import torch
        return torch.stack(self.fields()).view(NFIELDS, *self.params.shape)

    def set_state(self, st, n: int = 0):
        """Write a (20, nz, ny, nx) array (torch or numpy) into the current
        position buffer and the momenta, and set the step index to n.  The
        handle keeps its kernel choice, tuning, overlap tolerance and record
        ring.  Not for ensemble boxes, whose step index the ensemble tracks."""
        if self._owner is not None:
            raise U1U1Error(-8, "set_state is not available for ensemble boxes")
        import torch
        t = torch.as_tensor(st).to(device=self.device, dtype=self.dtype).reshape(NFIELDS, -1)
        cur = self.current()[1]
        for f in range(NPOS):
            self.pos[cur][f].copy_(t[f])
        for f in range(NMOM):
            self.mom[f].copy_(t[NPOS + f])
        torch.cuda.synchronize(self.device)
        check(lib().u1u1_set_params(self._h, ctypes.byref(self.params.c()), int(n)))

    def set_kernel(self, kernel: int):
        check(lib().u1u1_set_kernel(self._h, int(kernel)))

    def set_tile_waves(self, waves: int):
        """z-chunking of the tiled plain step (one of the tuner's wave targets)."""
        check(lib().u1u1_set_tile_waves(self._h, int(waves)))

    def autotune(self, cache_path=None, stream=None) -> dict:
        """Pick the step kernel and z-chunking by timing (state unchanged)."""
        k, w = ctypes.c_int(), ctypes.c_int()
        check(lib().u1u1_autotune(self._h, str(cache_path).encode() if cache_path else None, ctypes.byref(k),
                                  ctypes.byref(w), _stream_ptr(stream)))
        return {"kernel": k.value, "waves": w.value}

    def kernel(self) -> int:
        k = ctypes.c_int()
        check(lib().u1u1_get_kernel(self._h, ctypes.byref(k)))
        return k.value

    # -- the hot path --
    def step(self, nsteps: int = 1, detect_every: int = 0, stream=None):
        check(lib().u1u1_step(self._h, int(nsteps), int(detect_every), _stream_ptr(stream)))

    def cool(self, dt: float, nsteps: int, stream=None):
        """Diffusive cooling flow of Eqs. 27-30; momenta are zero afterwards."""
        check(lib().u1u1_cool(self._h, float(dt), int(nsteps), _stream_ptr(stream)))

    def set_params(self, params: Params, n: int, stream=None):
        """Switch to another phase's time-dependent parameters at step index n."""
        check(lib().u1u1_set_params(self._h, ctypes.byref(params.c()), int(n)))
        self.params = params

    def set_overlap_tol(self, tol: int):
        check(lib().u1u1_set_overlap_tol(self._h, int(tol)))

    def detect_strings(self, tol: int = 1, cells: bool = False, windings: bool = False, stream=None) -> dict:
        import torch
        V = self.params.nsites
        cp = cq = w = None
        out_guarded = []
        if cells:  # one buffer, the p and q arrays its two rows (256-byte aligned)
            vpad = (V + 255) // 256 * 256
            cbuf = _guarded_empty(2 * vpad, torch.uint8, self.device, self._guard, out_guarded).view(2, vpad)[:, :V]
            cp, cq = cbuf[0], cbuf[1]
        if windings:
            w = _guarded_empty(6 * V, torch.int8, self.device, self._guard, out_guarded)
        out = _abi.CStrings()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        check(lib().u1u1_detect_strings(self._h, int(tol), ptr(cp), ptr(cq), ptr(w), ctypes.byref(out),
                                        _stream_ptr(stream)))
        if out_guarded:
            self._guard_hits += _guards_damaged(out_guarded)
        res = _abi.struct_to_dict(out)
        if cells:
            res["cells"] = cbuf.view(2, *self.params.shape)
        if windings:
            res["windings"] = w.view(2, 3, *self.params.shape)
        return res

    def pq_segments(self, tol: int = 1, min_cells: int = 41, labels: bool = False, stream=None) -> dict:
        """Robust-method bound-state segments (connected pq-cell components)."""
        import torch
        out_guarded = []
        lab = _guarded_empty(self.params.nsites, torch.int32, self.device, self._guard, out_guarded) if labels else None
        out = _abi.CSegments()
        check(lib().u1u1_pq_segments(self._h, int(tol), int(min_cells),
                                     ctypes.c_void_p(lab.data_ptr()) if lab is not None else None,
                                     ctypes.byref(out), _stream_ptr(stream)))
        if out_guarded:
            self._guard_hits += _guards_damaged(out_guarded)
        res = _abi.struct_to_dict(out)
        if labels:
            res["labels"] = lab.view(*self.params.shape)
        return res

    def diagnostics(self, stream=None) -> dict:
        out = _abi.CDiag()
        check(lib().u1u1_diagnostics(self._h, ctypes.byref(out), _stream_ptr(stream)))
        return _abi.struct_to_dict(out)

    def read_records(self, max_records: int = 1024, stream=None):
        s = (_abi.CStrings * max_records)()
        d = (_abi.CDiag * max_records)()
        cnt = ctypes.c_int()
        lost = ctypes.c_int64()
        check(lib().u1u1_read_records(self._h, s, d, int(max_records), ctypes.byref(cnt), ctypes.byref(lost),
                                      _stream_ptr(stream)))
        recs = [(_abi.struct_to_dict(s[k]), _abi.struct_to_dict(d[k])) for k in range(cnt.value)]
        return recs, lost.value

    # -- host transfer and checkpoints --
    def upload(self, host_fields, stream=None):
        """Enqueue host -> device copies of 20 host tensors (pinned recommended:
        pinned, 16-byte aligned tensors are copied by the SMs)."""
        arr = (ctypes.c_void_p * NFIELDS)(*[t.data_ptr() for t in host_fields])
        check(lib().u1u1_upload_state(self._h, arr, _stream_ptr(stream)))

    def download(self, host_fields, stream=None):
        arr = (ctypes.c_void_p * NFIELDS)(*[t.data_ptr() for t in host_fields])
        check(lib().u1u1_download_state(self._h, arr, _stream_ptr(stream)))

    def save(self, path: str, stream=None):
        check(lib().u1u1_save(self._h, str(path).encode(), _stream_ptr(stream)))

    def load(self, path: str, stream=None):
        check(lib().u1u1_load(self._h, str(path).encode(), _stream_ptr(stream)))


def _guard_zones(full, g):
    """The two guard zones of a guarded tensor (g elements each side) as
    integer views, and the pattern they hold: a NaN for floating-point
    arrays (a read past the array brings a NaN into the result), 0xA5 bytes
    otherwise."""
    import torch
    n = full.numel() - 2 * g
    if full.dtype == torch.float32:
        iv, pat, r = full.view(torch.int32), 0x7FA5A5A5, 1
    elif full.dtype == torch.float64:
        iv, pat, r = full.view(torch.int64), 0x7FF5A5A5A5A5A5A5, 1
    else:
        iv, pat, r = full.view(torch.uint8), 0xA5, full.element_size()
    return (iv[: g * r], iv[(g + n) * r:]), pat


def _guarded_empty(n: int, dtype, device, guard: int, guarded: list):
    """A flat tensor of n elements.  With guard > 0 (bytes, a multiple of 256)
    it is the middle of a larger tensor whose guard zones on both sides hold
    a fixed pattern; (full, g) is appended to guarded for checking."""
    import torch
    if not guard:
        return torch.empty(n, dtype=dtype, device=device)
    es = torch.empty(0, dtype=dtype).element_size()
    if guard % 256:
        raise ValueError("guard must be a multiple of 256 bytes")
    g = guard // es
    full = torch.empty(n + 2 * g, dtype=dtype, device=device)
    zones, pat = _guard_zones(full, g)
    for z in zones:
        z.fill_(pat)
    guarded.append((full, g))
    return full[g:g + n]


def _guards_damaged(guarded: list) -> int:
    """Number of guarded tensors with a changed guard zone (synchronises the
    device first)."""
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    bad = 0
    for full, g in guarded:
        zones, pat = _guard_zones(full, g)
        bad += int(any(not bool((z == pat).all()) for z in zones))
    return bad


def _alloc_fields(params: Params, dtype, device, guard: int = 0, guarded: list = None):
    V = params.nsites
    guarded = [] if guarded is None else guarded
    pos = [[_guarded_empty(V, dtype, device, guard, guarded) for _ in range(NPOS)] for _ in range(2)]
    mom = [_guarded_empty(V, dtype, device, guard, guarded) for _ in range(NMOM)]
    bufs = _abi.CBuffers()
    for k in range(2):
        for f in range(NPOS):
            bufs.pos[k][f] = pos[k][f].data_ptr()
    for f in range(NMOM):
        bufs.mom[f] = mom[f].data_ptr()
    return pos, mom, bufs


class Ensemble:
    """Independent lattices of uneven size advanced together (u1u1_ensemble_*).

    ``boxes[b]`` is a Lattice view of box b (detection, diagnostics, state);
    its tensors and handle belong to the ensemble."""

    def __init__(self, params_list, device="cuda", horizon: int = 0, stream=None, guard: int = 0):
        """guard: as for Lattice, for every box's field arrays and outputs."""
        import torch
        if not torch.cuda.is_available():
            raise U1U1Error(-4, "no CUDA device: libu1u1 has no CPU path")
        self.params = list(params_list)
        self.device = torch.device(device)
        nb = len(self.params)
        cps = (_abi.CParams * nb)(*[p.c() for p in self.params])
        bufs = (_abi.CBuffers * nb)()
        fields = []
        self._guarded = []
        for b, p in enumerate(self.params):
            check_params(p)
            dtype = torch.float64 if p.precision == FP64 else torch.float32
            pos, mom, cb = _alloc_fields(p, dtype, self.device, guard, self._guarded)
            bufs[b] = cb
            fields.append((pos, mom))
        self._fields = fields
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().u1u1_ensemble_create(cps, nb, bufs, int(horizon), _stream_ptr(stream), ctypes.byref(self._h)))
        self.boxes = []
        for b, p in enumerate(self.params):
            hb = ctypes.c_void_p()
            check(lib().u1u1_ensemble_lattice(self._h, b, ctypes.byref(hb)))
            pos, mom = fields[b]
            self.boxes.append(Lattice(p, device=device, guard=guard, _borrow=(pos, mom, hb, self)))

    def run(self, steps, mode: int = ENS_PERSISTENT, use_graph: bool = False, detect_every: int = 0, stream=None):
        """Advance box b by steps[b]; with detect_every > 0 the detection records
        go to each box's ring (``boxes[b].read_records()``)."""
        arr = (ctypes.c_int * len(self.params))(*[int(s) for s in steps])
        check(lib().u1u1_ensemble_run(self._h, arr, int(detect_every), int(mode), int(bool(use_graph)),
                                      _stream_ptr(stream)))

    def autotune(self, probe_steps: int = 4, stream=None) -> dict:
        """Pick the work-item z-chunk, the persistent kernel's tensor copies and
        the schedule by timing (states unchanged)."""
        m, lz = ctypes.c_int(), ctypes.c_int()
        check(lib().u1u1_ensemble_autotune(self._h, int(probe_steps), ctypes.byref(m), ctypes.byref(lz),
                                           _stream_ptr(stream)))
        return {"mode": m.value, "item_lz": lz.value, "persistent_tma": self.tuning()["persistent_tma"]}

    def tuning(self) -> dict:
        lz, t = ctypes.c_int(), ctypes.c_int()
        check(lib().u1u1_ensemble_get_tuning(self._h, ctypes.byref(lz), ctypes.byref(t)))
        return {"item_lz": lz.value, "persistent_tma": bool(t.value)}

    def set_tuning(self, item_lz: int = 32, persistent_tma: bool = True, stream=None):
        """Work-item z-chunk and the persistent kernel's tensor copies, without timing."""
        check(lib().u1u1_ensemble_set_tuning(self._h, int(item_lz), int(bool(persistent_tma)), _stream_ptr(stream)))

    def check_guards(self) -> int:
        """Number of guarded arrays of every box (fields and past outputs)
        whose guard zones were written."""
        return _guards_damaged(self._guarded) + sum(b._guard_hits for b in self.boxes)

    def status(self, stream=None) -> int:
        v = ctypes.c_int()
        check(lib().u1u1_ensemble_status(self._h, ctypes.byref(v), _stream_ptr(stream)))
        return v.value

    def set_wait_limit(self, ns: int):
        check(lib().u1u1_ensemble_set_wait_limit(self._h, int(ns)))

    def inject_unreachable_wait(self, enable: bool = True):
        check(lib().u1u1_ensemble_inject_unreachable_wait(self._h, int(bool(enable))))

    def close(self):
        if self._h:
            for b in self.boxes:
                b._h = ctypes.c_void_p()
            lib().u1u1_ensemble_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def nan_to_none(d: dict) -> dict:
    return {k: (None if isinstance(v, float) and math.isnan(v) else v) for k, v in d.items()}
