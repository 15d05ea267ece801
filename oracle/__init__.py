"""FP64 CPU oracle for the U(1)xU(1) lattice step (arXiv:2208.01525).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it and shares no code with it.

The arithmetic lives in ``u1u1_oracle.c`` (plain C, double precision, three
unfused passes per leapfrog step, Sec. III of the paper).  This module builds
it with gcc, wraps it with ctypes, and adds the host formulas of Sec. III.A
(Eqs. 31-37) that turn lattice sums into mean string separations, bound-state
fractions and velocity estimators.

State arrays are numpy float64 of shape (20, nz, ny, nx) in the field order
documented at the top of ``u1u1_oracle.c``.
"""
from __future__ import annotations

import contextlib
import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "u1u1_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_LIB_DIR, "liboracle.so")

NFIELDS = 20
# field indices (data format shared with the product library's state arrays)
PHI = ((0, 1), (2, 3))          # [sector][re/im]
A = ((4, 5, 6), (7, 8, 9))      # [sector][direction]
PI = ((10, 11), (12, 13))
E = ((14, 15, 16), (17, 18, 19))
POS_FIELDS = tuple(range(10))
MOM_FIELDS = tuple(range(10, 20))

DIAG_NAMES = (
    "kin_p", "kin_q", "grad_p", "grad_q", "el_p", "el_q", "mag_p", "mag_q", "pot", "vint",
    "lag", "energy", "rl_num", "rl_den", "rpq_num", "rpq_den",
    "gauss_sum_p", "gauss_sum_q", "charge_sum_p", "charge_sum_q", "pot_p", "pot_q",
    "gauss_max_p", "gauss_max_q", "phi_min_p", "phi_max_p", "phi_min_q", "phi_max_q",
    "nan_count",
)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("deta", ctypes.c_double), ("eta0", ctypes.c_double),
        ("m", ctypes.c_double), ("eta_ref", ctypes.c_double), ("beta", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("lambda_", ctypes.c_double * 2), ("e", ctypes.c_double * 2), ("sigma", ctypes.c_double * 2),
        ("kappa", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


@dataclass
class Params:
    """Model and lattice parameters, named after the paper's symbols."""
    nx: int
    ny: int
    nz: int
    dx: float = 0.5
    deta: float = 0.1
    eta0: float = 1.0
    m: float = 0.5
    eta_ref: float = 1.0
    beta: float = 1.0
    alpha: float = 2.0
    lam: tuple = (2.0, 2.0)
    e: tuple = (1.0, 1.0)
    sigma: tuple = (1.0, 1.0)
    kappa: float = 0.9
    seed: int = 1

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nsites(self):
        return self.nx * self.ny * self.nz

    def c(self) -> _CParams:
        cp = _CParams()
        cp.nx, cp.ny, cp.nz = self.nx, self.ny, self.nz
        cp.dx, cp.deta, cp.eta0 = self.dx, self.deta, self.eta0
        cp.m, cp.eta_ref, cp.beta, cp.alpha = self.m, self.eta_ref, self.beta, self.alpha
        cp.lambda_[:] = list(self.lam)
        cp.e[:] = list(self.e)
        cp.sigma[:] = list(self.sigma)
        cp.kappa = self.kappa
        cp.seed = self.seed & 0xFFFFFFFFFFFFFFFF
        return cp


_lib = None


def _load(path: str):
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(_CParams)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_coeffs.argtypes = [P, ctypes.c_long, dp]
    L.orc_init.argtypes = [P, dp]
    L.orc_scalar_kick.argtypes = [P, dp, ctypes.c_long, dp]
    L.orc_gauge_kick.argtypes = [P, dp, ctypes.c_long, dp]
    L.orc_step.argtypes = [P, dp, ctypes.c_long, ctypes.c_int, dp]
    L.orc_cool.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, dp]
    L.orc_windings.argtypes = [P, dp, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_cells.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_overlap.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.orc_overlap.restype = ctypes.c_long
    L.orc_diagnostics.argtypes = [P, dp, ctypes.c_long, dp, dp]
    L.orc_pq_mask.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.orc_components.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_diag_count.restype = ctypes.c_int
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_max_threads.restype = ctypes.c_int
    assert L.orc_diag_count() == len(DIAG_NAMES)
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def compile_variant(source: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (used by the tests that
    check that the pins catch planted mistakes)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", out_path, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call to another build of the source."""
    global _lib
    old = _lib
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = old


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def coeffs(p: Params, n: int) -> dict:
    """eta_n, a_n, c_n = a^{2 beta}, delta_n (Eq. 19), omega_n (Eq. 22), charge factor."""
    out = np.zeros(6)
    lib().orc_coeffs(ctypes.byref(p.c()), int(n), _dptr(out))
    return dict(eta=out[0], a=out[1], c=out[2], delta=out[3], omega=out[4], ctilde=out[5])


def new_state(p: Params) -> np.ndarray:
    return np.zeros((NFIELDS,) + p.shape, dtype=np.float64)


def init(p: Params) -> np.ndarray:
    """Random-phase initial conditions of Sec. III (SplitMix64 phases)."""
    st = new_state(p)
    lib().orc_init(ctypes.byref(p.c()), _dptr(st))
    return st


def _scratch(p: Params) -> np.ndarray:
    return np.zeros((10,) + p.shape, dtype=np.float64)


def step(p: Params, st: np.ndarray, n0: int, nsteps: int = 1) -> np.ndarray:
    """Advance st (in place) by nsteps leapfrog steps starting at step index n0."""
    assert st.shape == (NFIELDS,) + p.shape
    lib().orc_step(ctypes.byref(p.c()), _dptr(st), int(n0), int(nsteps), _dptr(_scratch(p)))
    return st


def kicks(p: Params, st: np.ndarray, n: int):
    """Half-step momenta (pi^{n+1/2} [4,...], E^{n+1/2} [6,...]) without drifting."""
    pi_new = np.zeros((4,) + p.shape)
    e_new = np.zeros((6,) + p.shape)
    lib().orc_scalar_kick(ctypes.byref(p.c()), _dptr(st), int(n), _dptr(pi_new))
    lib().orc_gauge_kick(ctypes.byref(p.c()), _dptr(st), int(n), _dptr(e_new))
    return pi_new, e_new


def cool(p: Params, st: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """Diffusive cooling flow of Eqs. 27-30 (forward Euler, in place)."""
    lib().orc_cool(ctypes.byref(p.c()), _dptr(st), float(dt), int(nsteps), _dptr(_scratch(p)))
    return st


def windings(p: Params, st: np.ndarray):
    """Signed plaquette windings W[2, 3, nz, ny, nx] (int8) and branch-cut flags."""
    W = np.zeros((2, 3) + p.shape, dtype=np.int8)
    F = np.zeros((2, 3) + p.shape, dtype=np.uint8)
    lib().orc_windings(ctypes.byref(p.c()), _dptr(st), W.ctypes.data, F.ctypes.data)
    return W, F


def cells(p: Params, W: np.ndarray) -> np.ndarray:
    """Per-sector cell arrays [2, nz, ny, nx] (uint8): sum of |W| over the 6 faces."""
    W = np.ascontiguousarray(W, dtype=np.int8)
    C = np.zeros((2,) + p.shape, dtype=np.uint8)
    lib().orc_cells(ctypes.byref(p.c()), W.ctypes.data, C.ctypes.data)
    return C


def overlap(p: Params, anchor: np.ndarray, other: np.ndarray, tol: int) -> int:
    """Number of anchor cells with a non-zero other cell within tol cells."""
    a = np.ascontiguousarray(anchor, dtype=np.uint8)
    o = np.ascontiguousarray(other, dtype=np.uint8)
    return int(lib().orc_overlap(ctypes.byref(p.c()), a.ctypes.data, o.ctypes.data, int(tol)))


def pq_mask(p: Params, anchor: np.ndarray, other: np.ndarray, tol: int) -> np.ndarray:
    """Cells of the fast method's bound-state overlap (uint8 0/1)."""
    a = np.ascontiguousarray(anchor, dtype=np.uint8)
    o = np.ascontiguousarray(other, dtype=np.uint8)
    m = np.zeros(p.shape, dtype=np.uint8)
    lib().orc_pq_mask(ctypes.byref(p.c()), a.ctypes.data, o.ctypes.data, int(tol), m.ctypes.data)
    return m


def components(p: Params, mask: np.ndarray) -> np.ndarray:
    """Periodic 26-connected components: smallest site index per component, -1 outside."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    lab = np.zeros(p.shape, dtype=np.int64)
    lib().orc_components(ctypes.byref(p.c()), m.ctypes.data, lab.ctypes.data)
    return lab


def segments(p: Params, st: np.ndarray, tol: int = 1, min_cells: int = 41) -> dict:
    """Robust-method bound-state segments (Sec. III.B, Eq. 38): connected
    components of the pq cells; a segment of N cells has length (N - 1) dx
    and counts when N > min_cells; N_pq segments, L_pq their total length,
    l_pq = L_pq / N_pq, xi_pq = sqrt(V / L_pq)."""
    W, _ = windings(p, st)
    C = cells(p, W)
    mask = pq_mask(p, C[0], C[1], tol)
    lab = components(p, mask)
    roots, sizes = np.unique(lab[lab >= 0], return_counts=True)
    keep = sizes > min_cells
    L = p.dx * float((sizes[keep] - 1).sum())
    n_seg = int(keep.sum())
    vol = p.nsites * p.dx ** 3
    return dict(n_cells=int(mask.sum()), n_components=int(len(roots)), n_segments=n_seg,
                largest=int(sizes.max()) if len(sizes) else 0, L_pq=L,
                l_pq=(L / n_seg) if n_seg else math.nan, xi_pq=_sqrt_ratio(vol, L),
                labels=lab, mask=mask)


def diagnostic_sums(p: Params, st: np.ndarray, n: int) -> dict:
    out = np.zeros(len(DIAG_NAMES))
    lib().orc_diagnostics(ctypes.byref(p.c()), _dptr(st), int(n), _dptr(out), _dptr(_scratch(p)))
    return dict(zip(DIAG_NAMES, out.tolist()))


# ---- host formulas of Sec. III.A -------------------------------------------

def _sqrt_ratio(num: float, den: float) -> float:
    if den == 0.0:
        return math.inf
    r = num / den
    return math.sqrt(r) if r >= 0.0 else math.nan


def strings(p: Params, st: np.ndarray, tol: int = 1) -> dict:
    """Windings, cell overlap and the string-length estimators.

    L_pq = dx * N_pq^cell (fast method, no off-by-one correction, Sec. III.B);
    L_s  = dx * sum_plaquettes |W_s| - L_pq (Sec. III.A);
    xi_s, xi_pq (Eq. 31), xi_W (Eq. 32), f_total (Eq. 34), f_p (Eq. 35).
    """
    W, F = windings(p, st)
    C = cells(p, W)
    absW = np.abs(W.astype(np.int64))
    n_p = int(absW[0].sum())
    n_q = int(absW[1].sum())
    both = (W[0] != 0) & (W[1] != 0)
    n_pq_cell = overlap(p, C[0], C[1], tol)
    n_pq_cell_q = overlap(p, C[1], C[0], tol)
    dx = p.dx
    vol = p.nsites * dx ** 3
    L_pq = dx * n_pq_cell
    L_p = dx * n_p - L_pq
    L_q = dx * n_q - L_pq
    tot = L_p + L_q + L_pq
    return dict(
        n_p=n_p, n_q=n_q, n_pq_plaq=int(both.sum()), n_pq_cell=n_pq_cell,
        n_pq_cell_q=n_pq_cell_q, n_flagged=int(F.sum()),
        max_abs_w=int(absW.max()) if absW.size else 0,
        nonzero_p=int((W[0] != 0).sum()), nonzero_q=int((W[1] != 0).sum()),
        n_w2_p=int((absW[0] >= 2).sum()), n_w2_q=int((absW[1] >= 2).sum()),
        n_cells_ge4_p=int((C[0] >= 4).sum()), n_cells_ge4_q=int((C[1] >= 4).sum()),
        L_p=L_p, L_q=L_q, L_pq=L_pq,
        xi_p=_sqrt_ratio(vol, L_p), xi_q=_sqrt_ratio(vol, L_q), xi_pq=_sqrt_ratio(vol, L_pq),
        xi_w=_sqrt_ratio(vol, tot),
        f_total=(L_pq / tot) if tot != 0 else math.nan,
        f_p=(L_pq / L_p) if L_p != 0 else math.nan,
        W=W, flags=F, cells=C,
    )


def diagnostics(p: Params, st: np.ndarray, n: int) -> dict:
    """Lattice sums plus xi_L (Eq. 33) and <v^2> (Eqs. 36-37) for W = L and W = V_int."""
    s = diagnostic_sums(p, st, n)
    dx3 = p.dx ** 3
    vol = p.nsites * dx3
    mu = 2.0 * math.pi * p.sigma[0] ** 2  # tension of a basic BPS string
    out = dict(s)
    cf = coeffs(p, n)
    out.update(eta=cf["eta"], a=cf["a"], n=n)
    out["energy_total"] = dx3 * s["energy"]
    out["lag_total"] = dx3 * s["lag"]
    out["xi_l"] = _sqrt_ratio(-mu * vol, dx3 * s["lag"])
    # per-sector Lagrangians (self-potential only, the interaction term left
    # out) and their separations with mu_s = 2 pi sigma_s^2 (unequal tensions)
    for k, sec in enumerate("pq"):
        lag_s = dx3 * ((s["kin_" + sec] - s["grad_" + sec] + s["el_" + sec] - s["mag_" + sec]) - s["pot_" + sec])
        out["lag_" + sec] = lag_s
        out["xi_l_" + sec] = _sqrt_ratio(-2.0 * math.pi * p.sigma[k] ** 2 * vol, lag_s)
    for tag, num, den in (("l", "rl_num", "rl_den"), ("pq", "rpq_num", "rpq_den")):
        R = s[num] / s[den] if s[den] != 0.0 else math.nan
        out["R_" + tag] = R
        out["v2_" + tag] = 2.0 * R / (1.0 + R) if R == R else math.nan
    for sec in ("p", "q"):
        cs = s["charge_sum_" + sec]
        out["gauss_rel_" + sec] = s["gauss_sum_" + sec] / cs if cs != 0.0 else math.nan
    return out
