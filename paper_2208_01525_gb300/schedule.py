"""Run schedule of the paper's production runs (Sec. III, Sec. V, Table 3).

A run is a list of phases applied to one lattice:

1. diffusive cooling (Eqs. 27-30) from eta = -10 to 1 in steps of 1/30;
2. a damping period from eta = 1 to 5 with a fast expansion law m_damp
   (0.95 before radiation, 0.75 before matter) at constant comoving width
   (beta = 0);
3. for physical runs, core growth with beta_growth < 0 up to the transition
   time eta_tr, then beta = 1 to the end, the scale factor normalised so that
   the string radius is 1 at the end; for constant-width runs, beta = 0 to the
   end.

Reading of the core-growth rule (Sec. V): during growth the scale factor is
normalised to 1 at the start of the phase, so the radius starts at 1 and
grows like a^{-beta_growth}; with the physical phase normalised to a = 1 at
the end, its radius at eta_tr is r_max = (eta_end / eta_tr)^{m/(1-m)}, and
beta_growth = -ln(r_max) / (m/(1-m) ln(eta_tr / eta_start)) makes the radius
and the coupling factor a^{2 beta} continuous at eta_tr.  With eta_start = 5,
eta_tr = 343 and r_max = 3 (radiation) or 9 (matter) this reproduces the
paper's beta_growth to 1e-4.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from dataclasses import dataclass

from . import Params


@dataclass
class Phase:
    kind: str            # "cool" or "leapfrog"
    nsteps: int
    dt: float = 0.0      # cooling step
    params: Params = None  # leapfrog phase parameters (eta0 = phase start, step index from 0)


def growth_beta(m: float, r_max: float, eta_start: float, eta_tr: float) -> float:
    pm = m / (1.0 - m)
    return -math.log(r_max) / (pm * math.log(eta_tr / eta_start))


def paper_schedule(base: Params, era: str = "radiation", physical: bool = True, eta_end: float = 1024.0,
                   eta_tr: float = 343.0, cool=(-10.0, 1.0, 1.0 / 30.0), damp=(1.0, 5.0)) -> list:
    """Phases of one run; lattice, couplings and seed come from base, Delta eta
    from base.deta."""
    m = 0.5 if era == "radiation" else 2.0 / 3.0
    m_damp = 0.95 if era == "radiation" else 0.75
    de = base.deta
    phases = [Phase("cool", int(round((cool[1] - cool[0]) / cool[2])), dt=cool[2])]

    def leap(eta_a, eta_b, **kw):
        n = int(round((eta_b - eta_a) / de))
        return Phase("leapfrog", n, params=dataclasses.replace(base, eta0=eta_a, **kw))

    phases.append(leap(damp[0], damp[1], m=m_damp, beta=0.0, eta_ref=damp[0]))
    if not physical:
        phases.append(leap(damp[1], eta_end, m=m, beta=0.0, eta_ref=damp[1]))
        return phases
    pm = m / (1.0 - m)
    r_max = (eta_end / eta_tr) ** pm
    bg = growth_beta(m, r_max, damp[1], eta_tr)
    phases.append(leap(damp[1], eta_tr, m=m, beta=bg, eta_ref=damp[1]))
    phases.append(leap(eta_tr, eta_end, m=m, beta=1.0, eta_ref=eta_end))
    return phases


RING_RECORDS = 1024  # capacity of a handle's detection-record ring (u1u1_read_records)


def _json_value(v):
    if isinstance(v, float) and not math.isfinite(v):
        return None
    return v


def record_line(phase: int, strings: dict, diag: dict) -> str:
    """One detection record as a JSON line: the phase index, the string
    estimators and the diagnostics (Sec. III.A, Eqs. 31-37); NaN and
    infinities (e.g. xi_W with no strings) are written as null."""
    rec = {"phase": phase,
           "strings": {k: _json_value(v) for k, v in strings.items()},
           "diag": {k: _json_value(v) for k, v in diag.items()}}
    return json.dumps(rec, allow_nan=False)


def run(lat, phases, detect_every: int = 0, log=None, stream=None) -> int:
    """Apply the phases to a Lattice (cooling, then leapfrog phases).

    With detect_every > 0 every leapfrog phase is stepped in chunks of at
    most RING_RECORDS detection periods, and each chunk's records are read
    before the next chunk starts, so no record is overwritten in the
    handle's ring however long the phase; with a log (a path, appended to,
    or a text file) every record goes to it as one JSON line
    (record_line).  Returns the number of records read."""
    if detect_every < 0:
        raise ValueError("detect_every must be >= 0")
    out = open(log, "a") if isinstance(log, (str, os.PathLike)) else log
    nrec = 0
    try:
        for i, ph in enumerate(phases):
            if ph.kind == "cool":
                lat.cool(ph.dt, ph.nsteps, stream=stream)
                continue
            lat.set_params(ph.params, 0)
            if detect_every == 0:
                lat.step(ph.nsteps, stream=stream)
                continue
            left = ph.nsteps
            while left > 0:
                chunk = min(left, RING_RECORDS * detect_every)
                lat.step(chunk, detect_every=detect_every, stream=stream)
                left -= chunk
                recs, lost = lat.read_records(max_records=RING_RECORDS, stream=stream)
                if lost:
                    raise RuntimeError(f"{lost} detection records were overwritten before they were read")
                nrec += len(recs)
                if out is not None:
                    for strings, diag in recs:
                        out.write(record_line(i, strings, diag) + "\n")
    finally:
        if out is not None and out is not log:
            out.close()
    return nrec
