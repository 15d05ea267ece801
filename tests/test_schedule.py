"""The run schedule (Sec. III, Sec. V, Table 3): the core-growth exponent
rule reproduces the paper's printed beta_growth, and (GPU) a compressed
schedule on a small lattice matches the oracle run through the same phases.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import schedule as S

HERE = os.path.dirname(os.path.abspath(__file__))


def table3():
    with open(os.path.join(HERE, "golden", "table3.json")) as f:
        return json.load(f)


def test_growth_beta_reproduces_table3():
    t = table3()
    for row in t["rows"]:
        if row["beta"] != 1.0:
            continue
        bg = S.growth_beta(row["m"], row["r_s_max"], t["damping"]["eta_end"], row["eta_tr"])
        assert abs(bg - row["beta_growth"]) < 1e-4 * abs(row["beta_growth"]), (bg, row)
        # the physical phase's radius at the transition, r = (eta_end/eta_tr)^{m/(1-m)}
        pm = row["m"] / (1 - row["m"])
        assert abs((t["eta_end"] / row["eta_tr"]) ** pm / row["r_s_max"] - 1) < 0.011


def test_schedule_phases_follow_table3():
    """Every row of Table 3 (golden file): cooling from eta = -10 to 1 in steps
    of 1/30; damping from eta = 1 to 5 at constant comoving width (beta = 0)
    with the row's m_damp; then, for physical runs, core growth with the row's
    beta_growth to eta_tr and beta = 1 to the end with a = 1 at the end, and
    for constant-width runs beta = 0 to the end."""
    t = table3()
    de = 0.1
    base = U.Params.cube(16, deta=de)
    cool, damp = t["cooling"], t["damping"]
    for row in t["rows"]:
        era = "radiation" if row["m"] == 0.5 else "matter"
        physical = row["beta"] == 1.0
        ph = S.paper_schedule(base, era, physical=physical, eta_end=t["eta_end"],
                              eta_tr=row["eta_tr"] if physical else 343.0)
        assert ph[0].kind == "cool" and abs(ph[0].dt - cool["deta"]) < 1e-15
        assert ph[0].nsteps == round((cool["eta_end"] - cool["eta_start"]) / cool["deta"])
        d = ph[1]
        assert d.kind == "leapfrog" and d.params.m == row["m_damp"] and d.params.beta == damp["beta"]
        assert d.params.eta0 == damp["eta_start"] and d.nsteps == round((damp["eta_end"] - damp["eta_start"]) / de)
        if physical:
            g, f = ph[2], ph[3]
            assert len(ph) == 4 and g.params.m == row["m"] and f.params.m == row["m"]
            # r_max from continuity at eta_tr, (eta_end / eta_tr)^{m/(1-m)}, is
            # within 1.1 % of the printed r_s_max, so beta_growth is within 1 %
            pm = row["m"] / (1 - row["m"])
            want = S.growth_beta(row["m"], (t["eta_end"] / row["eta_tr"]) ** pm, damp["eta_end"], row["eta_tr"])
            assert g.params.beta == want
            assert abs(g.params.beta - row["beta_growth"]) < 1e-2 * abs(row["beta_growth"])
            assert g.params.eta0 == damp["eta_end"] and g.nsteps == round((row["eta_tr"] - damp["eta_end"]) / de)
            assert f.params.beta == 1.0 and f.params.eta0 == row["eta_tr"] and f.params.eta_ref == t["eta_end"]
            assert f.nsteps == round((t["eta_end"] - row["eta_tr"]) / de)
        else:
            f = ph[2]
            assert len(ph) == 3 and f.params.m == row["m"] and f.params.beta == row["beta"] == 0.0
            assert f.params.eta0 == damp["eta_end"] and f.nsteps == round((t["eta_end"] - damp["eta_end"]) / de)


def test_schedule_phases_are_continuous():
    base = U.Params.cube(16, deta=0.1)
    ph = S.paper_schedule(base, "matter", physical=True, eta_end=20.0, eta_tr=12.0)
    assert [p.kind for p in ph] == ["cool", "leapfrog", "leapfrog", "leapfrog"]
    assert ph[0].nsteps == 330
    g, f = ph[2].params, ph[3].params
    cg = (12.0 / g.eta_ref) ** (2 * g.m / (1 - g.m) * g.beta)
    cf = (12.0 / f.eta_ref) ** (2 * f.m / (1 - f.m) * f.beta)
    assert abs(cg / cf - 1) < 1e-12  # a^{2 beta} continuous at the transition


def oracle_run(p, phases, st):
    for ph in phases:
        if ph.kind == "cool":
            O.cool(p, st, ph.dt, ph.nsteps)
            st[10:] = 0.0
        else:
            q = ph.params
            op = O.Params(q.nx, q.ny, q.nz, dx=q.dx, deta=q.deta, eta0=q.eta0, m=q.m, eta_ref=q.eta_ref, beta=q.beta,
                          alpha=q.alpha, lam=(q.lambda_p, q.lambda_q), e=(q.e_p, q.e_q),
                          sigma=(q.sigma_p, q.sigma_q), kappa=q.kappa, seed=q.seed)
            O.step(op, st, 0, ph.nsteps)
    return st


@pytest.mark.gpu
@pytest.mark.parametrize("era,physical,unequal", [("radiation", True, False), ("matter", True, False),
                                                  ("matter", False, False), ("radiation", True, True)])
def test_schedule_gpu_matches_oracle(era, physical, unequal):
    """The whole run schedule (cooling flow, damping, core growth, physical
    evolution), FP64 GPU against the oracle; the last case with every
    per-sector coupling different (the cooling flow's per-sector
    coefficients included)."""
    torch = pytest.importorskip("torch")
    kw = dict(lambda_p=2.0, lambda_q=1.62, e_p=1.0, e_q=0.9, sigma_p=1.0, sigma_q=0.8, kappa=0.5) if unequal else {}
    base = U.Params(nx=20, ny=16, nz=12, seed=21, precision=U.FP64, **kw)
    phases = S.paper_schedule(base, era, physical=physical, eta_end=9.0, eta_tr=7.0)
    lat = U.Lattice(base)
    S.run(lat, phases)
    got = lat.state().cpu().numpy()
    p0 = O.Params(20, 16, 12, seed=21, lam=(base.lambda_p, base.lambda_q), e=(base.e_p, base.e_q),
                  sigma=(base.sigma_p, base.sigma_q), kappa=base.kappa)
    ref = oracle_run(p0, phases, O.init(p0))
    # relative to each field's maximum, but never to a scale below the unit
    # vacuum value: after the heavily damped phase (m_damp gives delta ~ 2)
    # the momenta are many orders of magnitude below the fields
    scale = np.maximum(np.abs(ref).reshape(20, -1).max(axis=1), 1.0)
    err = np.abs(got - ref).reshape(20, -1).max(axis=1) / scale
    assert err.max() < 1e-10, err
    assert torch.cuda.is_available()


class RingLattice:
    """Host stand-in with a lattice handle's record semantics: a step whose
    input index n has n % detect_every == 0 appends a record, and the ring
    keeps the last 1024, counting the ones overwritten before being read."""

    def __init__(self):
        self.n = 0
        self.ring = []
        self.lost = 0
        self.calls = []

    def cool(self, dt, nsteps, stream=None):
        self.calls.append(("cool", nsteps))

    def set_params(self, params, n, stream=None):
        self.n = n

    def step(self, nsteps, detect_every=0, stream=None):
        self.calls.append(("step", nsteps))
        for _ in range(nsteps):
            if detect_every and self.n % detect_every == 0:
                self.ring.append(({"n": self.n, "xi_w": math.inf}, {"n": self.n, "lag": math.nan}))
                if len(self.ring) > 1024:
                    self.ring.pop(0)
                    self.lost += 1
            self.n += 1

    def read_records(self, max_records=1024, stream=None):
        recs, self.ring = self.ring[:max_records], self.ring[max_records:]
        lost, self.lost = self.lost, 0
        return recs, lost


def test_run_reads_every_record_of_long_phases(tmp_path):
    """A phase with more detections than the record ring holds is stepped in
    ring-sized chunks: every record reaches the JSON-lines log, in order,
    with non-finite values as null."""
    base = U.Params.cube(8, deta=0.1)
    phases = [S.Phase("cool", 5, dt=0.1), S.Phase("leapfrog", 2500, params=base),
              S.Phase("leapfrog", 7, params=base)]
    lat = RingLattice()
    log = tmp_path / "records.jsonl"
    assert S.run(lat, phases, detect_every=2, log=str(log)) == 1250 + 4
    assert lat.calls == [("cool", 5), ("step", 2048), ("step", 452), ("step", 7)]
    lines = [json.loads(s) for s in log.read_text().splitlines()]
    assert [r["phase"] for r in lines] == [1] * 1250 + [2] * 4
    assert [r["strings"]["n"] for r in lines] == list(range(0, 2500, 2)) + [0, 2, 4, 6]
    assert all(r["strings"]["xi_w"] is None and r["diag"]["lag"] is None for r in lines)
    # without detection a phase is one call and nothing is read
    lat = RingLattice()
    assert S.run(lat, phases) == 0 and lat.calls == [("cool", 5), ("step", 2500), ("step", 7)]


def test_run_reports_records_lost_before_it_started():
    lat = RingLattice()
    lat.step(1100, detect_every=1)  # 76 records overwritten before the run
    with pytest.raises(RuntimeError, match="overwritten"):
        S.run(lat, [S.Phase("leapfrog", 4, params=U.Params.cube(8))], detect_every=1)


@pytest.mark.gpu
def test_schedule_log_keeps_every_record_on_gpu(tmp_path):
    """A leapfrog phase with more detections (1100) than the record ring
    holds, on a lattice handle: the runner steps it in ring-sized chunks,
    every record reaches the log in order, the last one is what a standalone
    detection reports on the same state, and the state is that of a run
    without detection."""
    torch = pytest.importorskip("torch")
    base = U.Params.cube(16, m=0.5, beta=1.0, eta0=1.0, eta_ref=111.0, seed=8)
    lat = U.Lattice(base)
    log = tmp_path / "records.jsonl"
    assert S.run(lat, [S.Phase("leapfrog", 1100, params=base)], detect_every=1, log=str(log)) == 1100
    lines = [json.loads(s) for s in log.read_text().splitlines()]
    assert [r["strings"]["n"] for r in lines] == list(range(1100))
    assert all(r["phase"] == 0 for r in lines)
    ref = U.Lattice(base)
    ref.step(1099)
    s_ref = ref.detect_strings(tol=1)
    for k in ("n_p", "n_q", "nonzero_p", "nonzero_q", "n_pq_plaq", "n_pq_cell", "n_flagged"):
        assert lines[-1]["strings"][k] == s_ref[k], k
    ref.step(1)
    assert torch.equal(lat.state(), ref.state())
