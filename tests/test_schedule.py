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
