"""Failure detection on the host side: each library allocation of a lattice
handle, of its segment scratch, of an ensemble, of an ensemble run with
detection and of the ensemble autotuner is made to fail in turn.  Every such
call returns OUT_OF_MEMORY, releases what it had taken (the library's live
allocations go back to where they were, up to the schedules a run keeps
cached) and leaves the handle or ensemble usable: a run after the failures
gives the same state, bit for bit, as a run that saw none.  No GPU fault is
involved: the failing allocation never reaches the device.
"""
import math

import pytest

import paper_2208_01525_gb300 as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OUT_OF_MEMORY = -3


@pytest.fixture(autouse=True)
def disarm():
    U.inject_alloc_failure(0)
    yield
    U.inject_alloc_failure(0)


def live():
    return U.live_allocations()


def same(a: dict, b: dict) -> bool:
    """Equal dicts, NaN equal to NaN."""
    def eq(x, y):
        return x == y or (isinstance(x, float) and isinstance(y, float) and math.isnan(x) and math.isnan(y))
    return a.keys() == b.keys() and all(eq(a[k], b[k]) for k in a)


def fails_with_oom(fn):
    with pytest.raises(U.U1U1Error) as ei:
        fn()
    assert ei.value.code == OUT_OF_MEMORY, str(ei.value)


def test_lattice_creation_fails_cleanly_at_every_allocation():
    p = U.Params(nx=16, ny=12, nz=8, seed=3)
    base = live()
    lat = U.Lattice(p)
    n_alloc = live()[0] - base[0]
    ref = lat.state().clone()
    lat.close()
    assert live() == base and n_alloc >= 10
    for k in range(1, n_alloc + 1):
        U.inject_alloc_failure(k)
        fails_with_oom(lambda: U.Lattice(p))
        assert live() == base, k
    lat = U.Lattice(p)  # the hook fired and is disarmed
    assert torch.equal(lat.state(), ref)
    lat.close()
    assert live() == base


def test_segment_scratch_fails_cleanly():
    p = U.Params(nx=16, ny=16, nz=16, seed=4)
    lat = U.Lattice(p)
    lat.step(20)
    held = live()
    for k in range(1, 5):
        U.inject_alloc_failure(k)
        fails_with_oom(lambda: lat.pq_segments())
        assert live() == held, k
    first = lat.pq_segments()
    assert live()[0] == held[0] + 4
    assert same(lat.pq_segments(), first)
    lat.close()


def _ensemble_params():
    return [U.Params(nx=16, ny=12, nz=8, m=2.0 / 3.0, beta=b, eta0=1.0, eta_ref=4.0, seed=40 + i)
            for i, b in enumerate((1.0, 0.0, -1.0))]


def test_ensemble_creation_fails_cleanly_at_every_allocation():
    base = live()
    e = U.Ensemble(_ensemble_params())
    n_alloc = live()[0] - base[0]
    e.close()
    assert live() == base and n_alloc > 3 * 10
    for k in range(1, n_alloc + 1):
        U.inject_alloc_failure(k)
        fails_with_oom(lambda: U.Ensemble(_ensemble_params()))
        assert live() == base, k


@pytest.mark.parametrize("mode", [U.ENS_PERSISTENT, U.ENS_PER_STEP])
def test_ensemble_run_and_autotune_fail_cleanly(mode):
    """A detecting run (its schedule and detection plan are allocated on
    first use) and the autotuner (a copy of every box's state), failed at
    each of their allocations: a failed plan leaves only the run's schedule
    cached, a failed autotune nothing, and a run afterwards gives the states,
    records and allocation count of a run that never failed."""
    steps, de = [12, 9, 5], 4
    ref = U.Ensemble(_ensemble_params())
    before = live()
    ref.run(steps, mode=mode, use_graph=True, detect_every=de)
    n_run = live()[0] - before[0]
    ref_states = [b.state().clone() for b in ref.boxes]
    ref_recs = [b.read_records()[0] for b in ref.boxes]
    ref_tuning = ref.tuning()
    ref.close()
    probe = U.Ensemble(_ensemble_params())
    before = live()
    probe.run(steps, mode=mode, use_graph=True)  # without detection: the schedule alone
    n_sched = live()[0] - before[0]
    probe.close()
    assert n_sched >= 4 and n_run > n_sched

    for k in range(1, n_run + 1):
        e = U.Ensemble(_ensemble_params())
        held = live()
        U.inject_alloc_failure(k)
        fails_with_oom(lambda: e.run(steps, mode=mode, use_graph=True, detect_every=de))
        assert live()[0] == held[0] + (n_sched if k > n_sched else 0), k
        if k < n_run:
            e.close()
    # the autotuner's state copies: fail the first and the last box's
    for k in (1, 3):
        U.inject_alloc_failure(k)
        fails_with_oom(lambda: e.autotune(probe_steps=2))
        assert live() == held, k
    assert all(b.n == 0 for b in e.boxes)
    assert e.tuning() == ref_tuning  # a failed autotune keeps the previous choice
    e.run(steps, mode=mode, use_graph=True, detect_every=de)
    assert live()[0] == held[0] + n_run
    for b, st, recs in zip(e.boxes, ref_states, ref_recs):
        assert torch.equal(b.state(), st)
        got = b.read_records()[0]
        assert len(got) == len(recs) and len(got) > 0
        for (gs, gd), (rs, rd) in zip(got, recs):
            assert same(gs, rs) and same(gd, rd)
    e.close()
