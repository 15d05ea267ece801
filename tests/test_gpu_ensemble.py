"""Batched ensembles of independent boxes of uneven size: every box advanced
in an ensemble run matches the FP64 oracle stepped from the same initial
conditions (FP64 within 1e-10, FP32 within the field max-rel 1e-5) and equals
the same box advanced alone by the single-lattice tiled kernel, bit for bit,
in all three scheduling modes and through CUDA graph replays; the persistent
kernel's bounded dependency wait turns an unreachable wait into a reported
timeout."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2208_01525_gb300 as U
from gpu_helpers import field_maxrel, host_state, to_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# unequal sector couplings (Sec. VI) for the odd boxes of the oracle test
UNEQUAL = dict(lambda_p=2.0, lambda_q=1.62, e_p=1.0, e_q=0.9, sigma_p=1.0, sigma_q=0.8, kappa=0.5)


def box_params(prec=U.FP32, unequal_odd=False):
    """Uneven boxes, eras, beta and seeds (ragged tiles in x, y and z);
    with unequal_odd, the odd boxes take unequal sector couplings."""
    shapes = [(16, 16, 16), (24, 20, 12), (32, 8, 40), (8, 12, 4), (40, 24, 33), (12, 12, 12)]
    out = []
    for b, (nx, ny, nz) in enumerate(shapes):
        m = (0.5, 2.0 / 3.0)[b % 2]
        beta = (1.0, 0.0, -1.0)[b % 3]
        kw = UNEQUAL if unequal_odd and b % 2 else {}
        out.append(U.Params(nx=nx, ny=ny, nz=nz, m=m, beta=beta, eta0=1.0,
                            eta_ref=3.0 if beta > 0 else 1.0, seed=1000 + b, precision=prec, **kw))
    return out


def alone(p, nsteps):
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(nsteps)
    return lat.state()


@pytest.mark.parametrize("mode", [U.ENS_PERSISTENT, U.ENS_PER_STEP, U.ENS_UNBATCHED])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_ensemble_matches_single_boxes(mode, prec):
    ps = box_params(prec)
    steps = [10, 7, 13, 0, 5, 9]
    ens = U.Ensemble(ps)
    ens.run(steps, mode=mode)
    assert ens.status() == 0
    for b, p in enumerate(ps):
        assert ens.boxes[b].n == steps[b]
        assert torch.equal(ens.boxes[b].state(), alone(p, steps[b])), b
    ens.close()


@pytest.mark.parametrize("mode,graph", [(U.ENS_PERSISTENT, False), (U.ENS_PERSISTENT, True),
                                        (U.ENS_PER_STEP, False), (U.ENS_PER_STEP, True),
                                        (U.ENS_UNBATCHED, False)])
@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-10), (U.FP32, 1e-5)])
def test_ensemble_boxes_match_oracle(mode, graph, prec, tol):
    """Every box of an ensemble run against the FP64 oracle stepped from the
    box's own initial conditions (per-box seed, era, beta, couplings, size):
    FP64 within 1e-10, FP32 within the field max-rel 1e-5.  Half the boxes
    carry unequal sector couplings; graph runs are captured once and
    replayed, so each box takes twice its step count."""
    ps = box_params(prec, unequal_odd=True)
    steps = [10, 7, 9, 0, 5, 8]
    reps = 2 if graph else 1
    ens = U.Ensemble(ps)
    for _ in range(reps):
        ens.run(steps, mode=mode, use_graph=graph)
    torch.cuda.synchronize()
    assert ens.status() == 0
    for b, p in enumerate(ps):
        assert ens.boxes[b].n == reps * steps[b]
        op = to_oracle(p)
        ref = O.init(op)
        O.step(op, ref, 0, reps * steps[b])
        err = field_maxrel(host_state(ens.boxes[b]), ref)
        assert err.max() <= tol, (b, err)
    ens.close()


@pytest.mark.parametrize("mode", [U.ENS_PERSISTENT, U.ENS_PER_STEP])
def test_ensemble_graph_replays(mode):
    ps = box_params()
    steps = [3, 4, 1, 2, 5, 3]
    ens = U.Ensemble(ps)
    for _ in range(3):  # capture once, replay twice; odd counts flip buffers
        ens.run(steps, mode=mode, use_graph=True)
    torch.cuda.synchronize()
    assert ens.status() == 0
    for b, p in enumerate(ps):
        assert ens.boxes[b].n == 3 * steps[b]
        assert torch.equal(ens.boxes[b].state(), alone(p, 3 * steps[b])), b


def test_ensemble_mixed_with_box_handles():
    """Steps taken through a box's own handle between ensemble runs are
    picked up by the next run; detection on a box equals detection alone."""
    ps = box_params()
    ens = U.Ensemble(ps)
    ens.run([4] * 6, mode=U.ENS_PERSISTENT)
    ens.boxes[2].step(3)
    ens.run([2] * 6, mode=U.ENS_PERSISTENT)
    want = [6, 6, 9, 6, 6, 6]
    for b, p in enumerate(ps):
        assert ens.boxes[b].n == want[b]
        ref = U.Lattice(p, kernel=U.KERNEL_TILED)
        ref.step(want[b])
        assert torch.equal(ens.boxes[b].state(), ref.state()), b
        if b == 4:
            s1 = ens.boxes[b].detect_strings()
            s2 = ref.detect_strings()
            assert s1["n_p"] == s2["n_p"] and s1["n_pq_cell"] == s2["n_pq_cell"]


def test_ensemble_bounded_wait_reports_timeout():
    """A work item waiting for a count nothing reaches: the run ends with
    U1U1_ERR_TIMEOUT after the wait limit, no hang; the ensemble then
    refuses further runs."""
    ps = box_params()
    ens = U.Ensemble(ps)
    ens.set_wait_limit(50_000_000)  # 50 ms
    ens.inject_unreachable_wait(True)
    ens.run([3] * 6, mode=U.ENS_PERSISTENT)
    assert ens.status() == -5
    with pytest.raises(U.U1U1Error):
        ens.run([1] * 6)
    ens.close()
    # a fresh ensemble on the same device works normally afterwards
    ens2 = U.Ensemble(ps)
    ens2.run([2] * 6)
    assert ens2.status() == 0


def test_ensemble_errors():
    ps = box_params()
    ens = U.Ensemble(ps, horizon=16)
    with pytest.raises(U.U1U1Error):
        ens.run([-1, 0, 0, 0, 0, 0])
    with pytest.raises(U.U1U1Error):
        ens.run([17, 0, 0, 0, 0, 0])
    with pytest.raises(U.U1U1Error):
        ens.run([1] * 6, mode=U.ENS_UNBATCHED, use_graph=True)
    ens.run([0] * 6)
    assert all(b.n == 0 for b in ens.boxes)
    with pytest.raises(U.U1U1Error):
        U.Ensemble([ps[0], U.Params(nx=8, ny=8, nz=8, precision=U.FP64)])
    # box handles belong to the ensemble: their parameters live in its device
    # tables, so a phase switch is refused, and destroying one does nothing
    with pytest.raises(U.U1U1Error) as ei:
        ens.boxes[0].set_params(ps[0], 0)
    assert ei.value.code == -8
    h = ctypes.c_void_p()
    U.check(U.lib().u1u1_ensemble_lattice(ens._h, 1, ctypes.byref(h)))
    U.lib().u1u1_destroy(h)
    ens.run([2] * 6)
    assert all(b.n == 2 for b in ens.boxes) and ens.status() == 0
    ens.close()


def test_ensemble_autotune_keeps_states():
    """The ensemble tuner's probe runs leave every box's state and step index
    as they were; runs after tuning still equal the boxes stepped alone."""
    ps = box_params()
    ens = U.Ensemble(ps)
    ens.run([2] * 6)
    before = [b.state().clone() for b in ens.boxes]
    choice = ens.autotune(probe_steps=3)
    assert choice["mode"] in (U.ENS_PERSISTENT, U.ENS_PER_STEP) and choice["item_lz"] in (16, 32, 64, 128)
    for b, s in zip(ens.boxes, before):
        assert b.n == 2 and torch.equal(b.state(), s)
    ens.run([4] * 6, mode=choice["mode"])
    for b, p in enumerate(ps):
        assert torch.equal(ens.boxes[b].state(), alone(p, 6)), b


@pytest.mark.parametrize("mode,graph,ptma", [(U.ENS_PERSISTENT, False, True), (U.ENS_PERSISTENT, True, True),
                                             (U.ENS_PERSISTENT, False, False), (U.ENS_PERSISTENT, True, False),
                                             (U.ENS_PER_STEP, True, True), (U.ENS_UNBATCHED, False, True)])
@pytest.mark.parametrize("item_lz", [16, 64])
def test_ensemble_tensor_copy_boxes(mode, graph, ptma, item_lz):
    """FP32 boxes wide and tall enough to have interior tiles, whose ring
    slots the ensemble kernels fill by tensor copies from per-box tensor maps
    in device memory (the persistent kernel with tensor copies or with
    cp.async, a tuning choice), next to a box without interior tiles: every
    box equals the same box stepped alone, bit for bit, in every mode, for
    two work-item z-chunks and over graph replays."""
    shapes = [(104, 32, 20), (136, 40, 12), (16, 16, 16)]
    ps = [U.Params(nx=nx, ny=ny, nz=nz, m=0.5, beta=1.0, eta0=1.0, eta_ref=3.0, seed=2000 + b, precision=U.FP32)
          for b, (nx, ny, nz) in enumerate(shapes)]
    steps = [6, 9, 4]
    reps = 2 if graph else 1
    ens = U.Ensemble(ps)
    ens.set_tuning(item_lz=item_lz, persistent_tma=ptma)
    assert ens.tuning() == {"item_lz": item_lz, "persistent_tma": ptma}
    with pytest.raises(U.U1U1Error):
        ens.set_tuning(item_lz=48)
    for _ in range(reps):
        ens.run(steps, mode=mode, use_graph=graph)
    torch.cuda.synchronize()
    assert ens.status() == 0
    for b, p in enumerate(ps):
        assert ens.boxes[b].n == reps * steps[b]
        assert torch.equal(ens.boxes[b].state(), alone(p, reps * steps[b])), b
    ens.close()


def _same_record(a: dict, b: dict) -> bool:
    for k, v in b.items():
        w = a[k]
        if isinstance(v, float) and v != v:
            if w == w:
                return False
        elif w != v:
            return False
    return True


@pytest.mark.parametrize("mode,graph", [(U.ENS_PERSISTENT, False), (U.ENS_PERSISTENT, True),
                                        (U.ENS_PER_STEP, False), (U.ENS_PER_STEP, True),
                                        (U.ENS_UNBATCHED, False)])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_ensemble_detection_records_equal_single_boxes(mode, graph, prec):
    """Detection every 4 steps inside ensemble runs: each box's records (read
    from its own handle's ring) equal, field for field, the records of the
    same box stepped alone with fused detection (same windings and counts,
    same diagnostic sums bit for bit), and the states stay equal.  Box 2
    takes one step through its own handle first, so the boxes detect at
    different run steps; graph runs are captured and replayed, and the
    second run starts each box at another phase of the cadence."""
    de = 4
    ps = box_params(prec, unequal_odd=True)
    steps = [10, 7, 9, 0, 5, 8]
    reps = 2 if graph else 1
    ens = U.Ensemble(ps)
    ens.boxes[2].step(1)
    for _ in range(reps):
        ens.run(steps, mode=mode, use_graph=graph, detect_every=de)
    torch.cuda.synchronize()
    assert ens.status() == 0
    for b, p in enumerate(ps):
        ref = U.Lattice(p, kernel=U.KERNEL_TILED)
        if b == 2:
            ref.step(1)
        for _ in range(reps):
            ref.step(steps[b], detect_every=de)
        want, lost_w = ref.read_records()
        got, lost_g = ens.boxes[b].read_records()
        assert lost_w == lost_g == 0
        assert [r[0]["n"] for r in got] == [r[0]["n"] for r in want], b
        for (gs, gd), (ws, wd) in zip(got, want):
            assert _same_record(gs, ws), (b, gs["n"], gs, ws)
            assert _same_record(gd, wd), (b, gd["n"], gd, wd)
        assert torch.equal(ens.boxes[b].state(), ref.state()), b
    ens.close()


def test_ensemble_detection_overlap_tolerance_and_oracle():
    """The overlap tolerance of each box's handle applies to its detection
    records (tolerance 0 on box 1, 1 elsewhere), and a detected record of
    an FP64 box equals the oracle's strings on the oracle's own state."""
    import oracle as O
    ps = box_params(U.FP64)
    ens = U.Ensemble(ps)
    U.check(U.lib().u1u1_set_overlap_tol(ens.boxes[1]._h, 0))
    ens.run([8] * 6, mode=U.ENS_PER_STEP, detect_every=8)
    for b, p in enumerate(ps):
        recs, lost = ens.boxes[b].read_records()
        assert lost == 0 and [r[0]["n"] for r in recs] == [0]
        assert recs[0][0]["overlap_tol"] == (0 if b == 1 else 1)
    ens.run([8] * 6, mode=U.ENS_PERSISTENT, detect_every=8)
    op = to_oracle(ps[4])
    ref = O.init(op)
    O.step(op, ref, 0, 8)
    ores = O.strings(op, ref, tol=1)
    recs, _ = ens.boxes[4].read_records()
    s = recs[0][0]
    assert s["n"] == 8
    if ores["n_flagged"] == 0:
        for k in ("n_p", "n_q", "n_pq_plaq", "n_pq_cell", "n_pq_cell_q", "max_abs_w"):
            assert s[k] == ores[k], (k, s[k], ores[k])
    od = O.diagnostics(op, ref, 8)
    d = recs[0][1]
    for k in ("kin_p", "grad_q", "el_p", "mag_q", "pot", "vint"):
        assert abs(d[k] - od[k]) <= 1e-10 * max(abs(od[k]), abs(od["energy"])), k
    ens.close()


@pytest.mark.parametrize("mode", [U.ENS_PERSISTENT, U.ENS_PER_STEP])
def test_ensemble_detection_two_stage_finalize(mode):
    """A 256^3 box has more block partials (4712) than one finalize CTA
    takes, so its batched detection runs the two-stage merge, next to a box
    that needs one stage: both boxes' records equal those of the boxes
    stepped alone, sums bit for bit."""
    ps = [U.Params.cube(256, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=31),
          U.Params(nx=40, ny=24, nz=20, m=2.0 / 3.0, beta=0.0, eta0=1.0, eta_ref=1.0, seed=32)]
    ens = U.Ensemble(ps)
    ens.run([8, 8], mode=mode, use_graph=True, detect_every=4)
    for b, p in enumerate(ps):
        ref = U.Lattice(p, kernel=U.KERNEL_TILED)
        ref.step(8, detect_every=4)
        want, _ = ref.read_records()
        got, _ = ens.boxes[b].read_records()
        assert [r[0]["n"] for r in got] == [r[0]["n"] for r in want] == [0, 4]
        for (gs, gd), (ws, wd) in zip(got, want):
            assert _same_record(gs, ws) and _same_record(gd, wd), b
        ref.close()
    ens.close()
