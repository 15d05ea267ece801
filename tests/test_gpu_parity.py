"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Bars: FP64 GPU within 1e-10 of the oracle (summation order only),
FP32 within the field max-rel 1e-5 after 20 steps, windings and counts bit
exact on an identical snapshot except plaquettes flagged within 1e-4 of the
branch cut (Sec. III.A), diagnostics within the stated relative tolerances.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import _abi
import synth
from gpu_helpers import field_maxrel, gather_sites, host_state, patches, to_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KERNELS = [U.KERNEL_SIMPLE, U.KERNEL_AUTO]

# Unequal sector couplings (the unequal-tension case of Sec. VI): every
# per-sector coefficient of the step and of the diagnostics differs between
# p and q, so a p/q mix-up in any kernel changes the result.
UNEQUAL = dict(lambda_p=2.0, lambda_q=1.62, e_p=1.0, e_q=0.9, sigma_p=1.0, sigma_q=0.8, kappa=0.5)
COUPLINGS = {"equal": {}, "unequal": UNEQUAL}


def radiation(n, nsteps, **kw):
    """The 64^3-style configuration: dx 0.5, deta 0.1, radiation, beta = 1,
    lambda = 2, e = 1, sigma = 1, kappa = 0.9, eta0 = 1, a = 1 at the end."""
    d = dict(m=0.5, beta=1.0, eta0=1.0, eta_ref=1.0 + 0.1 * nsteps)
    d.update(kw)
    if isinstance(n, int):
        return U.Params.cube(n, **d)
    return U.Params(nx=n[0], ny=n[1], nz=n[2], **d)


@pytest.mark.parametrize("prec", [U.FP64, U.FP32])
def test_initial_conditions_match_oracle(prec):
    p = U.Params(nx=20, ny=12, nz=8, seed=77, sigma_p=1.0, sigma_q=0.8, precision=prec)
    lat = U.Lattice(p)
    st = host_state(lat)
    ref = O.init(to_oracle(p))
    tol = 4e-16 if prec == U.FP64 else 1.2e-7
    assert np.abs(st - ref).max() <= tol
    # the other ping-pong buffer is zeroed too
    other = torch.stack(lat.pos[1]).double().abs().max().item()
    assert other == 0.0


@pytest.mark.parametrize("couplings", sorted(COUPLINGS))
@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_matches_oracle_full_run(kernel, couplings):
    """64^3, 160 steps to eta = 17 (radiation, beta = 1), FP64 vs oracle,
    with equal couplings and with every per-sector coupling different."""
    p = radiation(64, 160, precision=U.FP64, seed=1, **COUPLINGS[couplings])
    lat = U.Lattice(p, kernel=kernel)
    lat.step(160)
    ref = O.init(to_oracle(p))
    O.step(to_oracle(p), ref, 0, 160)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() < 1e-10, err


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", [(36, 20, 12), (4, 4, 4), (8, 12, 36)])
@pytest.mark.parametrize("cfg", [dict(m=2.0 / 3.0, beta=0.0), dict(m=0.5, beta=-1.0, eta_ref=1.0),
                                 dict(m=0.0, beta=1.0)])
def test_fp64_ragged_boxes_all_eras(kernel, shape, cfg):
    p = radiation(shape, 12, precision=U.FP64, seed=5, **cfg)
    lat = U.Lattice(p, kernel=kernel)
    st0 = synth.random_state(p.shape, seed=9, a_amp=1.0, mom_amp=0.5)
    lat.set_state(st0, n=3)
    lat.step(12)
    ref = st0.copy()
    O.step(to_oracle(p), ref, 3, 12)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() < 1e-11, err


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-11), (U.FP32, 1e-5)])
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("cfg", [dict(m=2.0 / 3.0, beta=0.0), dict(m=0.5, beta=-1.0, eta_ref=1.0),
                                 dict(m=0.0, beta=1.0)])
def test_unequal_couplings_ragged_boxes(prec, tol, kernel, cfg):
    """Unequal couplings in both sectors on a ragged box from a rough state
    (momenta and links of every sign), in every era: FP64 within 1e-11 and
    FP32 within the field max-rel 1e-5 of the oracle after 12 steps."""
    p = radiation((36, 20, 12), 12, precision=prec, seed=5, **cfg, **UNEQUAL)
    lat = U.Lattice(p, kernel=kernel)
    st0 = synth.random_state(p.shape, seed=19, a_amp=1.0, mom_amp=0.5)
    lat.set_state(st0, n=3)
    lat.step(12)
    ref = st0.copy()
    O.step(to_oracle(p), ref, 3, 12)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() <= tol, err


@pytest.mark.parametrize("couplings", sorted(COUPLINGS))
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("cfg", [dict(m=0.5, beta=1.0), dict(m=2.0 / 3.0, beta=0.0),
                                 dict(m=0.5, beta=-1.0, eta_ref=1.0)])
def test_fp32_matches_oracle_20_steps(kernel, cfg, couplings):
    """FP32 bulk vs FP64 oracle: field max-rel <= 1e-5 after 20 steps."""
    p = radiation(64, 640, precision=U.FP32, seed=2, **cfg, **COUPLINGS[couplings])
    lat = U.Lattice(p, kernel=kernel)
    lat.step(20)
    ref = O.init(to_oracle(p))
    O.step(to_oracle(p), ref, 0, 20)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-11), (U.FP32, 1e-5)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_cooling_matches_oracle(prec, tol, kernel):
    """The diffusive cooling flow (Eqs. 27-30): 30 forward-Euler steps from a
    rough state, with unequal couplings and kappa != 0 (which the flow
    leaves out), against the oracle's flow; the momenta are zero after."""
    p = U.Params(nx=36, ny=20, nz=12, seed=5, precision=prec, **UNEQUAL)
    lat = U.Lattice(p, kernel=kernel)
    st0 = synth.random_state(p.shape, seed=29, a_amp=1.0, mom_amp=0.5)
    lat.set_state(st0, n=0)
    dt = 0.1 * p.dx ** 2
    lat.cool(dt, 30)
    ref = st0.copy()
    O.cool(to_oracle(p), ref, dt, 30)
    got = host_state(lat)
    err = field_maxrel(got[:10], ref[:10])
    assert err.max() <= tol, err
    assert not got[10:].any()


def _windings_compare(p, st_gpu_lat):
    res = st_gpu_lat.detect_strings(tol=1, cells=True, windings=True)
    snap = host_state(st_gpu_lat)
    op = to_oracle(p)
    W, F = O.windings(op, snap)
    Wg = res["windings"].cpu().numpy().astype(np.int64)
    flag = F != 0
    ok = ~flag
    assert np.array_equal(Wg[ok], W[ok].astype(np.int64))
    ores = O.strings(op, snap, tol=1)
    nflag = int(flag.sum())
    assert abs(res["n_p"] - ores["n_p"]) <= nflag and abs(res["n_q"] - ores["n_q"]) <= nflag
    if nflag == 0:
        for k in ("n_p", "n_q", "nonzero_p", "nonzero_q", "n_pq_plaq", "n_pq_cell", "n_pq_cell_q",
                  "max_abs_w", "n_w2_p", "n_w2_q", "n_cells_ge4_p", "n_cells_ge4_q"):
            assert res[k] == ores[k], (k, res[k], ores[k])
        assert np.array_equal(res["cells"].cpu().numpy(), ores["cells"])
        for k in ("L_p", "L_q", "L_pq", "xi_p", "xi_q", "xi_pq", "xi_w", "f_total", "f_p"):
            assert res[k] == ores[k] or (math.isnan(res[k]) and math.isnan(ores[k])), k
    return res, ores, nflag


def test_fp32_tensor_copy_tiles_match_oracle():
    """A 136 x 40 x 24 box mixes tiles whose position ring is filled by
    tensor copies (halo inside the lattice) with tiles at the edges, whose
    halo wraps around and which use cp.async: 20 FP32 steps with a fused
    detection step stay within the FP32 tolerance of the FP64 oracle, the
    windings match it on unflagged plaquettes and the diagnostics agree."""
    p = U.Params(nx=136, ny=40, nz=24, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=12, precision=U.FP32)
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(20, detect_every=10)
    recs, lost = lat.read_records()
    assert lost == 0 and len(recs) == 2
    ref = O.init(to_oracle(p))
    O.step(to_oracle(p), ref, 0, 20)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() <= 1e-5, err
    res, ores, nflag = _windings_compare(p, lat)
    d = lat.diagnostics()
    od = O.diagnostics(to_oracle(p), host_state(lat), lat.n)
    assert abs(d["energy"] - od["energy"]) <= 1e-4 * abs(od["energy"])


def test_copy_wait_timeout_is_reported():
    """The tiled kernels' waits for their tensor copies are bounded: with the
    test hook making every slot expect more bytes than its copies deliver,
    the waits run out after 50 ms, the step finishes, and the next
    synchronising call of the handle that launched it reports TIMEOUT
    (once).  Another handle, synchronised in between, reports nothing: each
    handle has its own status word.  With the hook off, the same box steps
    normally again and matches the oracle."""
    p = U.Params(nx=136, ny=40, nz=24, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=12, precision=U.FP32)
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    other = U.Lattice(p, kernel=U.KERNEL_TILED)
    other.step(2)
    U.check(U.lib().u1u1_inject_copy_timeout(1, 50_000_000))
    try:
        lat.step(2)
        torch.cuda.synchronize()
        # the untouched handle synchronises first and sees no timeout
        assert other.read_records() == ([], 0)
        other.detect_strings()
        other.diagnostics()
        with pytest.raises(U.U1U1Error) as ei:
            lat.read_records()
        assert ei.value.code == -5 and "tensor copy" in str(ei.value)  # TIMEOUT
    finally:
        U.check(U.lib().u1u1_inject_copy_timeout(0, 2_000_000_000))
    lat.read_records()  # reported once
    other.close()
    lat.close()
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(6)
    assert lat.read_records()[1] == 0
    ref = O.init(to_oracle(p))
    O.step(to_oracle(p), ref, 0, 6)
    err = field_maxrel(host_state(lat), ref)
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("couplings", sorted(COUPLINGS))
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("kernel", KERNELS)
def test_windings_bit_exact_on_snapshot(prec, kernel, couplings):
    p = radiation(64, 640, precision=prec, seed=3, **COUPLINGS[couplings])
    lat = U.Lattice(p, kernel=kernel)
    lat.step(30)
    res, ores, nflag = _windings_compare(p, lat)
    assert res["n_p"] > 100  # the early network is dense
    assert res["n_flagged"] == ores["n_flagged"] or prec == U.FP32


@pytest.mark.parametrize("kernel", KERNELS)
def test_windings_rough_random_state(kernel):
    """Windings of every sign and large link angles (rough synthetic state)."""
    p = U.Params(nx=24, ny=16, nz=12, m=0.0, precision=U.FP64)
    lat = U.Lattice(p, kernel=kernel)
    lat.set_state(synth.random_state(p.shape, seed=4, a_amp=4.0))
    res, ores, nflag = _windings_compare(p, lat)
    assert res["max_abs_w"] >= 1


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", [(9, 22, 40), (13, 7, 32)])
def test_windings_fp32_rough_ragged_with_zero_field(kernel, shape):
    """FP32 windings on a rough state, on boxes that leave ragged windows
    in x and y, with phi = 0 planted at one site of each sector: every
    unflagged plaquette matches the oracle, and the plaquettes around the
    zero sites (12 per sector) are flagged."""
    nz, ny, nx = shape
    p = U.Params(nx=nx, ny=ny, nz=nz, m=0.0, precision=U.FP32)
    st = synth.random_state(p.shape, seed=11, a_amp=4.0)
    st[0][2, 3, 5] = st[1][2, 3, 5] = 0.0
    st[2][4, 1, 7] = st[3][4, 1, 7] = 0.0
    lat = U.Lattice(p, kernel=kernel)
    lat.set_state(st)
    res, ores, nflag = _windings_compare(p, lat)
    assert ores["n_flagged"] >= 24 and res["n_flagged"] >= 24
    assert res["max_abs_w"] >= 1


def test_cell_arrays_any_alignment():
    """Cell arrays written to 16-byte aligned buffers (the vectorised cell
    pass) and to buffers offset by one byte (the bytewise pass) agree with
    each other and with the oracle's cells, and so do the counts."""
    import ctypes
    p = radiation(64, 640, precision=U.FP32, seed=8)
    lat = U.Lattice(p)
    lat.step(24)
    ref = lat.detect_strings(tol=1, cells=True)
    V = p.nsites
    raw = torch.zeros(2 * V + 32, dtype=torch.uint8, device="cuda")
    cp, cq = raw.data_ptr() + 1, raw.data_ptr() + V + 17
    out = _abi.CStrings()
    U.check(U.lib().u1u1_detect_strings(lat._h, 1, ctypes.c_void_p(cp), ctypes.c_void_p(cq), None,
                                        ctypes.byref(out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    odd = _abi.struct_to_dict(out)
    got = torch.stack([raw[1:1 + V], raw[V + 17:V + 17 + V]]).view(2, *p.shape)
    assert torch.equal(got.cpu(), ref["cells"].cpu())
    for k in ("n_p", "n_q", "n_pq_cell", "n_pq_cell_q", "n_cells_ge4_p", "n_cells_ge4_q", "n_flagged"):
        assert odd[k] == ref[k], k
    snap = host_state(lat)
    ores = O.strings(to_oracle(p), snap, tol=1)
    W, F = O.windings(to_oracle(p), snap)
    if int((F != 0).sum()) == 0:
        assert np.array_equal(ref["cells"].cpu().numpy(), ores["cells"])
        assert ref["n_pq_cell"] == ores["n_pq_cell"]


@pytest.mark.parametrize("tol", [1, 0])
def test_overlap_rows_of_1024(tol):
    """Rows of 1024 cells take the warp-per-row overlap pass (x neighbours
    by shuffle, periodic across the row's ends).  On a 1024 x 10 x 6 box of a
    rough state its counts equal a brute-force overlap of the same cell
    arrays (27-cell neighbourhood for tol 1, the cell itself for tol 0), in
    both anchorings; the windings match the oracle on unflagged plaquettes
    and the overlap count is within the reach of the flagged ones."""
    p = U.Params(nx=1024, ny=10, nz=6, m=0.0, precision=U.FP64)
    lat = U.Lattice(p)
    lat.set_state(synth.random_state(p.shape, seed=21, a_amp=1.5))
    res, ores, nflag = _windings_compare(p, lat) if tol == 1 else (None, None, None)
    res = lat.detect_strings(tol=tol, cells=True)
    cells = res["cells"].cpu().numpy()
    P, Q = cells[0] > 0, cells[1] > 0

    def dilate(m):
        out = np.zeros_like(m)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out |= np.roll(m, (dz, dy, dx), axis=(0, 1, 2))
        return out

    dq, dp = (dilate(Q), dilate(P)) if tol == 1 else (Q, P)
    assert res["n_pq_cell"] == int((P & dq).sum())
    assert res["n_pq_cell_q"] == int((Q & dp).sum())
    assert res["n_pq_cell"] > 1000
    if tol == 1:
        assert abs(res["n_pq_cell"] - ores["n_pq_cell"]) <= 2 * 27 * nflag


def test_higher_winding_census():
    """Crossing strings: the cells shared by two strings read 4 and are
    counted as the oracle counts them."""
    shape = (8, 12, 16)
    nz, ny, nx = shape
    for prec in (U.FP32, U.FP64):
        p = U.Params(nx=nx, ny=ny, nz=nz, m=0.0, precision=prec)
        st = np.zeros((20,) + shape)
        f = synth.crossing_vortices(shape)
        st[0], st[1] = f.real, f.imag
        st[2] = 1.0
        lat = U.Lattice(p)
        lat.set_state(st)
        r = lat.detect_strings(tol=1)
        assert r["n_cells_ge4_p"] == 8 and r["n_w2_p"] == 0 and r["max_abs_w"] == 1
        assert r["n_cells_ge4_q"] == 0 and r["n_p"] == 4 * nz + 4 * nx


def test_planted_vortices_detected():
    """Four planted strings: |W| = 1 once per z-plane at the expected
    plaquettes, cell value 2 (Sec. III.B), overlap counts by displacement."""
    shape = (6, 12, 16)
    nz, ny, nx = shape
    for shift, want0, want1 in ((0, 4 * nz, 4 * nz), (1, 0, 4 * nz), (2, 0, 0)):
        p = U.Params(nx=nx, ny=ny, nz=nz, m=0.0, precision=U.FP32)
        st = np.zeros((20,) + shape)
        vm = synth.vortex_map(shape)
        st[0], st[1] = vm.real, vm.imag
        vq = np.roll(vm, shift, axis=2)
        st[2], st[3] = vq.real, vq.imag
        lat = U.Lattice(p)
        lat.set_state(st)
        r0 = lat.detect_strings(tol=0, cells=True)
        r1 = lat.detect_strings(tol=1)
        assert r0["n_p"] == 4 * nz and r0["n_q"] == 4 * nz and r0["n_flagged"] == 0
        assert r0["n_pq_cell"] == want0 and r1["n_pq_cell"] == want1
        assert int(r0["cells"][0].sum().item()) == 2 * 4 * nz


ERAS = {"radiation_beta1": {}, "matter_beta0": dict(m=2.0 / 3.0, beta=0.0),
        "radiation_growth": dict(m=0.5, beta=-1.0, eta_ref=1.0)}


@pytest.mark.parametrize("era", sorted(ERAS))
@pytest.mark.parametrize("couplings", sorted(COUPLINGS))
@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-10), (U.FP32, 2e-5)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_diagnostics_match_oracle(prec, tol, kernel, couplings, era):
    """Every diagnostic sum and estimator of Sec. III.A against the oracle on
    the same state, in the radiation era with beta = 1, the matter era with
    beta = 0 and the core-growth regime (beta = -1): the coupling factor
    a^{2 beta}, the gauge-energy factor 1/(2 e^2 c) and the Gauss charge
    factor of the previous step all enter the sums."""
    p = radiation((32, 24, 16), 100, precision=prec, seed=6, **COUPLINGS[couplings], **ERAS[era])
    lat = U.Lattice(p, kernel=kernel)
    lat.step(25)
    d = lat.diagnostics()
    snap = host_state(lat)
    od = O.diagnostics(to_oracle(p), snap, 25)
    scale = abs(od["energy"])
    for k in ("kin_p", "kin_q", "grad_p", "grad_q", "el_p", "el_q", "mag_p", "mag_q", "pot", "vint",
              "pot_p", "pot_q", "lag", "energy", "rl_num", "rl_den", "rpq_num", "rpq_den"):
        ref = od[k]
        s = scale if k in ("lag", "pot", "vint") else max(abs(ref), 1e-300)
        if k.startswith("r"):
            s = max(abs(od["rl_den"]), abs(od["rl_num"]), abs(ref))
        assert abs(d[k] - ref) <= tol * s, (k, d[k], ref)
    for k in ("lag_p", "lag_q"):
        assert abs(d[k] - od[k]) <= tol * p.dx ** 3 * scale, (k, d[k], od[k])
    for k in ("xi_l", "xi_l_p", "xi_l_q", "v2_l", "v2_pq"):
        if math.isnan(od[k]):  # xi_L is undefined while the Lagrangian sum is positive
            assert math.isnan(d[k]), k
        else:
            assert abs(d[k] - od[k]) <= 50 * tol * abs(od[k]), (k, d[k], od[k])
    assert d["has_gauss"] == 1
    for sec in "pq":
        gscale = od["charge_sum_" + sec] / p.nsites + 1e-300
        assert d["gauss_max_" + sec] <= max(od["gauss_max_" + sec], 0) + tol * 10 * max(1.0, gscale)
    for k in ("phi_min_p", "phi_max_p", "phi_min_q", "phi_max_q"):
        assert abs(d[k] - od[k]) <= tol * 10, k
    assert d["nan_count"] == 0


@pytest.mark.parametrize("prec", [U.FP64, U.FP32])
def test_gauss_law_preserved(prec):
    """Sec. IV: Gauss's law holds to round-off from the random-phase start."""
    p = radiation(48, 200, precision=prec, seed=8)
    lat = U.Lattice(p)
    for _ in range(4):
        lat.step(10)
        d = lat.diagnostics()
        for sec in "pq":
            bound = 1e-12 if prec == U.FP64 else 2e-5
            assert d["gauss_max_" + sec] < bound, (lat.n, sec, d["gauss_max_" + sec])


@pytest.mark.parametrize("era", sorted(ERAS))
@pytest.mark.parametrize("couplings", sorted(COUPLINGS))
@pytest.mark.parametrize("kernel", KERNELS)
def test_fused_detection_equals_standalone(kernel, couplings, era):
    """A step fused with detection records exactly what the standalone
    detection and diagnostics report on the same input state, in each era."""
    p = radiation(40, 400, precision=U.FP32, seed=10, **COUPLINGS[couplings], **ERAS[era])
    a = U.Lattice(p, kernel=kernel)
    b = U.Lattice(p, kernel=kernel)
    a.step(16)
    b.step(16)
    s_ref = a.detect_strings(tol=1)
    d_ref = a.diagnostics()
    b.step(32, detect_every=16)
    recs, lost = b.read_records()
    assert lost == 0 and [r[0]["n"] for r in recs] == [16, 32]
    s, d = recs[0]
    for k, v in s_ref.items():
        assert s[k] == v or (isinstance(v, float) and math.isnan(v) and math.isnan(s[k])), k
    for k in ("kin_p", "grad_q", "el_p", "mag_q", "pot", "vint", "lag", "energy", "rl_num", "rpq_den",
              "xi_l", "v2_l", "v2_pq", "phi_min_p", "phi_max_q"):
        assert d[k] == d_ref[k], (k, d[k], d_ref[k])
    assert d["has_gauss"] == 0
    # the run continued: both handles are at the same step and agree
    a.step(32)
    assert torch.equal(a.state(), b.state())


def test_fp32_vs_fp64_gpu_256():
    """The 256^3 configuration: FP32 step vs FP64 GPU step over the first 20
    steps (the oracle is compared at sampled sites in the full-size test)."""
    p32 = radiation(256, 640, precision=U.FP32, seed=1)
    p64 = radiation(256, 640, precision=U.FP64, seed=1)
    a = U.Lattice(p32)
    a.step(20)
    sa = a.state().double().cpu().numpy()
    del a
    b = U.Lattice(p64)
    b.step(20)
    sb = host_state(b)
    err = field_maxrel(sa, sb)
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("n,prec", [(256, U.FP32), (1024, U.FP32), (256, U.FP64), (1024, U.FP64)])
def test_full_size_sampled_sites(n, prec):
    """Full-size lattice in the benchmark's launch configuration: after 20
    steps, one more step at 192 random sites equals the oracle's step of a
    5^3 periodic patch around each site (the centre update depends only on
    its radius-1 neighbourhood), and the windings there match; any-size
    properties (even cells, sum of cells = 2 sum |W|) hold everywhere.  The
    largest case is the FP64 1024^3 box (258 GB of fields)."""
    if n == 1024:
        import gc
        gc.collect()  # handles and tensors of earlier tests
        torch.cuda.empty_cache()
        free = torch.cuda.mem_get_info()[0]
        need = 150e9 if prec == U.FP32 else 285e9
        if free < need:
            pytest.skip(f"needs ~{need / 1e9:.0f} GB of free device memory")
    p = radiation(n, 2560 if n == 1024 else 640, precision=prec, seed=4)
    lat = U.Lattice(p)
    if n == 1024 and prec == U.FP64:
        lat.set_kernel(U.KERNEL_TILED)  # the benchmark's FP64 leg: tiled kernel, default chunking (no room to tune)
    else:
        lat.autotune()  # the benchmark's launch configuration: kernel and z-chunking by timing
    lat.step(20)
    sites = synth.site_sample(p.shape, 192, seed=n)
    pt = patches(lat.fields(), p.shape, sites, radius=2)
    lat.step(1)
    got = gather_sites(lat.fields(), p.shape, sites)
    op = to_oracle(p)
    op.nx = op.ny = op.nz = 5
    want = np.zeros_like(got)
    for k in range(len(sites)):
        st = np.ascontiguousarray(pt[k])
        O.step(op, st, 20, 1)
        want[k] = st[:, 2, 2, 2]
    scale = np.abs(want).max(axis=0)
    rel = (np.abs(got - want).max(axis=0) / np.where(scale > 0, scale, 1.0))
    assert rel.max() <= (1e-6 if prec == U.FP32 else 1e-12), rel
    # windings at the sampled sites on the current snapshot
    res = lat.detect_strings(tol=1, cells=True, windings=True)
    pt = patches(lat.fields(), p.shape, sites, radius=2)
    Wg = res["windings"]
    s = torch.as_tensor(sites, device=Wg.device)
    wg = Wg[:, :, s[:, 0], s[:, 1], s[:, 2]].cpu().numpy()
    for k in range(len(sites)):
        W, F = O.windings(op, np.ascontiguousarray(pt[k]))
        ok = F[:, :, 2, 2, 2] == 0
        assert np.array_equal(wg[:, :, k][ok], W[:, :, 2, 2, 2][ok].astype(wg.dtype))
    cells = res["cells"]
    assert not (cells % 2).any().item()

    def total(t):  # int64 sum in z-slabs: a whole-lattice int64 temporary would not fit next to FP64 1024^3
        return sum(int(t[..., z:z + 64, :, :].abs().sum(dtype=torch.int64).item()) for z in range(0, n, 64))

    for sec in range(2):
        assert total(cells[sec]) == 2 * total(Wg[sec])
    assert res["n_p"] == total(Wg[0])


def test_beyond_two_to_the_31_sites():
    """An FP32 box past 2^31 sites, 1024 x 1024 x 2056 (2.16e9 sites, 259 GB
    of fields): half of 192 sampled sites lie in the top eight planes, where
    site offsets exceed 2^31, and after 20 steps one more step there equals
    the oracle's step of each site's 5^3 patch; the detection of the whole
    box keeps its any-size properties (cells even, their sum twice the
    winding total, the top planes included)."""
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < 272e9:
        pytest.skip("needs ~270 GB of free device memory")
    n, nz = 1024, 2056
    p = radiation((n, n, nz), 2560, precision=U.FP32, seed=6)
    assert p.nsites > 2 ** 31
    lat = U.Lattice(p)
    lat.set_kernel(U.KERNEL_TILED)  # default chunking: no room for the tuner's copy of the momenta
    lat.step(20)
    top = synth.site_sample((8, n, n), 96, seed=1) + np.array([nz - 8, 0, 0])
    sites = np.concatenate([top, synth.site_sample(p.shape, 96, seed=2)])
    assert ((sites[:, 0] * n + sites[:, 1]) * n + sites[:, 2] >= 2 ** 31).sum() == 96
    pt = patches(lat.fields(), p.shape, sites, radius=2)
    lat.step(1)
    got = gather_sites(lat.fields(), p.shape, sites)
    op = to_oracle(p)
    op.nx = op.ny = op.nz = 5
    want = np.zeros_like(got)
    for k in range(len(sites)):
        st = np.ascontiguousarray(pt[k])
        O.step(op, st, 20, 1)
        want[k] = st[:, 2, 2, 2]
    scale = np.abs(want).max(axis=0)
    rel = np.abs(got - want).max(axis=0) / np.where(scale > 0, scale, 1.0)
    assert rel.max() <= 1e-6, rel
    res = lat.detect_strings(tol=1, cells=True)
    cells = res["cells"]
    slabs = [(z, min(z + 64, nz)) for z in range(0, nz, 64)]  # no whole-box temporaries
    assert not any((cells[:, a:b] & 1).any().item() for a, b in slabs)
    for sec, key in ((0, "n_p"), (1, "n_q")):
        tot = sum(int(cells[sec, a:b].sum(dtype=torch.int64).item()) for a, b in slabs)
        assert tot == 2 * res[key] and res[key] > 0, (sec, tot, res[key])
    assert cells[:, nz - 8:].any().item()


def test_band_order_covers_every_tile():
    """The tiled plain step hands tiles out in bands of tile rows, each band
    through all its z-chunks.  On 1024 x 136 x 8 (17 rows of 32 tiles: one
    band of 14 rows and a shorter last band at three CTAs per SM, each
    column cut into z-chunks of 32, 32 and 8 planes) two steps of the tiled
    kernel agree with the one-thread-per-site kernel, which has no bands, to
    rounding: a tile or chunk left out would keep its input values."""
    p = U.Params(nx=1024, ny=136, nz=72, m=0.5, beta=1.0, eta0=1.0, eta_ref=2.0, seed=15, precision=U.FP32)
    st = synth.random_state(p.shape, seed=16, a_amp=1.0, mom_amp=0.5)
    out = []
    for kernel in (U.KERNEL_TILED, U.KERNEL_SIMPLE):
        lat = U.Lattice(p, kernel=kernel, init=False)
        lat.set_state(st, n=0)
        if kernel == U.KERNEL_TILED:
            lat.set_tile_waves(256)
        lat.step(2)
        out.append(host_state(lat))
        lat.close()
    err = field_maxrel(out[0], out[1])
    assert err.max() < 1e-5, err


def test_wave_targets_agree_bit_exact():
    """Every z-chunking the autotuner may choose gives the same fields bit for
    bit, since each site's update does not depend on where its z-chunk
    starts.  On a 1024 x 1024 x 300 box the wave targets 8 .. 256 cut z into
    chunks of 300, 150, 75, 38 (ragged last chunk of 34) and 32 (ragged last
    chunk of 12) planes, so chunk prologues and their carries fall on
    different planes; 1024-wide rows put most tiles on tensor copies."""
    import gc
    gc.collect()  # earlier tests' objects, and the blocks the allocator keeps for them
    torch.cuda.empty_cache()
    free = torch.cuda.mem_get_info()[0]
    if free < 100e9:
        pytest.skip("needs ~90 GB of free device memory")
    p = radiation((1024, 1024, 300), 320, precision=U.FP32, seed=21)
    ref = None
    for w in (8, 16, 32, 64, 128, 256):
        lat = U.Lattice(p, kernel=U.KERNEL_TILED)
        lat.set_tile_waves(w)
        lat.step(4)
        got = [t.clone() for t in lat.fields()]
        lat.close()
        del lat
        if ref is None:
            ref = got
            continue
        for f, (a, b) in enumerate(zip(got, ref)):
            assert torch.equal(a, b), (w, f)
        del got
    del ref
    torch.cuda.empty_cache()


def test_checkpoint_resume_bit_exact(tmp_path):
    p = radiation(24, 50, precision=U.FP32, seed=12)
    a = U.Lattice(p)
    a.step(7)
    path = str(tmp_path / "ckpt.u1u1")
    a.save(path)
    a.step(9)
    b = U.Lattice(p, init=False)
    b.load(path)
    assert b.n == 7
    b.step(9)
    assert torch.equal(a.state(), b.state())


def test_checkpoint_refusals_leave_the_state(tmp_path):
    """A checkpoint saved under other couplings, a truncated one and an
    overlong one are refused before anything is written: the handle keeps
    its state and step index, and the right file still loads afterwards."""
    import dataclasses
    p = radiation(16, 50, precision=U.FP32, seed=13)
    a = U.Lattice(p)
    a.step(5)
    path = tmp_path / "a.u1u1"
    a.save(str(path))
    data = path.read_bytes()
    (tmp_path / "short.u1u1").write_bytes(data[:-1])
    (tmp_path / "long.u1u1").write_bytes(data + b"\0")
    other = U.Lattice(dataclasses.replace(p, kappa=0.8))
    b = U.Lattice(p)
    for lat in (other, b):
        lat.step(3)
    cases = [(other, path, -1, "kappa"), (b, tmp_path / "short.u1u1", -9, "expected"),
             (b, tmp_path / "long.u1u1", -9, "expected")]
    for lat, f, code, word in cases:
        before = lat.state().clone()
        with pytest.raises(U.U1U1Error) as ei:
            lat.load(str(f))
        assert ei.value.code == code and word in str(ei.value)
        assert lat.n == 3 and torch.equal(lat.state(), before)
    b.load(str(path))
    assert b.n == 5 and torch.equal(b.state(), a.state())


@pytest.mark.parametrize("shape,prec", [((16, 8, 8), U.FP64), ((16, 8, 8), U.FP32), ((12, 6, 5), U.FP32)])
def test_upload_download_roundtrip(shape, prec):
    """State transfers: pinned, 16-byte aligned host tensors are copied by
    the SM kernel through their mapped address (a field is a whole number of
    16-byte words since nx is a multiple of 4); pageable tensors and pinned
    views at an 8-byte offset by the copy engines.  Every mix of the two
    lands bit for bit on the device and comes back unchanged."""
    p = U.Params(nx=shape[0], ny=shape[1], nz=shape[2], precision=prec)
    dt = torch.float64 if prec == U.FP64 else torch.float32
    V, nb = p.nsites, p.nsites * (8 if prec == U.FP64 else 4)
    lat = U.Lattice(p)
    st = torch.from_numpy(synth.random_state(p.shape, seed=1)).reshape(20, -1).to(dt)
    pinned = [st[f].contiguous().pin_memory() for f in range(20)]
    assert all(U.host_span_mapped(t.data_ptr(), nb) for t in pinned)
    pageable = [st[f].clone() for f in range(20)]
    assert not any(U.host_span_mapped(t.data_ptr(), nb) for t in pageable)
    block = torch.empty(V + 2, dtype=dt).pin_memory()
    assert not U.host_span_mapped(block.data_ptr(), 8)  # not a whole 16-byte word
    assert not U.host_span_mapped(block.data_ptr(), 1 << 40)  # beyond the allocation
    odd = block.view(torch.uint8)[8:8 + nb].view(dt)  # pinned, 8-byte offset
    odd.copy_(st[3])
    assert not U.host_span_mapped(odd.data_ptr(), nb)

    def expect_device():
        torch.cuda.synchronize()
        got = lat.fields()
        for f in range(20):
            assert torch.equal(got[f].cpu(), st[f]), f

    lat.upload(pinned)
    expect_device()
    mixed = [pinned[f] if f % 2 == 0 else pageable[f] for f in range(20)]
    mixed[3] = odd
    lat.upload(mixed)
    expect_device()
    outs = {
        "pinned": [torch.empty(V, dtype=dt).pin_memory() for _ in range(20)],
        "pageable": [torch.empty(V, dtype=dt) for _ in range(20)],
    }
    outs["mixed"] = [outs["pinned"][f] if f % 2 else outs["pageable"][f] for f in range(20)]
    for name, out in outs.items():
        for t in out:
            t.fill_(float("nan"))
        lat.download(out)
        torch.cuda.synchronize()
        assert all(torch.equal(out[f], st[f]) for f in range(20)), name


def test_upload_with_a_null_host_array_changes_nothing():
    """A NULL among the 20 host arrays is refused before any copy is
    enqueued: no field of the state changes."""
    import ctypes
    p = U.Params(nx=16, ny=8, nz=8, seed=3)
    lat = U.Lattice(p)
    before = lat.state().clone()
    host = [torch.full((p.nsites,), 7.0).pin_memory() for _ in range(20)]
    arr = (ctypes.c_void_p * 20)(*[t.data_ptr() for t in host])
    arr[7] = None
    assert U.lib().u1u1_upload_state(lat._h, arr, None) == -1
    torch.cuda.synchronize()
    assert torch.equal(lat.state(), before)


def test_vacuum_special_values():
    p = U.Params(nx=8, ny=8, nz=8, precision=U.FP64)
    lat = U.Lattice(p)
    st = np.zeros((20,) + p.shape)
    st[0] = 1.0
    st[2] = 1.0
    lat.set_state(st)
    r = lat.detect_strings()
    assert r["n_p"] == 0 and math.isinf(r["xi_w"]) and math.isnan(r["f_total"])
    lat.step(3)
    assert torch.equal(lat.state().cpu(), torch.from_numpy(st))


def test_set_state_keeps_the_handle():
    """set_state writes the current position buffer (here buffer 1, after an
    odd number of steps) and the momenta, sets the step index and keeps the
    handle's kernel choice; stepping on equals a fresh lattice given the same
    state."""
    p = U.Params(nx=16, ny=8, nz=8, seed=2)
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(3)
    st = synth.random_state(p.shape, seed=5)
    lat.set_state(st, n=7)
    assert lat.current() == (7, 1) and lat.kernel() == U.KERNEL_TILED
    assert torch.equal(lat.state().cpu(), torch.as_tensor(st).float())
    ref = U.Lattice(p, kernel=U.KERNEL_TILED)
    ref.set_state(st, n=7)
    lat.step(4)
    ref.step(4)
    assert torch.equal(lat.state(), ref.state())


def test_edge_cases_and_errors():
    p = U.Params(nx=8, ny=8, nz=8, m=0.0)
    lat = U.Lattice(p)
    s0 = lat.state().clone()
    lat.step(0)
    assert lat.n == 0 and torch.equal(lat.state(), s0)
    with pytest.raises(U.U1U1Error):
        lat.step(-1)
    with pytest.raises(U.U1U1Error):
        lat.detect_strings(tol=2)
    with pytest.raises(U.U1U1Error):
        U.Lattice(U.Params(nx=6, ny=8, nz=8))
    recs, lost = lat.read_records()
    assert recs == [] and lost == 0
    # detection ring overflow is reported, not silent
    lat.step(1100, detect_every=1)
    recs, lost = lat.read_records(max_records=2000)
    assert len(recs) == 1024 and lost == 1100 - 1024
    assert recs[-1][0]["n"] == 1099


def test_link_phase_routine_accuracy():
    """The FP32 cos/sin of link angles (reduction by 2 pi split in two
    floats, then the hardware sine and cosine, documented to 2^-21.41 on
    [-pi, pi]) stays within 6e-7 absolute of the double-precision values of
    the same FP32 angles, over the range lattices reach and far beyond it.
    The bound is set by what the step needs: with it the FP32 step stays
    within max-rel 6e-7 of the FP64 oracle after 20 steps at 64^3, against
    the 1e-5 the FP32 bulk is held to."""
    import ctypes
    th64 = torch.cat([torch.linspace(-50.0, 50.0, 2_000_001, dtype=torch.float64),
                      torch.tensor([0.0, -0.0, 1e-30, 3.0e3, -4095.0, 4097.0, 1.0e5, -2.5e6],
                                   dtype=torch.float64)])
    th = th64.float().cuda()
    sn = torch.empty_like(th)
    cs = torch.empty_like(th)
    U.check(U.lib().u1u1_eval_link_phase(ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(sn.data_ptr()),
                                         ctypes.c_void_p(cs.data_ptr()), th.numel(),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    ref = th.double()
    es = (sn.double() - torch.sin(ref)).abs().max().item()
    ec = (cs.double() - torch.cos(ref)).abs().max().item()
    assert es < 6e-7 and ec < 6e-7, (es, ec)


def test_fp64_link_phase_routine_accuracy():
    """The FP64 link-phase routine (table-driven: theta = m 2 pi/1024 + r)
    against the host's double-precision sine and cosine: within 2.5e-16
    absolute (about one ulp at 1) over the range lattices reach, at the
    rounding edges of m (odd multiples of pi/1024), on and beyond the exact
    range of the reduction (|theta| > 5.1e4 takes the library routine), and
    sin^2 + cos^2 = 1 to the same order."""
    import ctypes
    h = 2.0 * np.pi / 1024
    edges = np.concatenate([(np.arange(-3000, 3000) + 0.5) * h, np.arange(-3000, 3000) * h])
    edges = np.concatenate([edges, np.nextafter(edges, np.inf), np.nextafter(edges, -np.inf)])
    special = np.array([0.0, -0.0, 1e-300, 5e-324, np.pi, -np.pi, 2 * np.pi, 4.0e4, -5.1e4, 5.2e4, -6.0e4,
                        1.0e6, 1.0e9])
    th_h = np.concatenate([np.linspace(-60.0, 60.0, 1_000_001), edges, special])
    th = torch.from_numpy(th_h).cuda()
    sn = torch.empty_like(th)
    cs = torch.empty_like(th)
    U.check(U.lib().u1u1_eval_link_phase64(ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(sn.data_ptr()),
                                           ctypes.c_void_p(cs.data_ptr()), th.numel(),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    s_g, c_g = sn.cpu().numpy(), cs.cpu().numpy()
    es = np.abs(s_g - np.sin(th_h))
    ec = np.abs(c_g - np.cos(th_h))
    assert es.max() <= 2.5e-16 and ec.max() <= 2.5e-16, (es.max(), ec.max(), th_h[np.argmax(es)], th_h[np.argmax(ec)])
    assert np.abs(s_g * s_g + c_g * c_g - 1.0).max() <= 8e-16
    k0 = th_h.size - special.size
    assert s_g[k0] == 0.0 and s_g[k0 + 1] == 0.0 and c_g[k0] == 1.0 and c_g[k0 + 1] == 1.0


def test_edge_phase_routine_accuracy():
    """The FP32 edge phase arg(re + i im) (octant reduction + minimax
    polynomial) stays within 4e-7 rad of the double-precision arctangent of
    the same FP32 inputs, over all directions and magnitudes from 1e-30 to
    1e30, and follows atan2's conventions on the axes and at signed zeros
    (arg(+-0 - 0 i) = +-pi, arg(+-0 + 0 i) = +-0)."""
    import ctypes
    g = torch.Generator().manual_seed(11)
    n = 2_000_000
    ang = (torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1) * math.pi
    mag = torch.exp((torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1) * 69.0)
    re64 = torch.cat([mag * torch.cos(ang), torch.tensor([1.0, -1.0, 0.0, 0.0, 2.0, -2.0, 1.0, -1.0], dtype=torch.float64)])
    im64 = torch.cat([mag * torch.sin(ang), torch.tensor([0.0, 0.0, 1.0, -1.0, 2.0, 2.0, -1.0, -1.0], dtype=torch.float64)])
    re, im = re64.float(), im64.float()
    out = torch.empty_like(re).cuda()
    red, imd = re.cuda(), im.cuda()
    U.check(U.lib().u1u1_eval_edge_phase(ctypes.c_void_p(red.data_ptr()), ctypes.c_void_p(imd.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), re.numel(),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    ref = torch.atan2(im.double(), re.double())
    err = (out.cpu().double() - ref).abs()
    err = torch.minimum(err, 2 * math.pi - err)  # +-pi name the same direction
    assert err.max().item() < 4e-7, err.max().item()
    # signed zeros: the branch follows the signs exactly
    z = torch.tensor([0.0, -0.0, 0.0, -0.0], dtype=torch.float32)
    zi = torch.tensor([0.0, 0.0, -0.0, -0.0], dtype=torch.float32)
    zo = torch.empty(4, dtype=torch.float32, device="cuda")
    zr, zim = z.cuda(), zi.cuda()
    U.check(U.lib().u1u1_eval_edge_phase(ctypes.c_void_p(zr.data_ptr()), ctypes.c_void_p(zim.data_ptr()),
                                         ctypes.c_void_p(zo.data_ptr()), 4,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    want = torch.atan2(zi, z)
    got = zo.cpu()
    assert torch.equal(got, want) and torch.equal(torch.signbit(got), torch.signbit(want)), (got, want)


def test_autotune_keeps_state_and_reuses_cache(tmp_path):
    """The autotuner times its candidates on the handle's own state and
    restores it; a tuned handle then steps like an untuned one (bit for bit
    when the tiled kernel family is kept, to FP32 rounding otherwise); a
    second handle of the same shape takes the choice from the cache file."""
    p = radiation(96, 640, precision=U.FP32, seed=5)
    a = U.Lattice(p)
    a.step(5)
    s0 = a.state().clone()
    cache = str(tmp_path / "tune.txt")
    choice = a.autotune(cache_path=cache)
    assert torch.equal(a.state(), s0) and a.n == 5
    assert choice["kernel"] in (U.KERNEL_TILED, U.KERNEL_SIMPLE)
    b = U.Lattice(p)
    b.step(5)
    a.step(7)
    b.step(7)
    if choice["kernel"] == U.KERNEL_TILED:
        assert torch.equal(a.state(), b.state())
    else:
        err = field_maxrel(host_state(a), host_state(b))
        assert err.max() < 1e-6, err
    c = U.Lattice(p)
    assert c.autotune(cache_path=cache) == choice
    assert open(cache).read().count("96x96x96") == 1


def test_autotune_refuses_foreign_cache_entry(tmp_path):
    """A cache entry naming a wave count the tuner never picks (here 96) is
    refused before any launch: the block-partial buffers are sized for the
    tuner's own candidate grids.  The handle keeps its kernel choice."""
    p = radiation(64, 640, precision=U.FP32, seed=6)
    a = U.Lattice(p)
    cache = str(tmp_path / "tune.txt")
    choice = a.autotune(cache_path=cache)
    key = open(cache).read().split()[0]
    bad = str(tmp_path / "bad.txt")
    with open(bad, "w") as f:
        f.write(f"{key} {U.KERNEL_TILED} 96\n")
    b = U.Lattice(p)
    k0 = b.kernel()
    with pytest.raises(U.U1U1Error) as ei:
        b.autotune(cache_path=bad)
    assert ei.value.code == -1 and "96" in str(ei.value)  # INVALID_ARG
    assert b.kernel() == k0
    with open(bad, "w") as f:
        f.write(f"{key} 7 32\n")
    with pytest.raises(U.U1U1Error):
        b.autotune(cache_path=bad)
    # the same rule for a directly set chunking
    b.set_tile_waves(256)
    with pytest.raises(U.U1U1Error):
        b.set_tile_waves(96)
    assert choice["kernel"] in (U.KERNEL_TILED, U.KERNEL_SIMPLE)


def test_fp64_rate_probe():
    """The FP64 rate probe (the FP64 roofline's denominator) returns a rate
    between a tenth and twice GB300's nominal 1.25 TFLOP/s of non-tensor
    FP64, and the FP64 step, which does 389 FP64 operations per site,
    cannot run faster than that rate allows."""
    r = U.fp64_fma_rate()
    assert 0.125 < r < 2.5, r
    p = U.Params.cube(128, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=3, precision=U.FP64)
    lat = U.Lattice(p, kernel=U.KERNEL_TILED)
    lat.step(2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    lat.step(5)
    b.record()
    torch.cuda.synchronize()
    achieved = 389 * p.nsites * 5 / (a.elapsed_time(b) * 1e-3) / 1e12
    assert achieved < 1.05 * r, (achieved, r)


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("kernel", KERNELS)
def test_nan_fields_counted(prec, kernel):
    """NaN entries planted in a smooth state -- in a position, a momentum and
    an electric field at three sites, two of them at the same site, plus an
    infinity elsewhere -- are counted exactly as the oracle counts them (the
    infinity is not a NaN), by the diagnostics pass and by a fused
    detection step."""
    p = U.Params(nx=40, ny=16, nz=12, m=0.0, precision=prec)
    st = synth.smooth_state(p.shape, seed=3)
    st[0][3, 4, 5] = np.nan     # phi re
    st[12][3, 4, 5] = np.nan    # Psi re, same site
    st[17][7, 9, 33] = np.nan   # H_0
    st[8][1, 2, 3] = np.inf     # B_1
    lat = U.Lattice(p, kernel=kernel)
    lat.set_state(st)
    od = O.diagnostics(to_oracle(p), st, 0)
    assert od["nan_count"] == 3
    assert lat.diagnostics()["nan_count"] == 3
    lat.step(1, detect_every=1)
    (s, d), = lat.read_records()[0]
    assert d["nan_count"] == 3


def _swap_sectors(st):
    """phi <-> psi, A <-> B, Pi <-> Psi, E <-> H in a (20, ...) state."""
    idx = [2, 3, 0, 1, 7, 8, 9, 4, 5, 6, 12, 13, 10, 11, 17, 18, 19, 14, 15, 16]
    return st[idx]


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("kernel", KERNELS)
def test_sector_symmetries_on_gpu(prec, kernel):
    """The symmetries of Sec. II on the GPU kernels, bit for bit: exchanging
    the sectors' fields and couplings exchanges the results of 6 steps (a
    p/q mix-up of any per-sector coefficient or field index breaks it), the
    windings and string counts swap likewise; and with kappa = 0 the p
    sector evolves independently of anything done to the q sector."""
    kw = dict(m=0.5, beta=-1.0, eta0=1.0, eta_ref=1.0)
    p = U.Params(nx=36, ny=20, nz=12, precision=prec, **kw, **UNEQUAL)
    q = U.Params(nx=36, ny=20, nz=12, precision=prec, **kw, lambda_p=UNEQUAL["lambda_q"],
                 lambda_q=UNEQUAL["lambda_p"], e_p=UNEQUAL["e_q"], e_q=UNEQUAL["e_p"],
                 sigma_p=UNEQUAL["sigma_q"], sigma_q=UNEQUAL["sigma_p"], kappa=UNEQUAL["kappa"])
    st = synth.random_state(p.shape, seed=23, a_amp=1.0, mom_amp=0.5)
    a = U.Lattice(p, kernel=kernel)
    a.set_state(st)
    b = U.Lattice(q, kernel=kernel)
    b.set_state(_swap_sectors(st))
    sa, sb = a.detect_strings(tol=0), b.detect_strings(tol=0)
    for k1, k2 in (("n_p", "n_q"), ("nonzero_p", "nonzero_q"), ("n_w2_p", "n_w2_q")):
        assert sa[k1] == sb[k2] and sa[k2] == sb[k1], k1
    assert sa["n_pq_plaq"] == sb["n_pq_plaq"] and sa["n_pq_cell"] == sb["n_pq_cell_q"]
    a.step(6)
    b.step(6)
    assert torch.equal(a.state(), _swap_sectors(b.state()))
    # kappa = 0: the q sector cannot act on the p sector
    p0 = U.Params(nx=36, ny=20, nz=12, precision=prec, **kw, **dict(UNEQUAL, kappa=0.0))
    c = U.Lattice(p0, kernel=kernel)
    c.set_state(st)
    st2 = st.copy()
    st2[2:4] *= 1.7          # psi
    st2[[7, 8, 9]] += 0.3    # B
    st2[[12, 13]] -= 0.2     # Psi
    st2[[17, 18, 19]] *= 0.5  # H
    d = U.Lattice(p0, kernel=kernel)
    d.set_state(st2)
    c.step(6)
    d.step(6)
    pfields = [0, 1, 4, 5, 6, 10, 11, 14, 15, 16]
    assert torch.equal(c.state()[pfields], d.state()[pfields])


@pytest.mark.parametrize("prec,tol", [(U.FP64, 1e-10), (U.FP32, 2e-5)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_gauge_covariance_on_gpu(prec, tol, kernel):
    """Lattice gauge covariance of the GPU step (Sec. II covariant
    derivatives): stepping a gauge-transformed state (phi, pi -> e^{i Lambda}
    phi, pi; A_i -> A_i + (Lambda(x+i) - Lambda(x)) / dx) equals transforming
    the stepped state, the windings are unchanged on unflagged plaquettes and
    the diagnostic sums agree; on a box whose x extent mixes tensor-copy and
    cp.async tiles, with unequal couplings."""
    import pins
    p = U.Params(nx=136, ny=40, nz=12, m=0.5, beta=1.0, eta0=1.0, eta_ref=9.0, precision=prec, **UNEQUAL)
    op = to_oracle(p)
    st = synth.random_state(p.shape, seed=41, a_amp=1.0, mom_amp=0.5)
    lam = synth.gauge_parameter(p.shape, seed=42)
    a = U.Lattice(p, kernel=kernel)
    a.set_state(st)
    b = U.Lattice(p, kernel=kernel)
    b.set_state(pins.gauge_transform(op, st, lam))
    ra, rb = a.detect_strings(tol=1, windings=True), b.detect_strings(tol=1, windings=True)
    fa = ra["n_flagged"] + rb["n_flagged"]
    assert abs(ra["n_p"] - rb["n_p"]) <= fa and abs(ra["n_q"] - rb["n_q"]) <= fa
    if fa == 0:
        assert torch.equal(ra["windings"], rb["windings"])
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("kin_p", "kin_q", "grad_p", "grad_q", "el_p", "el_q", "mag_p", "mag_q", "pot", "vint", "rl_num"):
        assert abs(da[k] - db[k]) <= 10 * tol * max(1.0, abs(da[k])), (k, da[k], db[k])
    a.step(5)
    b.step(5)
    want = pins.gauge_transform(op, host_state(a), lam)
    err = field_maxrel(host_state(b), want)
    assert err.max() <= tol, err
