"""Benchmark of the U(1)xU(1) hot path: site-updates/s and HBM roofline.

Workload (default): the 1024^3 single-GPU machine of the paper's model in the
radiation era, dx = 0.5, deta = 0.1, beta = 1, lambda = 2, e = 1, sigma = 1,
kappa = 0.9, seeded random-phase initial conditions, FP32 bulk, winding
detection every 16 steps.  One benchmark "step" is one detection period: 16
leapfrog steps, the first fused with the diagnostic sums, the plaquette
windings of its input state (a separate kernel on the positions the step
leaves in place), the cell-overlap pass and the reduction finalize (every
row of the hot path).  value = site-updates/s over the timed
periods (one site-update advances all 20 real fields of both sectors by one
deta); inputs (86 GB) are far larger than L2, so no flush is needed.

Also reported: the step kernel's roofline (algorithmic 160 B/site over its
CUDA-event time against the measured HBM copy bandwidth), an end-to-end
number through the public API with host buffers (state uploaded from pinned
memory, per-period record reads, state downloaded), the FP64 step, and the
FP64 CPU oracle on a bounded sample of the same workload (cpu_baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-updates/s & % HBM roofline, FP32 vs FP64, U(1)xU(1) step at 1024^3"
BYTES_PER_SITE = {"fp32": 160, "fp64": 320}  # read 20 + write 20 words
# FP64 step: 126 DFMA + 60 DADD + 77 DMUL per site (ncu thread-instruction
# counts of one launch at 256^3) = 389 FP64 operations; its ceiling is the
# FP64 rate measured in the same run by the library's FMA probe (nominal
# GB300 non-tensor FP64: 1.25 TFLOP/s, used only if the probe fails)
FP64_FLOPS_PER_SITE = 389
FP64_INSTR_PER_SITE = 126 + 60 + 77  # FP64 pipe instructions (DFMA, DADD, DMUL) per site
FP64_NOMINAL_TFLOPS = 1.25
# standalone string detection: the windings kernel reads the ten position
# fields (40 B/site in FP32) and writes 2 face bytes per site, the cell pass
# reads those back and writes 0.25 B/site of masks
DETECT_BYTES_PER_SITE = {"fp32": 40 + 2 + 2 + 0.25, "fp64": 80 + 2 + 2 + 0.25}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# sources the leapfrog step kernel is compiled from: a recorded DRAM count is
# used only while their hash is the one it was taken with
STEP_KERNEL_SOURCES = ("paper_2208_01525_gb300/csrc/k_tiled.cu", "paper_2208_01525_gb300/csrc/site_math.cuh",
                       "paper_2208_01525_gb300/csrc/u1u1_internal.cuh")
TRAFFIC_RECORD = "profiles/leapfrog_step_fp32_1024cubed_dram.md"


def step_kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(n, tag, waves):
    """DRAM bytes (read + write) of one step-kernel launch from the committed
    ncu summary, or None when it was taken on another lattice, precision,
    z-chunking (wave target) or kernel source."""
    try:
        with open(os.path.join(ROOT, TRAFFIC_RECORD)) as f:
            kv = dict(line.split(":", 1) for line in f if line.startswith("record-"))
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if (int(kv["record-lattice"]) != n or kv["record-precision"] != tag
                or kv["record-source-sha256"] != step_kernel_hash()):
            return None
        return float(kv[f"record-dram-bytes-per-launch-w{waves}"])
    except (OSError, KeyError, ValueError):
        return None


def combine_ranks(ms, units_local, world, device=None):
    """Whole-job figures from each rank's timed region: the slowest rank's
    time (max over ranks) and the units all ranks processed (sum), giving
    value = units / time.  Without a process group (world 1) the local
    figures are returned."""
    units = float(units_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        tu = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        ms, units = float(tm.item()), float(tu.item())
    return ms, units / (ms * 1e-3)


def _cdiv(a, b):
    return -(-a // b)


def measure_partials(n, tiled):
    """Block partials a detection step of an n^3 lattice writes (the grid
    formulas of the library's measuring kernels: the step kernel's 32-wave
    z-chunking plus the windings kernel's on the tiled path; the simple
    kernel's fixed grid otherwise)."""
    if not tiled:
        return 152 * 8
    tiles = _cdiv(n, 32) * _cdiv(n, 8)
    chunks = max(1, _cdiv(152 * 3 * 32, tiles))
    lz = min(max(_cdiv(n, chunks), 32), n)
    step = tiles * _cdiv(n, lz)
    wt = _cdiv(n, 31) * _cdiv(n, 7)
    wc = max(1, min(_cdiv(152 * 3 * 16, wt), n // 32))
    return step + wt * _cdiv(n, _cdiv(n, wc))


def launches_per_period(n, de, tiled):
    """Kernel launches of one detection period: de step launches (the first
    one measuring), the windings kernel (tiled path), cell bits, overlap and
    the finalize (two stages above 2048 block partials)."""
    stage = 1 if measure_partials(n, tiled) > 2048 else 0
    return de + (1 if tiled else 0) + 2 + 1 + stage


def workload_params(U, n, precision, beta=1.0, seed=2024, nz=0):
    # 2560 steps to eta = 257 for the 1024^3 box; a = 1 at the end of the run.
    # nz > 0: an n x n x nz slab of the same workload (small profiling cases)
    return U.Params(nx=n, ny=n, nz=nz if nz > 0 else n, m=0.5, beta=beta, eta0=1.0, eta_ref=1.0 + 0.1 * 2560,
                    seed=seed, precision=precision)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        lines = list(self.f)
        os.unlink(self.f.name)
        return self.summarize(lines, self.uuid)

    @staticmethod
    def summarize(lines, uuid=None):
        """Median SM clock under load, maximum clock and the throttle reasons
        seen Active, from nvidia-smi CSV lines (FIELDS order, no header)."""
        rows = [ln.strip().split(", ") for ln in lines if ln.strip()]
        mine = [r for r in rows if uuid is None or uuid in r[0]] or rows
        sm = [float(r[1].split()[0]) for r in mine if len(r) > 2 and r[1].split()[0].replace(".", "").isdigit()]
        mx = [float(r[2].split()[0]) for r in mine if len(r) > 2 and r[2].split()[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in mine:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n=128, nsteps=16, detect=True):
    """The FP64 oracle, as it stands, on all host cores: one detection period
    (16 leapfrog steps plus windings, cells, overlap and diagnostics) on an
    n^3 box of the same model.  Returns (site-updates/s, seconds, cores)."""
    import oracle as O
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    p = O.Params(n, n, n, m=0.5, beta=1.0, eta0=1.0, eta_ref=1.0 + 0.1 * 2560, seed=2024)
    st = O.init(p)
    t0 = time.perf_counter()
    if detect:
        O.strings(p, st, tol=1)
        O.diagnostics(p, st, 0)
    O.step(p, st, 0, nsteps)
    dt = time.perf_counter() - t0
    return nsteps * n ** 3 / dt, dt, O.max_threads()


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores, each
    step one detection period on a 96^3 sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    n = args.ref_n
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    p = O.Params(n, n, n, m=0.5, beta=1.0, eta0=1.0, eta_ref=1.0 + 0.1 * 2560, seed=2024)
    st = O.init(p)
    step_n = 0

    def one_period():
        nonlocal step_n
        O.strings(p, st, tol=1)
        O.diagnostics(p, st, step_n)
        O.step(p, st, step_n, args.detect_every)
        step_n += args.detect_every

    for _ in range(args.warmup):
        one_period()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_period()
    dt = time.perf_counter() - t0
    value = args.steps * args.detect_every * n ** 3 / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"U(1)xU(1) leapfrog + detection every {args.detect_every} steps, radiation, "
                               f"beta=1, {n}^3 sample of the 1024^3 box (CPU oracle)",
                   "lattice": n, "detect_every": args.detect_every},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": O.max_threads(), "kind": "oracle",
                         "sample": f"{args.steps} detection periods of {args.detect_every} steps on {n}^3"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def period_rate(U, torch, p, de, periods, warmup, dev):
    """Detection periods of de steps (the first step of each fused with
    detection) on a fresh lattice of parameters p: site-updates/s, ms per
    period and the last record."""
    lat = U.Lattice(p, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        lat.step(de, detect_every=de)
    torch.cuda.synchronize()
    lat.read_records()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(periods):
        lat.step(de, detect_every=de)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / periods
    recs, _ = lat.read_records()
    lat.close()
    del lat
    torch.cuda.empty_cache()
    last = recs[-1] if recs else None
    return {"value": de * p.nsites / (ms * 1e-3), "unit": "site-updates/s", "ms_per_period": ms,
            "detect_every": de, "periods": periods,
            "last_record": None if last is None else {"n": last[0]["n"], "xi_w": last[0]["xi_w"],
                                                      "xi_l": last[1]["xi_l"], "v2_l": last[1]["v2_l"]}}


def config_legs(U, torch, dev, warmup):
    """The smaller configurations of the workload set, each a few timed
    detection periods: 256^3 radiation beta = 1 with detection every 10
    steps in FP32 and FP64 (640-step run to eta = 65), and 512^3 with full
    detection every 8 steps in the radiation and matter eras for beta = 1
    and beta = 0 (1280-step runs to eta = 129)."""
    out = {}
    for prec, tag in ((U.FP32, "fp32"), (U.FP64, "fp64")):
        p = U.Params.cube(256, m=0.5, beta=1.0, eta0=1.0, eta_ref=65.0, seed=1, precision=prec)
        out[f"256_radiation_beta1_{tag}"] = period_rate(U, torch, p, 10, 5, warmup, dev)
    for m, era in ((0.5, "radiation"), (2.0 / 3.0, "matter")):
        for beta in (1.0, 0.0):
            p = U.Params.cube(512, m=m, beta=beta, eta0=1.0, eta_ref=129.0 if beta > 0 else 1.0, seed=3,
                              precision=U.FP32)
            out[f"512_{era}_beta{int(beta)}_fp32"] = period_rate(U, torch, p, 8, 5, warmup, dev)
    return out


def ensemble_bench(U, torch, dev):
    """The batched configuration: 48 independent boxes (16 x 64^3, 16 x 128^3,
    16 x 192^3), matter era, beta cycling 1, 0, -1, seeds 1000 + b, each run
    to half its light-crossing time (160 / 320 / 480 steps), FP32.  The
    library's ensemble autotuner picks the schedule (persistent or per-step),
    the work-item z-chunk and whether the persistent kernel uses tensor
    copies first; then each mode is timed on its second run (the first one
    captures the graph), without and with detection every 16 steps inside
    the run, and the speed-up over the unbatched loop is the tuned
    schedule's."""
    sizes = [64] * 16 + [128] * 16 + [192] * 16
    steps = [n * 5 // 2 for n in sizes]  # n dx / 2 in units of deta = 0.1
    ps = []
    for b, n in enumerate(sizes):
        beta = (1.0, 0.0, -1.0)[b % 3]
        eta_end = 1.0 + 0.1 * 2 * steps[b]
        ps.append(U.Params.cube(n, m=2.0 / 3.0, beta=beta, eta0=1.0, eta_ref=eta_end if beta > 0 else 1.0,
                                seed=1000 + b, precision=U.FP32))
    work = sum(s * n ** 3 for s, n in zip(steps, sizes))
    out = {"boxes": len(sizes), "site_updates_per_run": work, "steps": "160/320/480", "era": "matter",
           "beta": "1,0,-1 round-robin"}
    stream = torch.cuda.current_stream()
    modes = (("persistent_graph", U.ENS_PERSISTENT, True), ("per_step_graph", U.ENS_PER_STEP, True),
             ("unbatched", U.ENS_UNBATCHED, False))

    def timed(ens, mode, graph, de):
        ens.run(steps, mode=mode, use_graph=graph, detect_every=de)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.run(steps, mode=mode, use_graph=graph, detect_every=de)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        return {"ms": ms, "site_updates_per_s": work / (ms * 1e-3), "status": ens.status()}

    # one ensemble for every timed run (12 runs of up to 480 steps per box)
    ens = U.Ensemble(ps, device=dev, horizon=8192)
    out["autotuned"] = ens.autotune(probe_steps=24)
    # the schedule the tuner chose (persistent or per-step, both graph-captured)
    tuned = "persistent_graph" if out["autotuned"]["mode"] == U.ENS_PERSISTENT else "per_step_graph"
    out["tuned_schedule"] = tuned
    for name, mode, graph in modes:
        out[name] = timed(ens, mode, graph, 0)
    out["speedup_vs_unbatched"] = out[tuned]["site_updates_per_s"] / out["unbatched"]["site_updates_per_s"]
    # the tuned run against the copy bandwidth at the step's 160 algorithmic
    # bytes per site update (whole run: every launch of the graph counted)
    hbm, kind = peaks()
    gbs = out[tuned]["site_updates_per_s"] * BYTES_PER_SITE["fp32"] / 1e9
    out["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                       "peak_kind": kind, "bytes_per_site": BYTES_PER_SITE["fp32"]}
    # the same runs with detection every 16 steps inside the run (windings,
    # cells, overlap and diagnostic sums of every box, records in each box's
    # ring); batched modes detect all boxes of a run step in one launch per pass
    for bx in ens.boxes:
        bx.read_records(max_records=1024)
    det = {"detect_every": 16}
    for name, mode, graph in modes:
        det[name] = timed(ens, mode, graph, 16)
        det[name]["records"] = sum(len(bx.read_records(max_records=1024)[0]) for bx in ens.boxes)
    det["speedup_vs_unbatched"] = det[tuned]["site_updates_per_s"] / det["unbatched"]["site_updates_per_s"]
    out["with_detection"] = det
    ens.close()
    del ens
    torch.cuda.empty_cache()
    # the small-box class alone (16 x 64^3), where per-box launches cannot fill the GPU
    small = [p for p, n in zip(ps, sizes) if n == 64]
    ssteps = [s_ for s_, n in zip(steps, sizes) if n == 64]
    swork = sum(s_ * 64 ** 3 for s_ in ssteps)
    res = {}
    ens = U.Ensemble(small, device=dev, horizon=2048)
    res["autotuned"] = ens.autotune(probe_steps=24)
    for name, mode, graph in (("persistent_graph", U.ENS_PERSISTENT, True), ("per_step_graph", U.ENS_PER_STEP, True),
                              ("unbatched", U.ENS_UNBATCHED, False)):
        ens.run(ssteps, mode=mode, use_graph=graph)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.run(ssteps, mode=mode, use_graph=graph)
        b.record(stream)
        torch.cuda.synchronize()
        res[name] = swork / (a.elapsed_time(b) * 1e-3)
    ens.close()
    del ens
    torch.cuda.empty_cache()
    stuned = "persistent_graph" if res["autotuned"]["mode"] == U.ENS_PERSISTENT else "per_step_graph"
    out["small_boxes_64"] = {"site_updates_per_s": res, "tuned_schedule": stuned,
                             "speedup_vs_unbatched": res[stuned] / res["unbatched"]}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2208_01525_gb300 as U

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.n
    prec = U.FP64 if args.precision == "fp64" else U.FP32
    tag = "fp64" if prec == U.FP64 else "fp32"
    # independent realisations per rank (replicas: the path has no exchange step)
    p = workload_params(U, n, prec, seed=2024 + rank, nz=args.nz)
    lat = U.Lattice(p, device=dev, kernel=args.kernel)
    tune = None
    if args.waves > 0:
        # a fixed z-chunking of the tiled kernel instead of the autotuner's
        lat.set_kernel(U.KERNEL_TILED)
        lat.set_tile_waves(args.waves)
        tune = {"kernel": U.KERNEL_TILED, "waves": args.waves, "fixed": True}
    elif args.tune and args.kernel == U.KERNEL_AUTO:
        # the library's autotuner picks the step kernel and its z-chunking
        # on this lattice (timed on the lattice's own state, restored)
        tune = lat.autotune()
    kernel_used = lat.kernel()
    waves_used = tune["waves"] if tune else 32  # the library's default wave target
    de = args.detect_every
    V = p.nsites
    stream = torch.cuda.current_stream()

    # warm-up periods
    for _ in range(args.warmup):
        lat.step(de, detect_every=de)
    torch.cuda.synchronize()
    lat.read_records()

    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "")) or None
    sampler = ClockSampler(uuid)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        lat.step(1, detect_every=de)          # fused step + detection, overlap, finalize
        ev[k][1].record(stream)
        lat.step(de - 1, detect_every=de)     # plain fused kick-drift steps
        ev[k][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms, value = combine_ranks(t_start.elapsed_time(t_end), args.steps * de * V, world, dev)
    recs, lost = lat.read_records()
    plain_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / (args.steps * (de - 1))
    det_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    peak, peak_kind = peaks()
    achieved = BYTES_PER_SITE[tag] * V / (plain_ms * 1e-3) / 1e9
    last = recs[-1] if recs else None

    # standalone passes on the current state (no step): the diagnostics pass
    # (all sums and the Gauss residual; reads positions and momenta, 80 B/site
    # in FP32) and string detection (windings of the positions, cells,
    # overlap); each call ends with its record copied to the host
    passes = None
    if args.passes:
        passes = {}
        for name, fn in (("diagnostics", lat.diagnostics), ("detect_strings", lat.detect_strings)):
            fn()
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            t_ms = min(ts)
            passes[name] = {"ms": t_ms, "sites_per_s": V / (t_ms * 1e-3)}
        del fn  # the bound method would keep the lattice (and its fields) alive
        rd = BYTES_PER_SITE[tag] // 2 * V  # the pass reads the 20 words of every site once
        passes["diagnostics"]["hbm_frac"] = rd / (passes["diagnostics"]["ms"] * 1e-3) / 1e9 / peak
        passes["diagnostics"]["bytes_per_site"] = BYTES_PER_SITE[tag] // 2
        db = DETECT_BYTES_PER_SITE[tag]
        passes["detect_strings"]["hbm_frac"] = db * V / (passes["detect_strings"]["ms"] * 1e-3) / 1e9 / peak
        passes["detect_strings"]["bytes_per_site"] = db

    # end-to-end through the public API with host buffers
    e2e = None
    if args.e2e:
        host = [torch.empty(V, dtype=lat.dtype, pin_memory=True) for _ in range(20)]
        lat.download(host)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        lat.upload(host)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            lat.step(de, detect_every=de)
            lat.read_records()                # D2H of the period's record + host epilogue
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lat.download(host)
        torch.cuda.synchronize()
        barrier()
        t3 = time.perf_counter()
        e2e_s = t3 - t0
        state_bytes = 20 * V * lat.dtype.itemsize
        rec_bytes = 360  # one detection record copied per period
        _, e2e_value = combine_ranks(e2e_s * 1e3, args.steps * de * V, world, dev)
        e2e = {"value": e2e_value, "unit": "site-updates/s",
               "h2d_bytes_per_step": state_bytes / args.steps,
               "d2h_bytes_per_step": state_bytes / args.steps + rec_bytes,
               "what": "upload state from pinned host, K periods each followed by a record read, "
                       "download state",
               "transfer": ("SM copy kernel through the mapped host address"
                            if all(U.host_span_mapped(t.data_ptr(), t.numel() * t.element_size()) for t in host)
                            else "copy engines"),
               "upload_s": t1 - t0, "periods_s": t2 - t1, "download_s": t3 - t2}
        del host

    lat.close()
    del lat
    gc.collect()
    torch.cuda.empty_cache()

    # the core-growth case of the same box (beta = -1, unit width at the
    # start: a = 1 at eta0), same kernel choice, a few detection periods
    beta_m1 = None
    if args.beta_m1_steps > 0:
        pb = U.Params.cube(n, m=0.5, beta=-1.0, eta0=1.0, eta_ref=1.0, seed=2024 + rank, precision=prec)
        latb = U.Lattice(pb, device=dev, kernel=kernel_used)
        if kernel_used == U.KERNEL_TILED:
            latb.set_tile_waves(waves_used)
        for _ in range(args.warmup):
            latb.step(de, detect_every=de)
        torch.cuda.synchronize()
        latb.read_records()
        evb = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.beta_m1_steps)]
        for k in range(args.beta_m1_steps):
            evb[k][0].record(stream)
            latb.step(1, detect_every=de)
            evb[k][1].record(stream)
            latb.step(de - 1, detect_every=de)
            evb[k][2].record(stream)
        torch.cuda.synchronize()
        tb = sum(e[0].elapsed_time(e[2]) for e in evb) / args.beta_m1_steps
        pl = sum(e[1].elapsed_time(e[2]) for e in evb) / (args.beta_m1_steps * (de - 1))
        recb, _ = latb.read_records()
        beta_m1 = {"beta": -1.0, "lattice": n, "periods": args.beta_m1_steps, "ms_per_period": tb,
                   "value": de * V / (tb * 1e-3), "unit": "site-updates/s",
                   "detect_ms_per_period": sum(e[0].elapsed_time(e[1]) for e in evb) / args.beta_m1_steps,
                   "plain_ms_per_launch": pl,
                   "hbm_frac": BYTES_PER_SITE[tag] * V / (pl * 1e-3) / 1e9 / peak,
                   "last_record": None if not recb else {"n": recb[-1][0]["n"], "xi_w": recb[-1][0]["xi_w"],
                                                          "f_total": recb[-1][0]["f_total"]}}
        latb.close()
        del latb
        gc.collect()
        torch.cuda.empty_cache()

    # FP64 step throughput (same box when it fits)
    fp64 = None
    if args.fp64_n > 0 and prec == U.FP32:
        n64 = args.fp64_n
        p64 = workload_params(U, n64, U.FP64, seed=2024 + rank)
        # 30 field arrays plus the handle's scratch (face bytes, masks, partials)
        need = (30 * 8 + 3) * p64.nsites
        free = torch.cuda.mem_get_info(dev)[0]
        if free <= need:
            fp64 = {"lattice": n64, "skipped": f"needs {need / 1e9:.1f} GB, {free / 1e9:.1f} GB free"}
        else:
            # the FP64 ceiling measured on this device (FMA probe, no setting changed)
            try:
                fp64_peak, fp64_kind = U.fp64_fma_rate(), "measured (FP64 FMA probe)"
            except U.U1U1Error:
                fp64_peak, fp64_kind = FP64_NOMINAL_TFLOPS, "nominal"
            lat64 = U.Lattice(p64, device=dev, kernel=args.kernel)
            lat64.step(2)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat64.step(args.fp64_steps)
            b.record(stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b) / args.fp64_steps
            # the FP64 step is bound by GB300's FP64 arithmetic, not by HBM:
            # FP64_FLOPS_PER_SITE from ncu instruction counts (DFMA x 2 + DADD
            # + DMUL per site) against the FP64 rate measured above
            tflops = FP64_FLOPS_PER_SITE * p64.nsites / (t64 * 1e-3) / 1e12
            fp64 = {"lattice": n64, "value": p64.nsites / (t64 * 1e-3), "unit": "site-updates/s",
                    "ms_per_step": t64,
                    "hbm_frac": BYTES_PER_SITE["fp64"] * p64.nsites / (t64 * 1e-3) / 1e9 / peak,
                    # instr_frac: the same time against the probe's rate of FP64
                    # instructions (one FMA = two operations), counting DADD and
                    # DMUL, which occupy the pipe like an FMA, as one each
                    "roofline": {"bound": "alu", "achieved": tflops, "peak": fp64_peak,
                                 "unit": "TFLOP/s (FP64)", "frac": tflops / fp64_peak,
                                 "peak_kind": fp64_kind, "flops_per_site": FP64_FLOPS_PER_SITE,
                                 "instr_per_site": FP64_INSTR_PER_SITE,
                                 "instr_frac": FP64_INSTR_PER_SITE * p64.nsites / (t64 * 1e-3) / 1e12 / (fp64_peak / 2)},
                    "steps": args.fp64_steps}
            lat64.close()
            del lat64
            torch.cuda.empty_cache()

    ens = None
    if args.ensemble:
        ens = ensemble_bench(U, torch, dev)

    configs = None
    if args.configs:
        configs = config_legs(U, torch, dev, args.warmup)

    cpu = None
    if rank == 0 and args.cpu:
        v, dt, cores = cpu_baseline(args.cpu_n)
        cpu = {"value": v, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"one detection period (16 steps + windings, overlap, diagnostics) on "
                         f"{args.cpu_n}^3, {dt:.1f} s"}

    if rank == 0:
        box = f"{n}^3" if args.nz <= 0 else f"{n}x{n}x{args.nz} slab"
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if tag == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": f"U(1)xU(1) {box} leapfrog, radiation era, beta=1, detection every {de} "
                                   f"steps (one step = {de} leapfrog steps)",
                       "lattice": n, "dx": 0.5, "deta": 0.1, "detect_every": de,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "autotuned": tune},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": (recorded_traffic(n, tag, waves_used)
                                                                if kernel_used != U.KERNEL_SIMPLE else None),
                         "traffic_unit": "bytes per launch", "peak_kind": peak_kind,
                         "kernel": "leapfrog step", "bytes_per_site": BYTES_PER_SITE[tag],
                         "ms_per_launch": plain_ms},
            "detect_ms_per_period": det_ms,
            "passes": passes,
            "clocks": clocks,
            "gpu_launches": args.steps * launches_per_period(n, de, kernel_used != U.KERNEL_SIMPLE),
            "e2e": e2e,
            "fp64": fp64,
            "beta_m1": beta_m1,
            "ensemble": ens,
            "configs": configs,
            "cpu_baseline": cpu,
            "records_lost": lost,
            "last_record": None if last is None else {
                "n": last[0]["n"], "xi_w": last[0]["xi_w"], "f_total": last[0]["f_total"],
                "xi_l": last[1]["xi_l"], "v2_l": last[1]["v2_l"]},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=0, help="planes of an n x n x nz slab (default: a cube)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--detect-every", type=int, default=16)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--fp64-n", type=int, default=1024)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--beta-m1-steps", type=int, default=5,
                    help="detection periods timed on the beta = -1 (core growth) box; 0 skips it")
    ap.add_argument("--cpu-n", type=int, default=128)
    ap.add_argument("--ref-n", type=int, default=96)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
    ap.add_argument("--no-ensemble", dest="ensemble", action="store_false")
    ap.add_argument("--no-passes", dest="passes", action="store_false")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the 256^3 and 512^3 configuration legs")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--waves", type=int, default=0,
                    help="fixed wave target of the tiled step kernel (8 .. 256) instead of autotuning")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
