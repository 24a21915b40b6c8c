"""Benchmark of the GB300 3D-ACA tensor path (one JSON line on rank 0).

Workload (default): the batched, uneven-block configuration, a finned
machine housing (closed cylinder r = 0.1 m, length 0.3 m, 12 fins 5 mm thick,
end caps; 28,704 flat triangles, 1 % vertex jitter), Galerkin single layer
P0 x P0, c = 343 m/s, gCQ contour of 2-stage Radau IIA for 256 geometrically
graded steps (ratio 1.01, T = 0.015 s; 256 contour points, 128 unique), PCA
cluster tree with leaf size 64 and eta = 2, 3D-ACA at eps = 1e-4 (face ACA
1e-6), Sauter-Schwab with 5 Gauss points per variable, one persistent launch
per phase under captured graphs, autotuned far launch; apply with 16
right-hand sides.  Other workloads (--workload): icospheres with 1280 and
5120 triangles (BDF2 N = 64, c = 1; single and double layer) and housings of
about 60k and 80k triangles (256 / 512 contour points; 32 right-hand sides at
80k).  The 80k housing is not the default: one step takes about 13 s, so the
default 20 timed + 5 warm-up steps would hold the GPU for over 5 minutes.

One step = the whole path: block cluster tree, compression (touching-pair
table, near-field entries, near and far 3D-ACA) and one multi-frequency
apply.  Metric (value): operator entries evaluated per second, every entry
A(i, j, s_k) that the compression's kernels evaluate counted once per
evaluation (near-field tensor, far-field fibres, frequency tubes); the
dense-equivalent rate (rows * cols * N_Q / step) and the time to the tensor
are reported beside it.  Inputs are resident in HBM before the timed region;
the e2e figure repeats the step through the host-buffer API (mesh upload,
tree, compression, apply with host W and y).

--impl reference times the FP64 CPU oracle (the reference arm of this
comparison) on a bounded block sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2505_00715_gb300.inputs import graded_steps, housing, icosphere, random_weights  # noqa: E402

WORKLOADS = {
    # icospheres (R = 1, c = 1) with BDF2 convolution quadrature
    "sphere1280_slp_bdf2_N64": dict(level=3, op="SLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                    ng=5, nrhs=16, c=1.0),
    "sphere5120_slp_bdf2_N64": dict(level=4, op="SLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                    ng=5, nrhs=16, c=1.0),
    "sphere5120_dlp_bdf2_N64": dict(level=4, op="DLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                    ng=5, nrhs=16, c=1.0),
    "sphere5120_adlp_bdf2_N64": dict(level=4, op="ADLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                     ng=5, nrhs=16, c=1.0),
    # finned machine housings (c = 343 m/s) with the gCQ contour of 2-stage Radau
    # IIA over geometrically graded steps (T = 0.015 s); 512 steps are graded so
    # that dt_max / dt_min equals that of 256 steps of ratio 1.01
    # a smaller housing of the same recipe (9024 triangles): one-launch profiling captures
    "housing9k_slp_gcq256": dict(housing=10000, op="SLP", gcq=(256, 1.01, 0.015), leaf=64, eta=2.0, eps=1e-4,
                                 eps_aca=1e-6, ng=5, nrhs=16, c=343.0),
    "housing30k_slp_gcq256": dict(housing=30000, op="SLP", gcq=(256, 1.01, 0.015), leaf=64, eta=2.0, eps=1e-4,
                                  eps_aca=1e-6, ng=5, nrhs=16, c=343.0),
    "housing60k_slp_gcq256": dict(housing=60000, op="SLP", gcq=(256, 1.01, 0.015), leaf=64, eta=2.0, eps=1e-4,
                                  eps_aca=1e-6, ng=5, nrhs=16, c=343.0),
    "housing80k_slp_gcq512": dict(housing=80000, op="SLP", gcq=(512, 1.01 ** (255.0 / 511.0), 0.015), leaf=64,
                                  eta=2.0, eps=1e-4, eps_aca=1e-6, ng=5, nrhs=32, c=343.0),
}


def workload_mesh(cfg):
    return housing(cfg["housing"], seed=0) if "housing" in cfg else icosphere(cfg["level"])


def workload_freqs(td, ctx, cfg):
    if "gcq" in cfg:
        nq, ratio, T_end = cfg["gcq"]
        dts = graded_steps(nq, ratio, T_end)
        return td.Freqs.gcq(ctx, dts, td.RADAU2, nq, rho=1.0)
    return td.Freqs.bdf2(ctx, cfg["N"], cfg["dt"])


def job_throughput(local_ms_total, units_per_step, steps, world, dist=None):
    """Whole-job throughput of N independent replicas (weak scaling): the
    timed region is the slowest rank's (max over ranks), every rank processed
    units_per_step units per step.  Returns (value per second, max ms)."""
    total_ms = float(local_ms_total)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * float(units_per_step) * steps / (total_ms / 1e3), total_ms


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_problem(cfg):
    """The workload for the oracle: mesh, unique frequencies, tree, operator."""
    import oracle as orc
    V, T = workload_mesh(cfg)
    m = orc.Mesh(V, T)
    if "gcq" in cfg:
        nq, ratio, T_end = cfg["gcq"]
        dts = graded_steps(nq, ratio, T_end)
        s, _, _ = orc.freqs_gcq(dts.min(), dts.max(), 1, nq, len(dts), rho=1.0)
        su = s[:nq // 2]  # points l and NQ-1-l are conjugate
    else:
        s = orc.freqs_bdf2(cfg["N"], cfg["dt"])
        su = s[:cfg["N"] // 2 + 1]  # points k and N-k are conjugate
    cols = 1 if cfg["op"] == "DLP" else 0
    tr = orc.Tree(m, 0, cols, cfg["leaf"], cfg["eta"])
    return m, su, tr, getattr(orc, cfg["op"])


def oracle_sample_mask(blocks, per_sample, offset, seed=3):
    """Deterministic block sample stratified by size: the blocks in
    decreasing order of rows * cols (ties by depth-first index) are cut into
    strata of k = ceil(nblocks / per_sample) consecutive blocks, the members
    of every stratum are put in a seeded random order, and sample `offset`
    takes member `offset` of every stratum.  Every sample then has the
    workload's size mix, each block is equally likely to be in it, and
    offsets 0..k-1 give disjoint samples."""
    nb = len(blocks)
    sz = (blocks[:, 1] - blocks[:, 0]).astype(np.int64) * (blocks[:, 3] - blocks[:, 2])
    order = np.lexsort((np.arange(nb), -sz))
    k = max(1, -(-nb // max(1, per_sample)))
    rng = np.random.default_rng(seed)
    mask = np.zeros(nb, dtype=bool)
    for a in range(0, nb, k):
        stratum = order[a:a + k]
        mask[stratum[rng.permutation(len(stratum))[offset % len(stratum)]]] = True
    return mask, k


def oracle_baseline(cfg, problem=None, per_sample=24, offset=0):
    """Oracle 3D-ACA compression (FP64, OpenMP over blocks) of a stratified
    block sample of the workload (oracle_sample_mask), timed on the host
    cores block by block.  Cost model: the blocks are independent and the
    whole workload (thousands of blocks) spreads over the host cores, so its
    rate is cores x (entries evaluated / summed single-block seconds); value
    is that rate in entries evaluated per second (the unit of the GPU line).
    The wall-clock rate of the sample itself is reported beside it (a small
    sample leaves cores idle behind its largest block)."""
    import oracle as orc
    m, su, tr, op = problem or oracle_problem(cfg)
    mask, k = oracle_sample_mask(tr.blocks, per_sample, offset)
    t0 = time.perf_counter()
    X = orc.Tensor(m, op, su, tr, cfg["eps"], cfg["eps_aca"], c=cfg["c"], ng=cfg["ng"], block_mask=mask)
    wall = time.perf_counter() - t0
    ev, secs = X.stats["evals"], X.stats["block_seconds"]
    cores = os.cpu_count()
    return {"value": cores * ev / secs, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "sample": "oracle 3D-ACA compression (FP64, OpenMP over blocks) of %d of the workload's %d blocks "
                      "(stratified by size: one block of each run of %d in size order, sample %d), %.3e entries "
                      "evaluated in %.1f s summed over the blocks (%.1f s wall); value = cores x entries / summed "
                      "block seconds (independent blocks spread over the cores)" % (
                          int(mask.sum()), len(mask), k, offset, ev, secs, wall),
            "evals": ev, "block_seconds": secs, "wall_seconds": wall, "wall_value": ev / wall}


def run_reference(args, cfg, wl_name):
    """The oracle as the reference arm: step j compresses the j-th of the
    disjoint stratified block samples (oracle_sample_mask); value = cores x
    entries evaluated / summed block seconds over the timed steps."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    prob = oracle_problem(cfg)
    ev = secs = wall = 0.0
    info = None
    for k in range(args.warmup + args.steps):
        info = oracle_baseline(cfg, problem=prob, per_sample=args.ref_blocks, offset=k)
        if k >= args.warmup:
            ev += info["evals"]
            secs += info["block_seconds"]
            wall += info["wall_seconds"]
    v = info["cores"] * ev / secs
    sample = ("oracle 3D-ACA compression (FP64, OpenMP over blocks), one stratified sample of about %d blocks per "
              "step (disjoint samples), %.3e entries evaluated in %.1f s summed over the blocks of the timed steps "
              "(%.1f s wall); value = cores x entries / summed block seconds" % (args.ref_blocks, ev, secs, wall))
    line = {"impl": "reference", "metric": "entries/s", "value": v, "unit": "entries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": wl_name},
            "ms_per_step": 1e3 * wall / args.steps, "wall_value": ev / wall,
            "cpu_baseline": {"value": v, "unit": "entries/s", "cores": info["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="housing30k_slp_gcq256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--ref-blocks", type=int, default=24, help="blocks per oracle sample (each step of "
                    "--impl reference; twice as many for cpu_baseline)")
    ap.add_argument("--no-predictor", action="store_true", help="time the form without the rank predictor")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-recompress", action="store_true", help="skip the QR + SVD recompression measurement")
    args = ap.parse_args()
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg, args.workload)

    import torch
    import paper_2505_00715_gb300 as td

    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_base = oracle_baseline(cfg, per_sample=2 * args.ref_blocks)  # host cores, before any timed GPU work

    ctx = td.Context(local)
    stream = ctx.stream
    # roofline denominators of the compression's pipes, measured on this GPU
    # before any timed work (special-function unit, FP32 and FP64 FMA)
    pipe_peaks = {k: ctx.measure_peak(k) for k in ("sfu", "fma32", "fma64", "pair64")}
    V, T = workload_mesh(cfg)
    mesh = td.Mesh(ctx, V, T)
    freqs = workload_freqs(td, ctx, cfg)
    cfg = dict(cfg, Nu=freqs.Nu)
    op = getattr(td, cfg["op"])
    colb = td.P1 if cfg["op"] == "DLP" else td.P0
    nrows, ncols = mesh.ndof(td.P0), mesh.ndof(colb)
    NQ = freqs.NQ
    nrhs = cfg["nrhs"]
    W_host = random_weights(NQ, ncols, nrhs, seed=1)
    W = torch.as_tensor(W_host, dtype=torch.complex64, device=dev)
    y = torch.empty((nrows, nrhs), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    # rank predictor: trained on the GPU (untimed) from the plain method's own
    # face ranks on smaller spheres (320 and 1280 triangles, SLP and DLP)
    if args.no_predictor:
        model, pinfo = None, {"disabled": True}
    else:
        model, pinfo = train_predictor(td, ctx, cfg, dev)
    tuned = None
    if not args.no_autotune:
        # project autotuner: launch shape of the persistent far-field phase (untimed)
        tr0 = td.Tree(mesh, td.P0, colb, cfg["leaf"], cfg["eta"])
        tuned = td.autotune(mesh, op, freqs, tr0, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=td.MIXED, c=cfg["c"],
                            ng=cfg["ng"], model=model)
        if not args.no_fp64 and "level" in cfg:
            # (on the housings one FP64 compression takes tens of seconds: the
            # FP64 form keeps the default launch shape there)
            td.autotune(mesh, op, freqs, tr0, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=td.FP64, c=cfg["c"],
                        ng=cfg["ng"])

    def step(prec=td.MIXED, Wd=W, yd=y, use_model=True):
        tree = td.Tree(mesh, td.P0, colb, cfg["leaf"], cfg["eta"])
        X = td.compress(mesh, op, freqs, tree, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=prec, c=cfg["c"],
                        ng=cfg["ng"], model=model if use_model else None)
        e_apply0 = torch.cuda.Event(enable_timing=True)
        e_apply1 = torch.cuda.Event(enable_timing=True)
        e_apply0.record(stream)
        X.apply_weighted(Wd, yd)
        e_apply1.record(stream)
        return X, (e_apply0, e_apply1)

    def timed(n, prec=td.MIXED, Wd=W, yd=y, use_model=True):
        # keeps the last step's tensor only (a housing tensor holds tens of GB)
        out = []
        X = None
        for i in range(n):
            if out:
                out[-1] = out[-1][:3] + (None,)
            X = None
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            X, (a0, a1) = step(prec, Wd, yd, use_model)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append((e0.elapsed_time(e1), a0.elapsed_time(a1), X.stats(), X))
        return out

    for _ in range(args.warmup):
        timed(1)
    with ClockSampler(local) as clk:
        res = timed(args.steps)
    ms = [r[0] for r in res]
    st = res[-1][2]
    X = res[-1][3]
    # first apply of a fresh tensor (inside the step: builds the apply plan)
    # and the steady-state apply of the same tensor (plan built, L2 flushed)
    apply_first_ms = statistics.median([r[1] for r in res])
    apply_ms = steady_apply_ms(res[-1][3], W, y, flush, stream)
    represented = float(nrows) * ncols * NQ
    # units of a step: the operator entries its compression evaluated
    evaluated = statistics.mean([float(r[2]["entries_regular"] + r[2]["entries_tube"]) for r in res])
    value, total_ms = job_throughput(sum(ms), evaluated, args.steps, world, dist)
    blocks = X.partition()
    apply_gflops = apply_flops(X, blocks, NQ, nrhs) / (apply_ms / 1e3) / 1e9
    # QR + SVD recompression of the last tensor's far faces (Sec. 4, H-matrix
    # variant) at eps_aca: time, storage and the apply afterwards (untimed step)
    recompression = None
    if not args.no_recompress:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        X.recompress(cfg["eps_aca"])
        e1.record(stream)
        torch.cuda.synchronize()
        st_rc = X.stats()
        for _ in range(2):
            X.apply_weighted(W, y)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        a0.record(stream)
        X.apply_weighted(W, y)
        a1.record(stream)
        torch.cuda.synchronize()
        recompression = {"eps": cfg["eps_aca"], "ms": e0.elapsed_time(e1),
                         "stored_complex_before": st["stored_complex"], "stored_complex_after": st_rc["stored_complex"],
                         "sum_face_rank_before": st["sum_face_rank"], "sum_face_rank_after": st_rc["sum_face_rank"],
                         "apply_ms_after": a0.elapsed_time(a1)}
    X = None
    res = [r[:3] for r in res]

    # same step without the predictor, and the plain FP64 GPU form
    r_np = timed(2, use_model=False)
    no_pred = {"step_ms": statistics.median([r[0] for r in r_np]),
               "time_to_tensor_s": statistics.median([r[2]["ms_total"] for r in r_np]) / 1e3,
               "phase_ms": {k: r_np[-1][2][k] for k in ("ms_plan", "ms_singular", "ms_near", "ms_far")},
               "aca_tests": r_np[-1][2]["aca_tests"], "pool_first_values": r_np[-1][2]["pool_first"]}
    del r_np
    fp64 = None
    if not args.no_fp64:
        W64 = torch.as_tensor(W_host, dtype=torch.complex128, device=dev)
        y64 = torch.empty((nrows, nrhs), dtype=torch.complex128, device=dev)
        if "level" in cfg:
            timed(1, td.FP64, W64, y64, use_model=False)  # warm-up where a step is short
        r64 = timed(1, td.FP64, W64, y64, use_model=False)
        s64 = r64[0][2]
        X64 = r64[0][3]
        fp64 = {"step_ms": r64[0][0], "time_to_tensor_s": s64["ms_total"] / 1e3,
                "apply_ms": r64[0][1], "apply_gflops": apply_flops(X64, X64.partition(), NQ, nrhs) / (r64[0][1] / 1e3) / 1e9,
                "entries_per_s": (s64["entries_regular"] + s64["entries_tube"]) / (r64[0][0] / 1e3),
                "dense_equivalent_entries_per_s": represented / (r64[0][0] / 1e3),
                "roofline": roofline_fp64(s64, cfg, X64.partition(), pipe_peaks),
                "apply_roofline": apply_roofline(s64, cfg, NQ, ncols, nrows, nrhs, r64[0][1], 16),
                "phase_ms": {k: s64[k] for k in ("ms_plan", "ms_singular", "ms_near", "ms_far")},
                "sum_rank": s64["sum_rank"], "stored_complex": s64["stored_complex"]}
        del X64, W64, y64, r64

    # e2e through the host-buffer API
    yh = torch.empty((nrows, nrhs), dtype=torch.complex64).pin_memory()
    Wh = torch.as_tensor(W_host.astype(np.complex64)).pin_memory()
    e2e_ms = []
    for k in range(max(1, min(3, args.steps)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = td.Mesh(ctx, V, T)
        tr2 = td.Tree(m2, td.P0, colb, cfg["leaf"], cfg["eta"])
        X2 = td.compress(m2, op, freqs, tr2, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=td.MIXED, c=cfg["c"],
                         ng=cfg["ng"], model=model)
        X2.apply_weighted_host(Wh, yh)
        dt = (time.perf_counter() - t0) * 1e3
        if k > 0:
            e2e_ms.append(dt)
        del X2, tr2, m2
    e2e_med = statistics.median(e2e_ms)
    e2e = {"value": world * evaluated / (e2e_med / 1e3), "unit": "entries/s",
           "h2d_bytes_per_step": int(V.nbytes + T.nbytes + Wh.numel() * 8),
           "d2h_bytes_per_step": int(yh.numel() * 8), "ms_per_step": e2e_med}

    peaks, peak_kind = load_peaks()
    apply_roof = apply_roofline(st, cfg, NQ, ncols, nrows, nrhs, apply_ms, 8)
    clocks = clk.summary()
    roof = roofline(st, cfg, blocks, peaks, peak_kind, clocks, args.workload, pipe_peaks)
    if rank == 0:
        line = {
            "metric": "entries/s", "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "triangles": int(nrows), "cols": int(ncols), "N_Q": int(NQ),
                       "unique_freqs": int(freqs.Nu), "leaf": cfg["leaf"], "eta": cfg["eta"], "eps": cfg["eps"],
                       "eps_aca": cfg["eps_aca"], "ng": cfg["ng"], "nrhs": nrhs,
                       "form": "mixed" + ("" if model is None else " + rank predictor"),
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_tensor_s": st["ms_total"] / 1e3,
            "entries_evaluated_per_step": evaluated,
            "dense_equivalent_entries_per_s": world * represented * args.steps / (total_ms / 1e3),
            "phase_ms": {k: st[k] for k in ("ms_plan", "ms_singular", "ms_near", "ms_far")},
            "apply_ms": apply_ms, "apply_first_ms": apply_first_ms, "apply_gflops": apply_gflops,
            # the apply against HBM: algorithmic bytes = the compressed tensor read once
            # (faces and fibres) + W read once + y written once
            "apply_roofline": apply_roof,
            # entries the compression evaluated, by kind: regular FP32 entries (near tensor
            # and far fibres), frequency tubes at the pivots, touching pairs (FP64 geometry)
            # integrated per unique frequency
            "entries_evaluated": {"regular_fp32": st["entries_regular"], "tube_fp32": st["entries_tube"],
                                  "touching_pair_frequencies": st["pairs_singular"]},
            "compression": {"stored_complex": st["stored_complex"], "dense_complex": st["dense_complex"],
                            "rate": st["stored_complex"] / st["dense_complex"], "sum_rank": st["sum_rank"],
                            "max_rank": st["max_rank"], "nblocks": st["nblocks"], "nfar": st["nfar"],
                            "sum_face_rank": st["sum_face_rank"], "pool_growths": st["pool_growths"],
                            "aca_tests": st["aca_tests"]},
            "predictor": dict(pinfo, pool_first_values=st["pool_first"], without=no_pred),
            "autotuned": tuned and {"far_threads_per_cta": tuned[0], "far_ctas_per_sm": tuned[1],
                                    "touching_pair_freqs_per_pass": tuned[2], "near_freqs_per_pass": tuned[3]},
            "recompression": recompression,
            "fp64_form": fp64,
            "e2e": e2e,
            "roofline": roof,
            "clocks": clocks,
            # per timed step: the compression's kernels (touching table, near entries and
            # near 3D-ACA per batch, far 3D-ACA) and the apply's three (GEMM, T, y)
            "gpu_launches": int(sum(r[2]["launches"] + 3 for r in res)),
            "cpu_baseline": cpu_base and {k: cpu_base[k] for k in ("value", "unit", "cores", "kind", "sample")},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


BIN_EDGES = np.array([1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64])


def harvest_training_set(td, ctx, dev, levels=(3, 4, 5)):
    """(far block, frequency, face-ACA rank bin) samples from the plain
    method's own compressions of the sphere configurations: icospheres of the
    given levels (1280 / 5120 / 20480 triangles), single layer P0 x P0 and
    double layer P0 x P1, BDF2 frequency sets N = 64, dt = 0.05 and N = 16,
    dt = 0.1 (c = 1, leaf 32, eta 2, face ACA at 1e-6)."""
    import torch
    xs, ys = [], []
    for lev in levels:
        V, T = icosphere(lev)
        m = td.Mesh(ctx, V, T)
        for N, dt in ((64, 0.05), (16, 0.1)):
            f = td.Freqs.bdf2(ctx, N, dt)
            for op, cb in ((td.SLP, td.P0), (td.DLP, td.P1)):
                tr = td.Tree(m, td.P0, cb, 32, 2.0)
                x, r = td.harvest(m, op, f, tr, eps_aca=1e-6, c=1.0, ng=5)
                xs.append(x)
                ys.append(torch.as_tensor(np.searchsorted(BIN_EDGES, r.cpu().numpy()).astype(np.int32), device=dev))
    return torch.cat(xs), torch.cat(ys)


def predictor_accuracy(td, model, mesh, op, freqs, tree, cfg):
    """Bin accuracy of the model on a workload (its own plain face ranks)."""
    xw, rw = td.harvest(mesh, op, freqs, tree, eps_aca=cfg["eps_aca"], c=cfg["c"], ng=cfg["ng"])
    yw = np.searchsorted(BIN_EDGES, rw.cpu().numpy())
    pw = model.predict(xw).cpu().numpy()
    return {"samples": int(len(yw)), "bin_accuracy": float(np.mean(pw == yw)),
            "within_one_bin": float(np.mean(np.abs(pw - yw) <= 1)), "under_predicted": float(np.mean(pw < yw)),
            "majority_bin_share": float(np.max(np.bincount(yw, minlength=16)) / max(1, len(yw)))}


def train_predictor(td, ctx, cfg, dev):
    t0 = time.perf_counter()
    x, y = harvest_training_set(td, ctx, dev)
    model = td.Model(ctx, seed=2)
    loss = model.train(x, y, epochs=8, batch=4096, lr=3e-3, seed=3)
    t_train = time.perf_counter() - t0
    # accuracy on the benchmark workload itself (unseen mesh, frequencies and wave speed)
    V, T = workload_mesh(cfg)
    m = td.Mesh(ctx, V, T)
    f = workload_freqs(td, ctx, cfg)
    tr = td.Tree(m, td.P0, td.P1 if cfg["op"] == "DLP" else td.P0, cfg["leaf"], cfg["eta"])
    acc = predictor_accuracy(td, model, m, getattr(td, cfg["op"]), f, tr, cfg)
    return model, dict({"train_samples": int(len(y)), "train_loss": loss, "train_seconds": t_train,
                        "train_set": "icospheres 1280/5120/20480 triangles, SLP P0xP0 and DLP P0xP1, BDF2 N=64 "
                                     "dt=0.05 and N=16 dt=0.1, c=1: every (far block, unique frequency) face",
                        "note": "under_predicted = share of (far block, frequency) faces whose ACA continues "
                                "adaptively past the predicted first trip count"}, **acc)


def steady_apply_ms(X, W, y, flush, stream, reps=3):
    """Median of `reps` weighted applies of a tensor whose apply plan is built,
    the L2 flushed before each."""
    import torch
    X.apply_weighted(W, y)
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        X.apply_weighted(W, y)
        a1.record(stream)
        torch.cuda.synchronize()
        ts.append(a0.elapsed_time(a1))
    return statistics.median(ts)


def apply_roofline(st, cfg, NQ, ncols, nrows, nrhs, apply_ms, es):
    """The weighted apply against HBM: algorithmic bytes = the compressed
    tensor read once (faces and fibres) + W read once + y written once, es
    bytes per complex value."""
    peaks, kind = load_peaks()
    nbytes = float(es) * (st["stored_complex"] + float(NQ) * ncols * nrhs + float(nrows) * nrhs)
    gbs = nbytes / (apply_ms / 1e3) / 1e9
    return {"bound": "hbm", "unit": "GB/s", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
            "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None, "algorithmic_bytes": nbytes,
            "peak_source": kind + (" (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else "")}


def roofline_fp64(st, cfg, blocks, pipe_peaks):
    """Far phase of the plain FP64 form against the FP64 point-pair rate
    measured on this GPU (tdbem_measure_peak, the same operation on
    independent chains on every SM): its entries are 49 point pairs each
    (SLP; 6 x 49 per P1 column of the double layer)."""
    nI = (blocks[:, 1] - blocks[:, 0]).astype(np.int64)
    nJ = (blocks[:, 3] - blocks[:, 2]).astype(np.int64)
    near_entries = int(np.sum((nI * nJ)[blocks[:, 4] == 0])) * int(cfg["Nu"])
    ppe = 49 * 6 if cfg["op"] == "DLP" else 49
    pairs = (st["entries_regular"] - near_entries + st["entries_tube"]) * ppe
    ach = pairs / (st["ms_far"] / 1e3)
    peak = pipe_peaks.get("pair64") if pipe_peaks else None
    return {"bound": "alu", "kernel": "far 3D-ACA (k_far_aca, FP64)", "unit": "point pairs/s", "achieved": ach,
            "peak": peak, "frac": ach / peak if peak else None,
            "work": "%.3e point pairs in %.1f ms" % (pairs, st["ms_far"]),
            "peak_source": "measured: tdbem_measure_peak FP64 point-pair microbenchmark"}


def apply_flops(X, blocks, NQ, nrhs):
    """Algorithmic flops of eq. product: frequency contraction 8 NQ |J| nrhs per
    term, face products 8 nrhs per stored face entry, twice (conjugate half)."""
    r_b, k_b, _ = X.blocks()
    nI = (blocks[:, 1] - blocks[:, 0]).astype(np.float64)
    nJ = (blocks[:, 3] - blocks[:, 2]).astype(np.float64)
    far = blocks[:, 4] == 1
    flops_a = np.sum(r_b * nJ) * 8.0 * NQ * nrhs
    face_entries = np.sum(np.where(far, k_b * (nI + nJ), r_b * nI * nJ))
    return flops_a + face_entries * 8.0 * nrhs * 2.0


# DRAM bytes (read + write) of one far-kernel launch on the benchmark workload
# (the 30k-triangle housing, default launch shape), from a one-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, -k k_far_aca -c 1) of
# the kernel built from the sources whose digest is recorded; reported only
# while those sources are unchanged.
FAR_TRAFFIC = {"workload": "housing30k_slp_gcq256", "bytes": 1.16e12 + 92.45e9,
               "sources": ("k_aca.cu", "pair.cuh", "common.cuh"), "sha256_16": "93adeb8434f14377"}


def far_traffic(workload):
    import hashlib
    if workload != FAR_TRAFFIC["workload"]:
        return None
    h = hashlib.sha256()
    for f in FAR_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2505_00715_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return FAR_TRAFFIC["bytes"] if h.hexdigest()[:16] == FAR_TRAFFIC["sha256_16"] else None


def roofline(st, cfg, blocks, peaks, peak_kind, clocks, workload=None, pipe_peaks=None):
    """Dominant phase of the compression against its ALU roofline.

    Far-field 3D-ACA kernel: its algorithmic work is the entry generation,
    point-pair evaluations (49 per P0 x P0 entry) of which each needs four
    special-function-unit operations (rsqrt, exp2, sin, cos); peak = the
    special-function throughput measured on this GPU by tdbem_measure_peak
    (the same four operations), else 16 per clock per SM x 152 SMs x the
    sampled SM clock.  The fraction shows how far the kernel is from being
    bound by its entry arithmetic (the rest is ACA bookkeeping and latency)."""
    phases = {"singular": st["ms_singular"], "near": st["ms_near"], "far": st["ms_far"]}
    dom = max(phases, key=phases.get)
    clock_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if pipe_peaks and pipe_peaks.get("sfu"):
        sfu_peak = pipe_peaks["sfu"] / 1e12  # T SFU-ops/s, measured
        peak_source = "measured: tdbem_measure_peak special-function microbenchmark (rsqrt, ex2, sin, cos)"
    else:
        sfu_peak = 16.0 * 152 * clock_mhz * 1e6 / 1e12
        peak_source = "derived: 16 SFU ops/clk/SM x 152 SMs x %.0f MHz (sampled median)" % clock_mhz
    nI = (blocks[:, 1] - blocks[:, 0]).astype(np.int64)
    nJ = (blocks[:, 3] - blocks[:, 2]).astype(np.int64)
    near_entries = int(np.sum((nI * nJ)[blocks[:, 4] == 0])) * int(cfg["Nu"])
    pairs_per_entry = 49 * 6 if cfg["op"] == "DLP" else 49
    far_pairs = (st["entries_regular"] - near_entries + st["entries_tube"]) * pairs_per_entry
    achieved_far = far_pairs * 4.0 / (st["ms_far"] / 1e3) / 1e12
    out = {"bound": "alu", "kernel": "far 3D-ACA (k_far_aca)" if dom == "far" else dom, "unit": "TSFU-op/s",
           "achieved": achieved_far, "peak": sfu_peak, "frac": achieved_far / sfu_peak, "traffic": far_traffic(workload),
           "traffic_unit": "bytes per far launch (DRAM read + write, ncu)",
           "work": "%.3e point pairs x 4 SFU ops in %.1f ms" % (far_pairs, st["ms_far"]),
           "peak_source": peak_source,
           "measured_pipe_peaks_per_s": pipe_peaks,
           "phase_ms": phases, "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": peak_kind}
    if dom != "far":
        out["note"] = "dominant phase is %s; the far-kernel figures are reported for comparison" % dom
    return out


if __name__ == "__main__":
    sys.exit(main())
