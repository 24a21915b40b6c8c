"""Benchmark of the GB300 3D-ACA tensor path (one JSON line on rank 0).

Workload (default, the 5120-triangle configuration): icosphere R = 1 with
5120 flat triangles, Galerkin single layer P0 x P0, wave speed 1, BDF2
convolution quadrature N = 64, dt = 0.05 (33 unique frequencies), PCA cluster
tree with leaf size 32 and eta = 2, 3D-ACA at eps = 1e-4 (face ACA 1e-6),
Sauter-Schwab with 5 Gauss points per variable; apply with 16 right-hand sides.

One step = the whole path: block cluster tree, compression (touching-pair
table, near-field entries, near and far 3D-ACA, one graph) and one
multi-frequency apply.  Metric: dense-equivalent tensor entries per second,
rows * cols * N_Q / step time.  Inputs are resident in HBM before the timed
region; the e2e figure repeats the step through the host-buffer API (mesh
upload, tree, compression, apply with host W and y).

--impl reference times the FP64 CPU oracle (the reference arm of this
comparison) on a bounded sample of the same workload.
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

from paper_2505_00715_gb300.inputs import icosphere, random_weights  # noqa: E402

WORKLOADS = {
    "sphere5120_slp_bdf2_N64": dict(level=4, op="SLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                    ng=5, nrhs=16, c=1.0),
    "sphere5120_dlp_bdf2_N64": dict(level=4, op="DLP", N=64, dt=0.05, leaf=32, eta=2.0, eps=1e-4, eps_aca=1e-6,
                                    ng=5, nrhs=16, c=1.0),
}


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


def oracle_baseline(cfg, target_s=15.0, max_stride=None):
    """Oracle compression of every stride-th block of the workload, timed on
    the host cores; returns dense-equivalent entries/s of the sampled blocks."""
    import oracle as orc
    V, T = icosphere(cfg["level"])
    m = orc.Mesh(V, T)
    s = orc.freqs_bdf2(cfg["N"], cfg["dt"])
    Nu = cfg["N"] // 2 + 1
    cols = 0 if cfg["op"] == "SLP" else 1
    tr = orc.Tree(m, 0, cols, cfg["leaf"], cfg["eta"])
    blocks = tr.blocks
    nb = len(blocks)
    op = getattr(orc, cfg["op"])
    # pilot: a sparse sample to estimate the cost per represented entry
    stride = max_stride or max(1, nb // 40)
    t0 = time.perf_counter()
    orc.Tensor(m, op, s[:Nu], tr, cfg["eps"], cfg["eps_aca"], c=cfg["c"], ng=cfg["ng"], block_stride=stride)
    t1 = time.perf_counter() - t0
    if t1 < target_s / 4 and stride > 1:
        stride = max(1, int(stride * t1 / target_s * 2))
        t0 = time.perf_counter()
        orc.Tensor(m, op, s[:Nu], tr, cfg["eps"], cfg["eps_aca"], c=cfg["c"], ng=cfg["ng"], block_stride=stride)
        t1 = time.perf_counter() - t0
    sel = blocks[np.arange(nb) % stride == 0]
    rep = float(np.sum((sel[:, 1] - sel[:, 0]).astype(np.int64) * (sel[:, 3] - sel[:, 2]))) * cfg["N"]
    return {"value": rep / t1, "unit": "entries/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle 3D-ACA compression (FP64, OpenMP over blocks) of every %d-th block (%d of %d blocks) "
                      "of the same workload, %.1f s; value = sampled blocks' rows*cols*N_Q / time" % (
                          stride, len(sel), nb, t1),
            "seconds": t1}


def run_reference(args, cfg, wl_name):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        info = oracle_baseline(cfg, target_s=args.ref_seconds)
        if k >= args.warmup:
            vals.append(info["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "entries/s", "value": v, "unit": "entries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": wl_name},
            "cpu_baseline": {"value": v, "unit": "entries/s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": v, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere5120_slp_bdf2_N64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
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
        cpu_base = oracle_baseline(cfg)  # host cores, before any timed GPU work

    ctx = td.Context(local)
    stream = ctx.stream
    V, T = icosphere(cfg["level"])
    mesh = td.Mesh(ctx, V, T)
    freqs = td.Freqs.bdf2(ctx, cfg["N"], cfg["dt"])
    op = getattr(td, cfg["op"])
    colb = td.P0 if cfg["op"] == "SLP" else td.P1
    nrows, ncols = mesh.ndof(td.P0), mesh.ndof(colb)
    NQ = freqs.NQ
    W_host = random_weights(NQ, ncols, cfg["nrhs"], seed=1)
    W = torch.as_tensor(W_host, dtype=torch.complex64, device=dev)
    y = torch.empty((nrows, cfg["nrhs"]), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def step(prec=td.MIXED, Wd=W, yd=y):
        tree = td.Tree(mesh, td.P0, colb, cfg["leaf"], cfg["eta"])
        X = td.compress(mesh, op, freqs, tree, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=prec, c=cfg["c"],
                        ng=cfg["ng"])
        e_apply0 = torch.cuda.Event(enable_timing=True)
        e_apply1 = torch.cuda.Event(enable_timing=True)
        e_apply0.record(stream)
        X.apply_weighted(Wd, yd)
        e_apply1.record(stream)
        return X, (e_apply0, e_apply1)

    def timed(n, prec=td.MIXED, Wd=W, yd=y):
        out = []
        for _ in range(n):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            X, (a0, a1) = step(prec, Wd, yd)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append((e0.elapsed_time(e1), a0.elapsed_time(a1), X.stats(), X))
        return out

    for _ in range(args.warmup):
        timed(1)
    with ClockSampler(local) as clk:
        res = timed(args.steps)
    ms = [r[0] for r in res]
    total_ms = sum(ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    st = res[-1][2]
    X = res[-1][3]
    apply_ms = statistics.median([r[1] for r in res])
    represented = float(nrows) * ncols * NQ
    value = world * represented * args.steps / (total_ms / 1e3)

    # apply flops (algorithmic, eq. product): frequency contraction 8*NQ*|J|*nrhs per
    # term, face products 8*nrhs per stored face entry, times 2 for the conjugate half
    r_b, k_b, _ = X.blocks()
    blocks = X.tree.blocks
    nI = (blocks[:, 1] - blocks[:, 0]).astype(np.float64)
    nJ = (blocks[:, 3] - blocks[:, 2]).astype(np.float64)
    far = blocks[:, 4] == 1
    nrhs = cfg["nrhs"]
    flops_a = np.sum(r_b * nJ) * 8.0 * NQ * nrhs
    face_entries = np.sum(np.where(far, k_b * (nI + nJ), r_b * nI * nJ))
    flops_b = face_entries * 8.0 * nrhs * 2.0
    apply_gflops = (flops_a + flops_b) / (apply_ms / 1e3) / 1e9

    # plain FP64 GPU form (same algorithm, all FP64)
    fp64 = None
    if not args.no_fp64:
        W64 = torch.as_tensor(W_host, dtype=torch.complex128, device=dev)
        y64 = torch.empty((nrows, nrhs), dtype=torch.complex128, device=dev)
        timed(1, td.FP64, W64, y64)
        r64 = timed(1, td.FP64, W64, y64)
        s64 = r64[0][2]
        X64 = r64[0][3]
        rb64, kb64, _ = X64.blocks()
        fa64 = np.sum(rb64 * nJ) * 8.0 * NQ * nrhs
        fb64 = np.sum(np.where(far, kb64 * (nI + nJ), rb64 * nI * nJ)) * 8.0 * nrhs * 2.0
        fp64 = {"step_ms": r64[0][0], "time_to_tensor_s": s64["ms_total"] / 1e3,
                "apply_ms": r64[0][1], "apply_gflops": (fa64 + fb64) / (r64[0][1] / 1e3) / 1e9,
                "entries_per_s": represented / (r64[0][0] / 1e3),
                "phase_ms": {k: s64[k] for k in ("ms_plan", "ms_singular", "ms_near", "ms_far")},
                "sum_rank": s64["sum_rank"], "stored_complex": s64["stored_complex"]}
        del X64, W64, y64

    # e2e through the host-buffer API
    e2e = None
    yh = torch.empty((nrows, nrhs), dtype=torch.complex64).pin_memory()
    Wh = torch.as_tensor(W_host.astype(np.complex64)).pin_memory()
    e2e_ms = []
    for k in range(max(1, min(3, args.steps)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = td.Mesh(ctx, V, T)
        tr2 = td.Tree(m2, td.P0, colb, cfg["leaf"], cfg["eta"])
        X2 = td.compress(m2, op, freqs, tr2, eps=cfg["eps"], eps_aca=cfg["eps_aca"], prec=td.MIXED, c=cfg["c"],
                         ng=cfg["ng"])
        X2.apply_weighted_host(Wh, yh)
        dt = (time.perf_counter() - t0) * 1e3
        if k > 0:
            e2e_ms.append(dt)
        del X2, tr2, m2
    e2e_med = statistics.median(e2e_ms)
    e2e = {"value": world * represented / (e2e_med / 1e3), "unit": "entries/s",
           "h2d_bytes_per_step": int(V.nbytes + T.nbytes + Wh.numel() * 8),
           "d2h_bytes_per_step": int(yh.numel() * 8), "ms_per_step": e2e_med}

    peaks, peak_kind = load_peaks()
    roof = roofline(st, cfg, peaks, peak_kind, clk.summary())
    if rank == 0:
        line = {
            "metric": "entries/s", "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "triangles": int(nrows), "cols": int(ncols), "N_Q": int(NQ),
                       "unique_freqs": int(freqs.Nu), "leaf": cfg["leaf"], "eta": cfg["eta"], "eps": cfg["eps"],
                       "eps_aca": cfg["eps_aca"], "ng": cfg["ng"], "nrhs": nrhs,
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_tensor_s": st["ms_total"] / 1e3,
            "phase_ms": {k: st[k] for k in ("ms_plan", "ms_singular", "ms_near", "ms_far")},
            "apply_ms": apply_ms, "apply_gflops": apply_gflops,
            "entries_evaluated_per_s": (st["entries_regular"] + st["entries_tube"]) / (st["ms_total"] / 1e3),
            "compression": {"stored_complex": st["stored_complex"], "dense_complex": st["dense_complex"],
                            "rate": st["stored_complex"] / st["dense_complex"], "sum_rank": st["sum_rank"],
                            "max_rank": st["max_rank"], "nblocks": st["nblocks"], "nfar": st["nfar"]},
            "fp64_form": fp64,
            "e2e": e2e,
            "roofline": roof,
            "clocks": clk.summary(),
            "gpu_launches": 5 * args.steps,
            "cpu_baseline": cpu_base and {k: cpu_base[k] for k in ("value", "unit", "cores", "kind", "sample")},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def roofline(st, cfg, peaks, peak_kind, clocks):
    """Dominant phase of the compression against its ALU peak (placeholder
    model refined with the ncu profile)."""
    phases = {"singular": st["ms_singular"], "near": st["ms_near"], "far": st["ms_far"]}
    dom = max(phases, key=phases.get)
    return {"bound": "alu", "kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "phase_ms": phases, "peak_source": peak_kind}


if __name__ == "__main__":
    sys.exit(main())
