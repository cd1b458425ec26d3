"""Benchmark: H^2 single-layer matvec on the 2,097,152-triangle unit sphere.

One step = one h2bem_apply (every stage of the H^2 product: permutation,
leaf forward transform, upward pass, coupling with on-the-fly S_ts, downward
pass, leaf backward transform, on-the-fly nearfield by the 7x7 Gauss rule and
Sauter-Schwab quadrature) on 8 seeded N(0,1) right-hand sides, m = 4, leaf 32,
eta = 2.  Metric: triangles x right-hand sides per second.

Arms
  ours (default)      CUDA path through the C ABI; headline = MIXED_FP32 tier
                      (FP32 farfield, regular-pair and edge/vertex Sauter-Schwab
                      point evaluation; FP64 pair set-up, partial sums and
                      accumulation), with the all-FP64 tier, the cached-singular
                      variants and the relative errors reported.
  --impl reference    the FP64 CPU oracle as it stands on the host cores: the
                      same H^2 operator of the 2,097,152-triangle sphere (m 4,
                      eta 2, leaf 32, 8 right-hand sides), each step the rows
                      of one cluster of tree level 6: their coupling,
                      downward, backward and nearfield, plus their share of
                      the whole tree's leaf forward and upward passes (timed
                      once), so the run takes a few minutes.

Multi-GPU (torchrun): the product does not shard across GPUs here; each rank
runs an independent replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2 SLP matvec triangles/s on 2M-tri sphere, mixed vs FP64, at stated rel. error"
UNIT = "triangles*rhs/s"

# Work units of the kernels.  Every kernel evaluation
# costs one hardware reciprocal square root (the MUFU unit, 16 per clock per
# SM), and the nearfield and coupling kernels are bound by that unit together
# with the FP32 issue slots around it, so their achieved rate is reported as
# kernel evaluations per second against the measured MUFU rate:
#   regular nearfield  49 evaluations per pair the kernel evaluates (regular_evals:
#                      every unordered regular pair once, both orders in diagonal blocks)
#   singular           points per canonical pair: identical 3q, edge-adjacent 5q^2,
#                      vertex-adjacent 2q^3 (FP32 in the mixed tiers, FP64 in the FP64 tier)
#   coupling           k^2 entries of S_ts per farfield block, plus 2 k^2 nrhs FP32 flops
PTS_SING = {0: 15, 1: 125, 2: 250}  # q = 5
# DRAM bytes (read + write) per launch of the regular nearfield kernel on this
# workload, from one ncu capture of the same kernel on the 524,288-triangle
# sphere, scaled by the 4x units (profiles/near_regular_mixed_slp_sphere524k.md)
TRAFFIC = {"near_regular": 4 * (117.23e6 + 17.04e6)}


def peaks():
    """Arithmetic peaks measured live by the microbenchmark csrc/peaks.cu
    (built with the library): FP32/FP64 FMA, FP32 MUFU rsqrt, FP64 MMA.  If it
    cannot run, unit counts x the maximum SM clock (152 SMs, 2070 MHz; FP32 128
    FMA, FP64 2 FMA, MUFU 16 per clock per SM).  HBM and bf16 from
    MEASURED_PEAKS.json when present."""
    p = {"sm": 152, "sm_mhz": 2070.0, "hbm_gbs": 6800.0, "src": "fallback"}
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p["hbm_gbs"] = mp["hbm_gbs"]
        p["sm_mhz"] = mp.get("sm_max_mhz", 2070.0)
        p["src"] = "measured"
    except Exception:
        pass
    clk = p["sm_mhz"] * 1e6
    p["fp32_tflops"] = p["sm"] * 128 * 2 * clk / 1e12
    p["fp64_tflops"] = p["sm"] * 2 * 2 * clk / 1e12
    p["rsqrt_tops"] = p["sm"] * 16 * clk / 1e12
    p["alu_src"] = "unit counts x max SM clock"
    exe = os.path.join(ROOT, "paper_2001_05523_gb300", "_build", "peaks")
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        m = json.loads(r.stdout.strip().splitlines()[-1])
        if r.returncode == 0 and m.get("status") == "no error":
            p["fp32_tflops"] = m["fp32_fma_tflops"]
            p["fp64_tflops"] = m["fp64_fma_tflops"]
            p["rsqrt_tops"] = m["rsqrt_f32_tops"]
            p["fp64_mma_tflops"] = m["fp64_mma_tflops"]
            p["rsqrt_f64_tops"] = m["rsqrt_f64_approx_tops"]
            p["alu_src"] = "measured (csrc/peaks.cu)"
    except Exception:
        pass
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = str(index)
        try:
            import torch

            u = str(torch.cuda.get_device_properties(index).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 5 + i and s[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(v: float, world: int, device) -> float:
    """The largest value over the ranks of the process group (the time of the
    slowest replica); the value itself with one process."""
    if world == 1:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units, over the slowest replica's time (weak scaling)."""
    return world * units_per_rank / seconds


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


SAMPLE_LEVEL = 6  # the host sample: the rows of one cluster of this tree level (about 1/64 of them)


def oracle_sample_setup(s: int, nrhs: int):
    """The oracle's H^2 operator of the benchmark's sphere (set-up, untimed) and
    the sample cluster: the first cluster of tree level SAMPLE_LEVEL in
    depth-first order (child 0 from the root, SAMPLE_LEVEL times)."""
    import oracle
    from paper_2001_05523_gb300 import inputs as I

    oracle.build()
    mesh = I.sphere(s)
    x = I.rhs(mesh.nt, nrhs)
    t0 = time.perf_counter()
    Ho = oracle.H2(mesh, oracle.SLP, m=4, eta=2.0, leaf=32)
    setup_s = time.perf_counter() - t0
    tr = Ho.tree()
    c0 = 0
    for _ in range(SAMPLE_LEVEL):
        if tr["child0"][c0] >= 0:
            c0 = int(tr["child0"][c0])
    rows = int(tr["end"][c0] - tr["begin"][c0])
    return Ho, x, c0, rows, mesh.nt, setup_s, oracle.num_threads()


def cpu_oracle_sample(s: int, nrhs: int, repeats: int):
    """The oracle's per-row cost of the full apply, from the sample: the leaf
    forward transformation and upward pass of the whole tree are timed once
    and charged to the sample rows in proportion (rows / n); the coupling,
    downward, backward and nearfield of the sample rows are timed in full
    (median of `repeats`).  Returns (seconds charged to the sample, rows,
    triangles, threads, set-up seconds, upward seconds, rows seconds)."""
    Ho, x, c0, rows, n, setup_s, cores = oracle_sample_setup(s, nrhs)
    t0 = time.perf_counter()
    xh = Ho.upward(x)
    t_up = time.perf_counter() - t0
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        Ho.matvec_subtree_from(c0, xh, x)
        ts.append(time.perf_counter() - t0)
    t_rows = float(np.median(ts))
    return t_rows + t_up * rows / n, rows, n, cores, setup_s, t_up, t_rows


def sample_text(rows: int, n: int, nrhs: int) -> str:
    return (f"oracle H2 SLP operator of the {n}-triangle sphere (m=4, eta=2, leaf 32, {nrhs} rhs), rows of one "
            f"level-{SAMPLE_LEVEL} cluster ({rows} triangles): coupling, downward, backward and nearfield of those "
            f"rows timed, plus rows/n of the timed leaf forward and upward passes of the whole tree; "
            f"value = rows x rhs / that time")


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    Ho, x, c0, rows, n, setup_s, cores = oracle_sample_setup(args.s, args.nrhs)
    t0 = time.perf_counter()
    xh = Ho.upward(x)
    t_up = time.perf_counter() - t0
    for _ in range(args.warmup):
        Ho.matvec_subtree_from(c0, xh, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ho.matvec_subtree_from(c0, xh, x)
    dt = (time.perf_counter() - t0) / args.steps + t_up * rows / n
    v = rows * args.nrhs / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"sphere_{n}_slp_m4_eta2_leaf32_nrhs{args.nrhs}", "sample_rows": rows,
                   "sample_level": SAMPLE_LEVEL, "setup_s": round(setup_s, 1), "upward_s": round(t_up, 2)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_text(rows, n, args.nrhs)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--s", type=int, default=512, help="sphere subdivisions (n = 8 s^2)")
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 tier")
    ap.add_argument("--tier", default="mixed_fp32", choices=["mixed_fp32", "mixed_tf32", "mixed_bf16"],
                    help="precision tier of the timed step (default mixed_fp32)")
    ap.add_argument("--store-near", action="store_true",
                    help="timed operator with the stored nearfield (opts.store_near): entries evaluated at "
                         "set-up, streamed in every apply")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the headline tier and the FP64 tier only (no variants or other workloads)")
    ap.add_argument("--gca", action="store_true",
                    help="timed operator with Green-cross-approximation bases (opts.basis = GCA; q 4, eps 1e-6)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="opts.autotune of the timed operators: 1 tunes at the first apply (default), "
                         "0 defaults, 2..37 a fixed launch variant (reproducible profiles)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2001_05523_gb300 import build as B

    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2001_05523_gb300 import h2bem as H
    from paper_2001_05523_gb300 import inputs as I

    mesh = I.sphere(args.s)
    n, nrhs = mesh.nt, args.nrhs
    xh_np = I.rhs(n, nrhs)
    x = torch.from_numpy(xh_np).to(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_tier(precision: str, cache: bool, steps: int, kernel: str = "slp", **kw):
        t0 = time.perf_counter()
        # autotune: the first warm-up apply times the launch variants and keeps the fastest
        op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=4, eta=2.0, leaf_size=32,
                        precision=precision, cache_singular=cache, autotune=args.autotune, **kw)
        setup_s = time.perf_counter() - t0
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            H.h2bem_apply(op.op, x, y, stream)
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            # back to back, as a caller applies the operator: the farfield passes run
            # on the operator's second stream concurrently with the nearfield
            H.h2bem_apply(op.op, x, y, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        # stage breakdown: the same number of timed applies, which run every stage
        # on `stream` one after the other and record its events (no host wait)
        e0.record(stream)
        for _ in range(steps):
            H.h2bem_apply_timed(op.op, x, y, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        timed_tier.ms_sequential = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        st = op.stats()  # stage times (CUDA events) of the last timed step
        return op, y.clone(), ms, np.array(st["stage_ms"]), st, setup_s

    results = {}
    with ClockSampler(local) as clk:
        kw_m = {"store_near": True} if args.store_near else {}
        if args.gca:
            kw_m["gca"] = True
        op_m, y_m, ms_m, stage_m, st_m, setup_m = timed_tier(args.tier, False, args.steps, **kw_m)
        ms_m_sequential = timed_tier.ms_sequential
    clocks = clk.summary()
    results["mixed_fp32"] = (ms_m, stage_m)
    # e2e through the public API with pinned host buffers (copies inside the timed region)
    xpin = torch.from_numpy(xh_np).pin_memory()
    ypin = torch.empty_like(xpin).pin_memory()
    H.h2bem_apply(op_m.op, xpin, ypin, stream)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.h2bem_apply(op_m.op, xpin, ypin, stream)  # synchronises the stream before returning
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
    torch.cuda.synchronize(dev)
    op_m.close()

    extra = {}
    if not args.no_fp64:
        op_d, y_d, ms_d, stage_d, st_d, setup_d = timed_tier("fp64", False, max(1, min(args.steps, 3)))
        op_d.close()
        results["fp64"] = (ms_d, stage_d)
        err_m = float(torch.linalg.norm(y_m - y_d) / torch.linalg.norm(y_d))
        extra["fp64"] = {"value": world * n * nrhs / (ms_d / 1e3), "ms_per_step": ms_d,
                         "stage_ms": [round(v, 3) for v in stage_d], "setup_s": round(setup_d, 2)}
        extra["speedup_mixed_vs_fp64"] = ms_d / ms_m
        extra["rel_err_mixed_vs_fp64"] = err_m
    if not args.no_fp64 and not args.no_extras:
        # cached singular entries (x-independent): both tiers
        opc, y_c, ms_c, stage_c, _, _ = timed_tier("mixed_fp32", True, args.steps)
        opc.close()
        extra["mixed_fp32_cached_singular"] = {"value": world * n * nrhs / (ms_c / 1e3), "ms_per_step": ms_c,
                                               "stage_ms": [round(v, 3) for v in stage_c]}
        opdc, _, ms_dc, stage_dc, _, _ = timed_tier("fp64", True, max(1, min(args.steps, 3)))
        opdc.close()
        extra["fp64_cached_singular"] = {"value": world * n * nrhs / (ms_dc / 1e3), "ms_per_step": ms_dc,
                                         "stage_ms": [round(v, 3) for v in stage_dc]}
        extra["speedup_mixed_vs_fp64_cached"] = ms_dc / ms_c
        # stored nearfield: every nearfield entry evaluated once at set-up (FP32 in the mixed
        # tier, FP64 in the FP64 tier) and streamed from HBM in every apply
        pk_h = peaks()["hbm_gbs"]
        stored = {}
        for prec, st_steps in (("mixed_fp32", args.steps), ("fp64", max(1, min(args.steps, 3)))):
            ops, y_s, ms_s, stage_s, st_s, setup_s = timed_tier(prec, False, st_steps, store_near=True)
            ops.close()
            es = 4 if prec == "mixed_fp32" else 8
            # algorithmic bytes of the nearfield stage: every entry once, x in the stored
            # precision, y written in FP64
            alg = st_s["near_pairs"] * es + n * nrhs * (es + 8)
            near_ms = float(stage_s[6])
            stored[prec] = {"value": world * n * nrhs / (ms_s / 1e3), "ms_per_step": ms_s,
                            "stage_ms": [round(v, 3) for v in stage_s], "setup_s": round(setup_s, 2),
                            "near_stored_bytes": st_s["near_stored_bytes"],
                            "near_stage_algorithmic_bytes": alg,
                            "near_stage_gbs": alg / (near_ms / 1e3) / 1e9,
                            "near_stage_frac_of_hbm_peak": alg / (near_ms / 1e3) / 1e9 / pk_h,
                            "rel_err_vs_fp64": float(torch.linalg.norm(y_s - y_d) / torch.linalg.norm(y_d))}
        extra["stored_nearfield"] = stored

    # tensor-core tiers of the coupling (tcgen05): same workload, error against the FP64 tier
    if not args.no_fp64 and not args.no_extras:
        tiers = {}
        for prec in ("mixed_tf32", "mixed_bf16"):
            opt, y_t, ms_t, stage_t, _, _ = timed_tier(prec, False, args.steps)
            opt.close()
            tiers[prec] = {"value": world * n * nrhs / (ms_t / 1e3), "ms_per_step": ms_t,
                           "stage_ms": [round(v, 3) for v in stage_t],
                           "rel_err_vs_fp64": float(torch.linalg.norm(y_t - y_d) / torch.linalg.norm(y_d))}
        extra["tensor_core_tiers"] = tiers
        # mixed tier variants: FP64 Sauter-Schwab points; leaf bases re-evaluated in every apply
        variants = {}
        # singular_fp64_cached: FP64 Sauter-Schwab values evaluated once at set-up and applied in FP64
        # (the placement north of the mixed tier: FP64 singular quadrature and accumulation)
        for name, cache_v, kw in (("singular_fp64", False, {"singular_fp64": True}),
                                  ("singular_fp64_cached", True, {"singular_fp64": True}),
                                  ("recompute_basis", False, {"recompute_basis": True})):
            opv, y_v, ms_v, stage_v, _, _ = timed_tier("mixed_fp32", cache_v, max(1, min(args.steps, 3)), **kw)
            opv.close()
            variants[name] = {"value": world * n * nrhs / (ms_v / 1e3), "ms_per_step": ms_v,
                              "stage_ms": [round(v, 3) for v in stage_v],
                              "rel_err_vs_fp64": float(torch.linalg.norm(y_v - y_d) / torch.linalg.norm(y_d))}
        extra["mixed_fp32_variants"] = variants

        # H^2 error of each tier against exact Galerkin rows (eq. (slp), the oracle's dense
        # rows: 24 seeded rows, all right-hand sides), Chebyshev m = 4 and GCA bases
        import oracle

        oracle.build()
        drows = np.random.default_rng(1).choice(n, 24, replace=False)
        dref = oracle.dense_rows(0, mesh, drows, xh_np)

        def dense_err(y_t):
            yy = y_t.cpu().numpy()[:, drows]
            return float(np.linalg.norm(yy - dref) / np.linalg.norm(dref))

        extra["h2_error_vs_dense_rows"] = {"rows": 24, "chebyshev_m4_fp64": dense_err(y_d),
                                           "chebyshev_m4_mixed": dense_err(y_m)}
        # Green cross approximation bases (section 4; q = 4 Gauss points per face axis,
        # ACA tolerance 1e-6, ranks <= 64): coupling and transfer matrices stored
        gca = {}
        y_g = {}
        for prec, st_steps in (("mixed_fp32", args.steps), ("fp64", max(1, min(args.steps, 3)))):
            opg, y_gp, ms_g, stage_g, st_g, setup_g = timed_tier(prec, False, st_steps, gca=True)
            opg.close()
            y_g[prec] = y_gp
            far_bytes = st_g["far_stored_bytes"]
            gca[prec] = {"value": world * n * nrhs / (ms_g / 1e3), "ms_per_step": ms_g,
                         "stage_ms": [round(v, 3) for v in stage_g], "setup_s": round(setup_g, 2),
                         "mean_rank": st_g["mean_rank"], "far_stored_bytes": far_bytes,
                         "coupling_gbs_of_stored": (far_bytes / (float(stage_g[3]) / 1e3)) / 1e9,
                         "h2_error_vs_dense_rows": dense_err(y_gp)}
        gca["rel_err_mixed_vs_fp64"] = float(torch.linalg.norm(y_g["mixed_fp32"] - y_g["fp64"]) /
                                             torch.linalg.norm(y_g["fp64"]))
        gca["speedup_mixed_vs_fp64"] = gca["fp64"]["ms_per_step"] / gca["mixed_fp32"]["ms_per_step"]
        extra["gca"] = gca
        del y_g
        # double layer K on the same sphere (m = 4): mixed and FP64 tiers, their difference
        dlp = {}
        y_k = {}
        for prec, st_steps in (("mixed_fp32", args.steps), ("fp64", max(1, min(args.steps, 3)))):
            opk, y_kp, ms_k, stage_k, _, setup_k = timed_tier(prec, False, st_steps, kernel="dlp")
            opk.close()
            y_k[prec] = y_kp
            dlp[prec] = {"value": world * n * nrhs / (ms_k / 1e3), "ms_per_step": ms_k,
                         "stage_ms": [round(v, 3) for v in stage_k], "setup_s": round(setup_k, 2)}
        dlp["rel_err_mixed_vs_fp64"] = float(torch.linalg.norm(y_k["mixed_fp32"] - y_k["fp64"]) /
                                             torch.linalg.norm(y_k["fp64"]))
        dlp["speedup_mixed_vs_fp64"] = dlp["fp64"]["ms_per_step"] / dlp["mixed_fp32"]["ms_per_step"]
        kref = oracle.dense_rows(1, mesh, drows, xh_np)
        dlp["h2_error_vs_dense_rows_fp64"] = float(np.linalg.norm(y_k["fp64"].cpu().numpy()[:, drows] - kref) /
                                                   np.linalg.norm(kref))
        extra["dlp"] = dlp
        del y_k

    # other workloads of the benchmark family (reported beside the headline)
    if not args.no_fp64 and not args.no_extras:
        # 64 uneven jittered meshes (sphere / ellipsoid / cube, 2k-65k triangles) as one
        # block-diagonal operator: forward SLP apply and gradients in x and the vertices
        fam = I.batch_meshes(64)
        for prec in ("fp64", "mixed_fp32"):
            Bop = H.BatchOperator(fam, kernel="slp", m=4, eta=2.0, leaf_size=32, precision=prec)
            xb = torch.from_numpy(I.rhs(Bop.n, 1, seed=3)).to(dev)
            wb = torch.from_numpy(I.rhs(Bop.n, 1, seed=4)).to(dev)
            yb = torch.empty_like(xb)
            gX = torch.empty((sum(mm.nv for mm in fam), 3), dtype=torch.float64, device=dev)
            gx = torch.empty_like(xb)
            for _ in range(2):
                H.h2bem_apply(Bop.op, xb, yb, stream)
                H.h2bem_grad(Bop.op, wb, xb, gX, gx, stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize(dev)
            ev[0].record(stream)
            H.h2bem_apply(Bop.op, xb, yb, stream)
            ev[1].record(stream)
            H.h2bem_grad(Bop.op, wb, xb, gX, gx, stream)
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            extra[f"batch64_{'fp64' if prec == 'fp64' else 'mixed'}"] = {
                "meshes": len(fam), "triangles": Bop.n, "apply_ms": ev[0].elapsed_time(ev[1]),
                "grad_x_and_vertices_ms": ev[1].elapsed_time(ev[2]),
                "apply_triangles_per_s": Bop.n / (ev[0].elapsed_time(ev[1]) / 1e3),
                "note": "gradient in FP64 in every tier"}
            Bop.close()
        # ellipsoid (1, 0.5, 0.25), 131,072 triangles, m = 5, 16 right-hand sides
        me = I.ellipsoid(128)
        xe = torch.from_numpy(I.rhs(me.nt, 16, seed=5)).to(dev)
        out_e = {}
        for prec in ("mixed_fp32", "mixed_tf32", "mixed_bf16", "fp64"):
            oe = H.Operator(me.vertices, me.triangles, kernel="slp", m=5, eta=2.0, precision=prec, autotune=1)
            ye = torch.empty_like(xe)
            for _ in range(2):
                H.h2bem_apply(oe.op, xe, ye, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            H.h2bem_apply(oe.op, xe, ye, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out_e[prec] = (e0.elapsed_time(e1), ye.clone())
            oe.close()
        out = {p_: {"ms": v[0], "triangles_rhs_per_s": me.nt * 16 / (v[0] / 1e3)} for p_, v in out_e.items()}
        for p_ in ("mixed_fp32", "mixed_tf32", "mixed_bf16"):
            out[p_]["rel_err_vs_fp64"] = float(torch.linalg.norm(out_e[p_][1] - out_e["fp64"][1]) /
                                               torch.linalg.norm(out_e["fp64"][1]))
        extra["ellipsoid131k_m5_16rhs"] = out

    # Dirichlet-to-Neumann solve (section 1, eq. (matrix_dtn)): G x = (M/2 + K) b
    # by the library's conjugate gradients, mixed tier, for the harmonic test
    # functions u1 = x1^2 - x3^2, u2 = g(., (1.2, 1.2, 1.2)), u3 = g(., (1, 0.25, 1));
    # b = L2 projection onto the triangles.  The condition number of G grows as
    # 1/h, so the matrix accuracy has to grow with n (section 5 raises the order
    # with n); at a fixed m = 4 the Neumann error stops improving past ~32k
    # triangles.  Two spheres one refinement apart at m = 6, eta = 1 show the
    # O(h) rate of the L2 Neumann error.
    if not args.no_fp64 and not args.no_extras:
        ru = np.array([0.5, 0.5, 0.0])  # edge-midpoint rule (exact for degree 2)
        rv = np.array([0.0, 0.5, 0.5])
        rw = np.array([1 / 3, 1 / 3, 1 / 3])

        def u_dn(k, p_):
            if k == 0:
                return p_[..., 0] ** 2 - p_[..., 2] ** 2, 2 * p_[..., 0] ** 2 - 2 * p_[..., 2] ** 2
            yv = np.array([1.2, 1.2, 1.2]) if k == 1 else np.array([1.0, 0.25, 1.0])
            dd = p_ - yv
            r = np.linalg.norm(dd, axis=-1)
            return 1 / (4 * np.pi * r), -(dd * p_).sum(-1) / (4 * np.pi * r ** 3)

        def dtn_case(s_dtn, m_dtn, eta_dtn, rtol):
            md = I.sphere(s_dtn)
            v = md.vertices
            ta, tb, tc = (v[md.triangles[:, q]] for q in range(3))
            pts = ta[:, None] + ru[None, :, None] * (tb - ta)[:, None] + rv[None, :, None] * (tc - ta)[:, None]
            area = 0.5 * np.linalg.norm(np.cross(tb - ta, tc - ta), axis=1)
            proj = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
            bvec = np.stack([(u_dn(k, pts)[0] * rw[None, :]).sum(1) for k in range(3)])
            t_set = time.perf_counter()
            # a solve applies G hundreds of times: nearfield entries stored once
            opG = H.Operator(v, md.triangles, kernel="slp", m=m_dtn, eta=eta_dtn, precision="mixed_fp32", autotune=1,
                             store_near=True)
            opK = H.Operator(v, md.triangles, kernel="dlp", m=m_dtn, eta=eta_dtn, precision="mixed_fp32", autotune=1)
            torch.cuda.synchronize(dev)
            t_set = time.perf_counter() - t_set
            bd = torch.from_numpy(np.ascontiguousarray(bvec)).to(dev)
            rhs_d = torch.empty_like(bd)
            xd_ = torch.empty_like(bd)
            H.h2bem_apply_mass(opK.op, 0.5, bd, rhs_d, stream)
            H.h2bem_cg(opG.op, rhs_d, xd_, rtol=1e-3, maxit=5, stream=stream)  # warm-up (tuning)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            H.h2bem_apply_mass(opK.op, 0.5, bd, rhs_d, stream)
            its, rel = H.h2bem_cg(opG.op, rhs_d, xd_, rtol=rtol, maxit=3000, stream=stream)
            torch.cuda.synchronize(dev)
            t_solve = time.perf_counter() - t0
            xs = xd_.cpu().numpy()
            l2 = {}
            for k, nm in enumerate(("u1", "u2", "u3")):
                dn = u_dn(k, proj)[1]
                l2[nm] = float(np.sqrt((area[:, None] * rw[None, :] * (xs[k][:, None] - dn) ** 2).sum() /
                                       (area[:, None] * rw[None, :] * dn ** 2).sum()))
            opG.close()
            opK.close()
            return {"triangles": md.nt, "m": m_dtn, "eta": eta_dtn, "rhs": 3, "iterations": its, "rtol": rtol,
                    "relres": rel, "setup_s": t_set, "solve_s": t_solve, "ms_per_iteration": 1e3 * t_solve / max(its, 1),
                    "store_near": True,
                    "neumann_l2_rel_err": l2}

        coarse = dtn_case(128, 6, 1.0, 1e-8)
        fine = dtn_case(256, 6, 1.0, 1e-8)
        extra["dtn_cg_mixed"] = {
            "coarse": coarse, "fine": fine,
            "observed_order": {nm: float(np.log2(coarse["neumann_l2_rel_err"][nm] / fine["neumann_l2_rel_err"][nm]))
                               for nm in ("u1", "u2", "u3")},
            "expected_order": 1.0}

    # hypersingular operator W on piecewise-linear functions (section 1) through its
    # single-layer representation W = sum_d C_d^T G C_d, on the same sphere: one
    # apply with nrhs vertex vectors (3 nrhs single-layer columns), the Rayleigh
    # quotient of the interpolated harmonic Y_2 (exact value 6/5 on the unit sphere)
    # and W 1 (zero: W annihilates constants)
    if not args.no_fp64 and not args.no_extras:
        opw = H.Operator(mesh.vertices, mesh.triangles, kernel="slp", m=4, eta=2.0, leaf_size=32,
                         precision=args.tier, autotune=args.autotune)
        nv = mesh.vertices.shape[0]
        xv = torch.from_numpy(I.rhs(nv, nrhs, seed=11)).to(dev)
        yv = torch.empty_like(xv)
        for _ in range(2):
            H.h2bem_apply_hypersingular(opw.op, xv, yv, stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            H.h2bem_apply_hypersingular(opw.op, xv, yv, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_w = e0.elapsed_time(e1) / 3
        vv = mesh.vertices
        u = 3 * vv[:, 2] ** 2 - (vv ** 2).sum(1)
        tt = mesh.triangles
        ar = 0.5 * np.linalg.norm(np.cross(vv[tt[:, 1]] - vv[tt[:, 0]], vv[tt[:, 2]] - vv[tt[:, 0]]), axis=1)
        ut = u[tt]
        uMu = float((ar / 12 * ((ut ** 2).sum(1) + ut.sum(1) ** 2)).sum())
        ud = torch.from_numpy(np.ascontiguousarray(np.stack([u, np.ones(nv)]))).to(dev)
        wu = torch.empty_like(ud)
        H.h2bem_apply_hypersingular(opw.op, ud, wu, stream)
        torch.cuda.synchronize(dev)
        wu = wu.cpu().numpy()
        opw.close()
        extra["hypersingular_w"] = {
            "vertices": nv, "rhs": nrhs, "single_layer_columns": 3 * nrhs, "ms_per_apply": ms_w,
            "vertex_rhs_per_s": nv * nrhs / (ms_w / 1e3), "tier": args.tier,
            "rayleigh_Y2": float(u @ wu[0] / uMu), "rayleigh_Y2_exact": 1.2,
            "W1_rel": float(np.abs(wu[1]).max() / np.abs(wu[0]).max())}

    # hybrid cross approximation (section 3) compressed into an H^2-matrix, on the
    # 131,072-triangle sphere (the host construction grows as n log n times the
    # blocks per cluster row: ~30 s here): set-up, apply in both tiers, mean rank,
    # stored bytes, the H^2 error against exact Galerkin rows beside the
    # Chebyshev bases' on the same rows
    if not args.no_fp64 and not args.no_extras:
        mh_ = I.sphere(128)
        xh_ = torch.from_numpy(I.rhs(mh_.nt, nrhs, seed=13)).to(dev)
        rows_h = np.random.default_rng(2).choice(mh_.nt, 24, replace=False)
        dref_h = oracle.dense_rows(0, mh_, rows_h, xh_.cpu().numpy())

        def rows_err(y_t):
            yy = y_t.cpu().numpy()[:, rows_h]
            return float(np.linalg.norm(yy - dref_h) / np.linalg.norm(dref_h))

        hca = {"triangles": mh_.nt, "m": 4, "eps_aca": 1e-6, "eps": 1e-6, "rhs": nrhs}
        y_h = {}
        for prec in ("mixed_fp32", "fp64"):
            t_set = time.perf_counter()
            oh = H.Operator(mh_.vertices, mh_.triangles, kernel="slp", m=4, eta=2.0, precision=prec, hca=True)
            torch.cuda.synchronize(dev)
            t_set = time.perf_counter() - t_set
            yh_ = torch.empty_like(xh_)
            for _ in range(2):
                H.h2bem_apply(oh.op, xh_, yh_, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(3):
                H.h2bem_apply(oh.op, xh_, yh_, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st_h = oh.stats()
            oh.close()
            y_h[prec] = yh_.clone()
            hca[prec] = {"ms_per_apply": e0.elapsed_time(e1) / 3, "setup_s": round(t_set, 2),
                         "triangles_rhs_per_s": mh_.nt * nrhs / (e0.elapsed_time(e1) / 3e3),
                         "mean_rank": st_h["mean_rank"], "far_stored_bytes": st_h["far_stored_bytes"],
                         "h2_error_vs_dense_rows": rows_err(yh_)}
        hca["rel_err_mixed_vs_fp64"] = float(torch.linalg.norm(y_h["mixed_fp32"] - y_h["fp64"]) /
                                             torch.linalg.norm(y_h["fp64"]))
        oc = H.Operator(mh_.vertices, mh_.triangles, kernel="slp", m=4, eta=2.0, precision="fp64")
        yc_ = torch.empty_like(xh_)
        H.h2bem_apply(oc.op, xh_, yc_, stream)
        torch.cuda.synchronize(dev)
        oc.close()
        hca["chebyshev_m4_h2_error_vs_dense_rows"] = rows_err(yc_)
        extra["hca_sphere131k"] = hca
        del y_h

    # double layer with piecewise-linear trial functions K1 (section 1, eq. (dlp) with
    # the hat functions) on the same sphere: forward (vertices -> triangles) and
    # transposed applies; its nearfield and Sauter-Schwab pairs are FP64 in every tier
    if not args.no_fp64 and not args.no_extras:
        op1 = H.Operator(mesh.vertices, mesh.triangles, kernel="dlp", m=4, eta=2.0, leaf_size=32,
                         precision=args.tier, autotune=args.autotune)
        nv = mesh.vertices.shape[0]
        xv1 = torch.from_numpy(I.rhs(nv, nrhs, seed=12)).to(dev)
        yt1 = torch.empty((nrhs, n), dtype=torch.float64, device=dev)
        yv1 = torch.empty_like(xv1)
        k1 = {"vertices": nv, "rhs": nrhs, "tier": args.tier}
        for tr, xin, yout in ((False, xv1, yt1), (True, yt1, yv1)):
            H.h2bem_apply_dlp_p1(op1.op, xin, yout, transpose=tr, stream=stream)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.h2bem_apply_dlp_p1(op1.op, xin, yout, transpose=tr, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            k1["transpose_ms" if tr else "forward_ms"] = e0.elapsed_time(e1)
        op1.close()
        extra["dlp_p1_k1"] = k1

    # Neumann-to-Dirichlet solve (section 1, eq. (neumann_to_dirichlet)):
    # (W + m m^T) x = (M1^T / 2 - K1^T) b + m (m . u) with piecewise-constant
    # Neumann data b (the L2 projection of du/dn) and piecewise-linear Dirichlet
    # values x (m the P1 mass row sums, fixing the constant), by the library's
    # conjugate gradients, mixed tier, for the same test functions; the L2 error
    # of x against u at the vertices, two spheres one refinement apart
    if not args.no_fp64 and not args.no_extras:
        def ntd_case(s_ntd, m_ntd, eta_ntd, rtol):
            import scipy.sparse as sps

            md = I.sphere(s_ntd)
            v, tri = md.vertices, md.triangles
            ta, tb, tc = (v[tri[:, q]] for q in range(3))
            ar = 0.5 * np.linalg.norm(np.cross(tb - ta, tc - ta), axis=1)
            pts = ta[:, None] + ru[None, :, None] * (tb - ta)[:, None] + rv[None, :, None] * (tc - ta)[:, None]
            proj = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
            bn = np.stack([(u_dn(k, proj)[1] * rw[None, :]).sum(1) for k in range(3)])
            uI = np.stack([u_dn(k, v)[0] for k in range(3)])
            loc = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
            Mp = sps.csr_matrix((np.concatenate([ar * loc[a, c] for a in range(3) for c in range(3)]),
                                 (np.concatenate([tri[:, a] for a in range(3) for _ in range(3)]),
                                  np.concatenate([tri[:, c] for _ in range(3) for c in range(3)]))),
                                shape=(md.nv, md.nv))
            mv = np.asarray(Mp.sum(1)).ravel()
            t_set = time.perf_counter()
            opG = H.Operator(v, tri, kernel="slp", m=m_ntd, eta=eta_ntd, precision="mixed_fp32", autotune=1,
                             store_near=True)
            opK = H.Operator(v, tri, kernel="dlp", m=m_ntd, eta=eta_ntd, precision="mixed_fp32", autotune=1)
            torch.cuda.synchronize(dev)
            t_set = time.perf_counter() - t_set
            bd = torch.from_numpy(np.ascontiguousarray(-bn)).to(dev)
            mvd = torch.from_numpy(mv).to(dev)
            ud = torch.from_numpy(uI).to(dev)
            rhs_d = torch.empty((3, md.nv), dtype=torch.float64, device=dev)
            xd_ = torch.empty_like(rhs_d)
            H.h2bem_apply_dlp_p1(opK.op, bd, rhs_d, transpose=True, alpha=-0.5, stream=stream)
            H.h2bem_cg_hypersingular(opG.op, mvd, rhs_d, xd_, rtol=1e-3, maxit=5, stream=stream)  # warm-up
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            H.h2bem_apply_dlp_p1(opK.op, bd, rhs_d, transpose=True, alpha=-0.5, stream=stream)
            rhs_d += (ud @ mvd)[:, None] * mvd[None, :]
            its, rel = H.h2bem_cg_hypersingular(opG.op, mvd, rhs_d, xd_, rtol=rtol, maxit=3000, stream=stream)
            torch.cuda.synchronize(dev)
            t_solve = time.perf_counter() - t0
            xs = xd_.cpu().numpy()
            l2 = {}
            for k, nm in enumerate(("u1", "u2", "u3")):
                e = xs[k] - uI[k]
                l2[nm] = float(np.sqrt(e @ (Mp @ e) / (uI[k] @ (Mp @ uI[k]))))
            opG.close()
            opK.close()
            return {"triangles": md.nt, "vertices": md.nv, "m": m_ntd, "eta": eta_ntd, "rhs": 3,
                    "iterations": its, "rtol": rtol, "relres": rel, "setup_s": t_set, "solve_s": t_solve,
                    "ms_per_iteration": 1e3 * t_solve / max(its, 1), "dirichlet_l2_rel_err": l2}

        coarse = ntd_case(64, 6, 1.0, 1e-9)
        fine = ntd_case(128, 6, 1.0, 1e-9)
        extra["ntd_cg_mixed"] = {
            "coarse": coarse, "fine": fine,
            "observed_order": {nm: float(np.log2(coarse["dirichlet_l2_rel_err"][nm] / fine["dirichlet_l2_rel_err"][nm]))
                               for nm in ("u1", "u2", "u3")},
            "expected_order": 2.0}

    # roofline of the dominant kernel of the headline tier
    pk = peaks()
    names = ["permute_in", "leaf_forward", "upward", "coupling", "downward", "leaf_backward", "near_regular",
             "near_singular"]
    dom = int(np.argmax(stage_m))
    sing = st_m["singular_pairs"]
    evals = {
        "near_regular": st_m["regular_evals"] * 49,
        "near_singular": sum(sing[t] * PTS_SING[t] for t in range(3)),
    }
    if not args.gca:  # GCA coupling matrices are stored, not generated
        evals["coupling"] = st_m["nfar"] * st_m["k"] ** 2
    kern = {}
    if args.store_near:
        # the nearfield stage streams stored entries: rated in bytes against the HBM peak
        for nm in ("near_regular", "near_singular"):
            evals.pop(nm)
        names[6] = "near_stored"
        alg = st_m["near_pairs"] * 4 + n * nrhs * (4 + 8)
        ms6 = float(stage_m[6])
        kern["near_stored"] = {"ms": round(ms6, 3), "bytes": int(alg), "gb_s": alg / (ms6 / 1e3) / 1e9,
                               "frac_of_hbm_peak": alg / (ms6 / 1e3) / 1e9 / pk["hbm_gbs"]}
    for nm, ev in evals.items():
        ms = float(stage_m[names.index(nm)])
        rate = ev / (ms / 1e3) / 1e9  # Geval/s
        kern[nm] = {"ms": round(ms, 3), "evals": int(ev), "geval_s": rate,
                    "frac_of_rsqrt_peak": rate / (pk["rsqrt_tops"] * 1e3)}
    if "coupling" in kern:
        kern["coupling"]["fp32_tflops"] = (st_m["nfar"] * st_m["k"] ** 2 * 2 * nrhs / (kern["coupling"]["ms"] / 1e3)
                                           / 1e12)
        kern["coupling"]["frac_of_fp32_peak"] = kern["coupling"]["fp32_tflops"] / pk["fp32_tflops"]
    else:
        kern["coupling"] = {"ms": round(float(stage_m[3]), 3), "stored_bytes": st_m["far_stored_bytes"],
                            "gb_s": st_m["far_stored_bytes"] / (float(stage_m[3]) / 1e3) / 1e9}
    dname = names[dom]
    if dname == "near_stored":
        roof = {"bound": "hbm", "kernel": dname, "achieved": kern[dname]["gb_s"], "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": kern[dname]["frac_of_hbm_peak"], "traffic": None,
                "peak_source": "MEASURED_PEAKS.json copy bandwidth", "all_kernels": kern}
    elif dname in kern:
        roof = {"bound": "alu", "kernel": dname, "achieved": kern[dname]["geval_s"],
                "peak": pk["rsqrt_tops"] * 1e3, "unit": "Geval/s", "frac": kern[dname]["frac_of_rsqrt_peak"],
                "traffic": TRAFFIC.get(dname),
                "peak_source": f"FP32 reciprocal square root rate, {pk['alu_src']} (one per kernel evaluation)",
                "all_kernels": kern, "peaks": {k_: v for k_, v in pk.items() if k_ != "src"}}
    else:
        roof = {"bound": "alu", "kernel": dname, "achieved": None, "peak": None, "unit": "Geval/s", "frac": None,
                "traffic": None, "all_kernels": kern}

    cpu = None
    if rank == 0 and not args.no_cpu:
        sec, rows_c, n_c, cores, setup_c, t_up, t_rows = cpu_oracle_sample(args.s, nrhs, 1)
        cpu = {"value": rows_c * nrhs / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample_text(rows_c, n_c, nrhs), "setup_s": round(setup_c, 1),
               "upward_s": round(t_up, 2), "rows_s": round(t_rows, 2)}

    value = replica_throughput(n * nrhs, ms_m / 1e3, world)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_m, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed tier: FP32 farfield, regular pairs and Sauter-Schwab pairs; "
                 "FP64 area scaling and accumulation of y)",
        "data": "synthetic",
        "config": {"workload": f"sphere_{n}_slp_m4_eta2_leaf32_nrhs{nrhs}", "n": n, "nrhs": nrhs, "m": 4,
                   "eta": 2.0, "leaf": 32, "tier": args.tier,
                   "nearfield": "stored (entries evaluated at set-up)" if args.store_near else "on the fly",
                   "farfield": "GCA bases, stored coupling" if args.gca else "Chebyshev bases, coupling on the fly",
                   "l2": "inputs exceed L2 (geometry 151 MB, x/y 134 MB, cluster vectors >400 MB per step)",
                   "parallelism": f"replicas{world}"},
        "stage_ms": {nm: round(float(v), 3) for nm, v in zip(names, stage_m)},
        "ms_per_step_sequential": ms_m_sequential,
        "timing_note": ("value: back-to-back applies, the farfield passes on the operator's second stream "
                        "concurrently with the nearfield; stage_ms and the roofline's kernel time: the same "
                        "number of timed applies right after, every stage on one stream (ms_per_step_sequential)"),
        "setup_s": round(setup_m, 2),
        "counts": {k: st_m[k] for k in ("nclusters", "nleaves", "nfar", "nnear", "near_pairs", "regular_pairs",
                                        "singular_pairs")},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": replica_throughput(n * nrhs, e2e_s, world), "unit": UNIT, "h2d_bytes_per_step": n * nrhs * 8,
                "d2h_bytes_per_step": n * nrhs * 8},
        "gpu_launches": int(st_m["launches"]) * args.steps,
        "launch_variant": {"near_persistent": st_m["launch_variant"][0], "near_ctas_per_sm": st_m["launch_variant"][1],
                           "coupling_slices": st_m["launch_variant"][2],
                           "coupling_persistent": st_m["launch_variant"][3], "autotuned": st_m["launch_variant"][4]},
        "clocks": clocks,
    }
    out.update(extra)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
