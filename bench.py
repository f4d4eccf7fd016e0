#!/usr/bin/env python
"""Throughput of the fast spectral collision operator Q^(pq) on GB300.

One step = one call of the C-ABI collision entry point over the whole
1-D-slab workload (24 spatial points x 4 species pairs = 96 Q^(pq)
evaluations at N = 32, M = 12, N_rho = 8, VSS omega = 0.75, alpha = 1.4),
inputs resident in HBM, L2 flushed (256 MiB write) before every timed step.

Prints ONE JSON line (rank 0).  Fields beyond the base contract:
  forms        evals/s and relative max-norm error vs the FP64 CPU oracle for
               every precision form measured (tensor-core FP32 vs FP64),
  roofline     the dominant kernel: algorithmic FLOPs per launch (5 N^3 log2 N per
               length-N axis pass of a 3-D transform, plus the elementwise work
               the method performs) / its average CUDA-event duration, against the
               tensor-core rate measured on this GPU by the library's own probe;
               beside it the executed dense-MMA FLOPs (the DFT contractions as
               GEMMs, all split products) under "executed_mma", and the whole
               step's algorithmic rate,
  cpu_baseline the FP64 oracle timed on this host's cores on a bounded sample,
  e2e          the same metric through the host-buffer C-ABI call,
  clocks       nvidia-smi samples taken during the timed region,
  step_ms_p10_p50_p90  the spread of the timed steps,
  kernels      per-kernel CUDA-event times from a profiled pass after the timed
               region (the library then issues its launches in one stream),
  alu_peaks    cuBLAS FP64 and FP32 (TF32 off) GEMM rates of this GPU,
  graph        the same call replayed from one CUDA graph,
  dg_step      one SSP-RK3 step of the 1-D DG heat-transfer slab,
  uneven_batch 256 uneven relaxation problems: separate calls, a graph of them,
               the batched rounds (eager and captured) and the batch as one
               work-list launch per N group,
  schedules    the benchmark call with per-stage launches and as one work-list launch,
  adjoint      the FP64 and 3xTF32 backward on the 64-point adjoint workload against their forwards,
  tensor_peaks the tensor pipe's tf32 and bf16 issue rates measured by the library's probe.

--impl reference times the FP64 CPU oracle (the only reference that exists:
the paper publishes no code) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Q^(pq) evals/s at N=32,M=12,Nrho=8: TC-FP32 vs FP64 on GB300, err vs FP64"
UNIT = "Q^(pq) evals/s"
WORKLOAD = "c2_slab_n32"
WORKLOAD_DESC = ("1-D DG slab: 8 elements x 3 Gauss points = 24 spatial points, 2 species (m = 1, 4), "
                 "VSS omega = 0.75, alpha = 1.4, N = 32 on [-10, 10]^3, M = 12 (icosahedron), N_rho = 8; "
                 "f = Hermite-perturbed Maxwellians (seed 2)")
# P100 FP64, Table 1 (N = 32, N_rho = 8, M = 12, mass ratio 1): 0.00287 s per evaluation
PAPER_EVALS_PER_S = 1.0 / 0.00287
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


# ------------------------------------------------------------ work models
def fft_flops(N):
    return 5.0 * N * math.log2(N)


def kernel_work(name, plan_info, P, S, RS):
    """Algorithmic FLOPs of one launch of a kernel class (the FFT count
    5 N log2 N per length-N complex transform plus the complex multiplies the
    method performs), used for the roofline's achieved rate."""
    N = int(plan_info["N"])
    E = min(int(plan_info["chunk"]), P)
    pen = N * N
    f = fft_flops(N)
    if name == "fp64_inv_first" or name == "fp64_inv":
        return E * RS * pen * 2 * (f + 6 * N)
    if name == "fp64_prod":
        return E * RS * pen * (3 * f + 3 * 6 * N)
    if name == "fp64_fwd":
        return E * RS * pen * f  # dominant instances act on the (r, s) grids
    if name == "fp64_mac":
        return E * RS * pen * (f + 10 * N)
    return None


# --------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1903_04670_gb300 import binding as B
    from paper_1903_04670_gb300 import distributed as D
    from paper_1903_04670_gb300 import workloads as W

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    dev = torch.cuda.current_device()
    pb = W.make_problem(WORKLOAD, points=args.points)
    P, S = pb["f"].shape[0], pb["f"].shape[1]
    RS = pb["M"] * pb["Nrho"]
    evals = P * S * S
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def make(prec):
        return B.Plan(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"], prec, P, dev)

    precisions = [args.precision] if args.precision != "auto" else ["fp32_tc", "bf16x3", "tf32", "fp64"]
    if args.precision == "auto" and not args.no_hermitian:
        # the declared Hermitian form (Nyquist planes removed, two points per grid slot)
        precisions += ["fp32_tc_hermitian", "fp64_hermitian"]
    forms = {}
    main = None
    for form in precisions:
        prec = form.replace("_hermitian", "")
        try:
            plan = make(prec)
            if form.endswith("_hermitian"):
                plan.set_hermitian(True)
            f = torch.from_numpy(pb["f"]).to("cuda", plan.dtype)
            Q = plan.collide(f)
            torch.cuda.synchronize()
        except B.DgfsError as e:
            if e.status == 5:
                forms[form] = {"unavailable": str(e)}
                continue
            raise
        if prec != "fp64" and not args.no_tune:
            plan.autotune(f, Q)  # the library's own launch-parameter search, outside the timed region
        steps = args.steps if main is None else max(2, min(args.steps, 3))
        for _ in range(args.warmup):
            plan.collide(f, Q)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        n0 = plan.launch_count()
        clocks = ClockSampler(dev) if main is None else None
        if clocks:
            clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            plan.collide(f, Q)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        per_step = sorted(a.elapsed_time(b) for a, b in ev)
        ms = sum(per_step)
        launches = plan.launch_count() - n0
        clk = clocks.stop() if clocks else None
        # per-kernel CUDA-event times: a profiling pass right after the timed
        # region, same calls; with its profiler on the library runs the plan's
        # launches in one stream, so each kernel's bracket is its own time
        psteps = max(2, min(steps, 20))
        plan.profile(True)
        for k in range(psteps):
            flush.zero_()
            plan.collide(f, Q)
        torch.cuda.synchronize()
        prof = plan.profile_read()
        plan.profile(False)
        if world > 1:
            ms = D.max_over_ranks(ms, device="cuda")
        value = world * evals * steps / (ms / 1e3)
        pct = lambda q: per_step[min(len(per_step) - 1, int(round(q * (len(per_step) - 1))))]
        rec = {"value": value, "ms_per_step": ms / steps, "steps": steps, "launches": launches,
               "step_ms_p10_p50_p90": [pct(0.1), pct(0.5), pct(0.9)], "profile_steps": psteps,
               "profile": prof, "plan": plan, "f": f, "Q": Q, "clocks": clk}
        forms[form] = rec
        if main is None:
            main = form

    if main is None:
        raise RuntimeError("no precision form could run")
    rec = forms[main]
    plan = rec["plan"]
    info = plan.info()
    out = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": rec["steps"],
           "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": rec["value"] / PAPER_EVALS_PER_S,
           "vs_baseline_ref": "P100 FP64, paper Table 1 (N=32, N_rho=8, M=12): 0.00287 s per evaluation",
           "dtype": "f64" if main == "fp64" else "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "points": P, "species": S,
                      "evals_per_step": evals, "precision": main, "rs_per_eval": RS,
                      "l2": "flushed before every timed step (256 MiB write, outside the events)",
                      "launch_parameters": "dgfs_plan_autotune before timing" if not args.no_tune else "defaults",
                      "launch": {k: int(info[k]) for k in ("chunk", "rs_blocks", "groups_a", "groups_b", "nterms")}
                      if main != "fp64" else None,
                      "parallelism": "replicas: every rank evaluates its own 96 (point, pair) operators"}}

    peaks, src = _peaks()
    if not args.no_peaks:
        out["alu_peaks"] = alu_peaks(torch)
        # the tensor-core denominators, measured here by the library's probe
        try:
            out["tensor_peaks"] = {"tf32": B.dgfs_probe_mma_rate(dev, "tf32", 4096),
                                   "bf16": B.dgfs_probe_mma_rate(dev, "bf16", 4096), "unit": "TFLOP/s",
                                   "how": "one CTA per SM issues 4096 back-to-back tcgen05 MMAs (M = 128, "
                                          "N = 256) into TMEM; best of three timed launches",
                                   "measured_peaks_json": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops",
                                                                                     "bf16_tflops_sustained")}}
        except B.DgfsError as e:
            out["tensor_peaks"] = {"error": str(e)}

    # roofline of the dominant kernel (by summed event time)
    prof = rec["profile"]
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, tot_ms) = dom
    work = kernel_work(name, info, P, S, RS)
    avg_s = tot_ms / cnt / 1e3
    if name.startswith("fp64"):
        if "alu_peaks" in out:
            peak = out["alu_peaks"]["fp64_gemm_tflops"] * 1e3
            psrc = "measured FP64 GEMM (cuBLAS) on this GPU"
        else:
            peak = 1250.0  # GFLOP/s: nominal GB300 FP64
            psrc = "nominal FP64 of the GB300 (1.25 TFLOP/s)"
        roof = {"bound": "alu", "achieved": work / avg_s / 1e9 if work else None, "peak": peak,
                "unit": "GFLOP/s", "peak_source": psrc}
    else:
        sigma = plan.pair_tables(0, 0, with_b=False)["sigma"]
        kind = "bf16" if main == "bf16x3" else "tf32"
        probe = out.get("tensor_peaks", {}).get(kind)
        if probe:
            peak, psrc = probe, ("tcgen05 kind::%s M = 128, N = 256 back-to-back issue rate on all SMs, measured "
                                 "in this run (dgfs_probe_mma_rate)" % ("tf32" if kind == "tf32" else "f16 (bf16)"))
        else:
            bf16 = peaks["bf16_tflops"]
            peak = bf16 * ((1.1 / 2.25) if kind == "tf32" else 1.0)
            psrc = "%s bf16 GEMM (%.1f TFLOP/s)%s" % (src, bf16, " x nominal tf32/bf16 1.1/2.25" if kind == "tf32"
                                                      else "")
        roof = tc_roofline(name, info, P, S, RS, avg_s, peak, psrc, cnt / rec["profile_steps"], sigma)
    roof["frac"] = roof["achieved"] / roof["peak"] if roof.get("achieved") else None
    roof["kernel"] = name
    roof["launches"] = cnt
    roof["avg_launch_ms"] = tot_ms / cnt
    roof["share_of_step"] = tot_ms / sum(v[1] for v in prof.values())
    roof["timing"] = ("CUDA events around each launch in a %d-step pass right after the timed region "
                      "(the library then issues the plan's launches in one stream)" % rec["profile_steps"])
    ppl = min(P, int(info["chunk"])) if not name.startswith("fp64") else None
    roof["traffic"], roof["traffic_source"] = ncu_traffic(name, P, ppl)
    # DRAM traffic of the three stage kernels per step against the step's
    # algorithmic bytes (f in, Q out, the b tables once): the cost of the
    # per-(r, s) intermediates that pass through HBM
    if not name.startswith("fp64"):
        tsum = 0.0
        for k in NCU_TRAFFIC_24PT:
            t, _ = ncu_traffic(k, P, ppl)
            if t is None or k not in prof:
                tsum = None
                break
            tsum += t * prof[k][0] / rec["profile_steps"]
        if tsum:
            ab = step_algorithmic_bytes(int(info["N"]), P, S, RS)
            roof["step_traffic"] = {"stage_kernels_bytes": tsum, "algorithmic_bytes": ab, "ratio": tsum / ab}
    # the whole step on the same peak: every kernel of the call, algorithmic FLOPs
    if not name.startswith("fp64"):
        sf = step_algorithmic_flops(int(info["N"]), P, S, RS)
        roof["step"] = {"achieved": sf / (rec["ms_per_step"] / 1e3) / 1e12, "unit": "TFLOP/s",
                        "frac": sf / (rec["ms_per_step"] / 1e3) / 1e12 / roof["peak"],
                        "work_per_step": sf, "work_unit": "algorithmic FLOPs of all evaluations of the step"}
    out["roofline"] = roof
    out["kernels"] = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items()}
    out["kernels_steps"] = rec["profile_steps"]
    out["gpu_launches"] = rec["launches"]
    out["step_ms_p10_p50_p90"] = rec["step_ms_p10_p50_p90"]
    out["clocks"] = rec["clocks"]

    # the two stage schedules of the tensor-core call (the autotuner keeps the
    # faster): per-stage launches on two streams, and one work-list launch
    if main != "fp64" and int(info["N"]) in (24, 32, 48) and not args.no_graph:
        chosen = plan.schedule()
        sch = {"chosen": chosen}
        for mode in (0, 1):
            plan.set_schedule(mode)
            for _ in range(2):
                plan.collide(rec["f"], rec["Q"])
            torch.cuda.synchronize()
            sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for a, b in sev:
                flush.zero_()
                a.record(stream)
                plan.collide(rec["f"], rec["Q"])
                b.record(stream)
            torch.cuda.synchronize()
            t = sorted(a.elapsed_time(b) for a, b in sev)[5]
            sch["launches" if mode == 0 else "work_list"] = {"ms_per_step": t, "evals_per_s": evals / (t / 1e3)}
        plan.set_schedule(chosen)
        plan.check()
        out["schedules"] = sch

    # the same call replayed from one CUDA graph: the host-side scheduling cost
    if not args.no_graph:
        g = B.dgfs_graph_capture([plan._h], [P], [rec["f"]], [rec["Q"]])
        try:
            for _ in range(2):
                B.dgfs_graph_launch(g, stream)
            torch.cuda.synchronize()
            gsteps = max(2, min(rec["steps"], 20))
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(gsteps)]
            for k in range(gsteps):
                flush.zero_()
                gev[k][0].record(stream)
                B.dgfs_graph_launch(g, stream)
                gev[k][1].record(stream)
            torch.cuda.synchronize()
            gms = sum(a.elapsed_time(b) for a, b in gev) / gsteps
            out["graph"] = {"ms_per_step": gms, "eager_ms_per_step": rec["ms_per_step"], "steps": gsteps,
                            "kernels_per_replay": B.dgfs_graph_kernel_count(g)}
        finally:
            B.dgfs_graph_destroy(g)

    # one SSP-RK3 step of the 1-D DG heat-transfer slab around the operator:
    # transport kernels plus three collision calls on all 48 points
    if not args.no_dg:
        sp = W.make_problem("c5_heat_slab_n32")
        splan = B.Plan(sp["N"], sp["L"], sp["M"], sp["Nrho"], sp["masses"], sp["pairs"], main,
                       sp["f"].shape[0], dev)
        slab = B.Slab(splan, sp["elements"], sp["order"], 0.0, 1.0, sp["walls"])
        fs = torch.from_numpy(sp["f"]).to("cuda", splan.dtype)
        dt = 1e-3  # below the SSP-RK3 / DG(K=3) CFL limit h_x / (5 max|c_x|) = 1.6e-3
        for _ in range(3):
            slab.step(fs, dt)
        torch.cuda.synchronize()
        dsteps = 10
        dev_ = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(dsteps)]
        for k in range(dsteps):
            flush.zero_()
            dev_[k][0].record(stream)
            slab.step(fs, dt)
            dev_[k][1].record(stream)
        torch.cuda.synchronize()
        dms = sum(a.elapsed_time(b) for a, b in dev_) / dsteps
        # transport / collision split from a profiled pass (one stream)
        splan.profile(True)
        for k in range(3):
            flush.zero_()
            slab.step(fs, dt)
        torch.cuda.synchronize()
        dprof = splan.profile_read()
        splan.profile(False)
        tr = sum(v[1] for k, v in dprof.items() if k.startswith("dg_")) / 3
        co = sum(v[1] for k, v in dprof.items() if not k.startswith("dg_")) / 3
        nev = 3 * sp["f"].shape[0] * S * S
        out["dg_step"] = {"workload": "c5_heat_slab_n32",
                          "description": "16 elements x 3 Gauss points, 2 species (m = 1, 2), VHS omega = 0.81, "
                                         "N = 32 on [-8, 8]^3, M = 12, N_rho = 8, diffuse walls at T = 1 and "
                                         "T = 2; SSP-RK3, dt = 1e-3",
                          "precision": main, "steps": dsteps, "ms_per_step": dms,
                          "collision_evals_per_step": nev, "evals_per_s": nev / (dms / 1e3),
                          "transport_kernel_ms_per_step": tr, "collision_kernel_ms_per_step": co}
        del slab, splan

    # the adjoint on the adjoint workload (64 points x 2 species x 32^3): one
    # dgfs_collide_backward of the FP64 plan and of the 3xTF32 plan (its
    # (r, s) loop on the tensor cores), each against one forward call of the
    # same plan; the omega gradient is requested in both
    if not args.no_adjoint:
        ap = W.make_problem("c4_adjoint_n32", points=args.adjoint_points)
        Pa = ap["f"].shape[0]
        aforms = args.adjoint_forms.split(",")
        fa = torch.from_numpy(ap["f"]).to("cuda", torch.float64)
        ga = torch.from_numpy(np.random.default_rng(4).normal(size=(Pa, S, S) + fa.shape[2:])).to("cuda")

        def tev(fn, reps=2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        adj = {"workload": "c4_adjoint_n32: %d points, 2 species (m = 1, 2), N = 32, M = 12, N_rho = 8" % Pa}
        df64 = None
        if "fp64" in aforms:
            p64 = B.Plan(ap["N"], ap["L"], ap["M"], ap["Nrho"], ap["masses"], ap["pairs"], "fp64", Pa, dev)
            Qa = p64.collide(fa)
            p64.backward(fa, ga)
            torch.cuda.synchronize()
            t_f = tev(lambda: p64.collide(fa, Qa))
            t_b = tev(lambda: p64.backward(fa, ga))
            df64, dw64 = p64.backward(fa, ga)
            del p64
            adj.update({"fp64_forward_ms": t_f, "fp64_backward_ms": t_b, "backward_over_forward": t_b / t_f,
                        "fp64_backward_evals_per_s": Pa * S * S / (t_b / 1e3)})
        if "fp32_tc" in aforms:
            adj.update(_tc_adjoint(ap, Pa, S, dev, fa, ga, tev, df64, dw64 if df64 is not None else None))
        if "fp64_backward_ms" in adj and "fp32_tc_backward_ms" in adj:
            adj["fp32_tc_backward_speedup_over_fp64"] = adj["fp64_backward_ms"] / adj["fp32_tc_backward_ms"]
        out["adjoint"] = adj

    # end to end through the host-buffer C-ABI call (pinned host memory)
    if not args.no_e2e:
        es = 8 if main == "fp64" else 4
        fh = torch.from_numpy(pb["f"]).to(plan.dtype).pin_memory()
        Qh = torch.empty(tuple(rec["Q"].shape), dtype=plan.dtype).pin_memory()
        plan.collide_host(fh, Qh)
        tot = 0.0
        for _ in range(rec["steps"]):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.collide_host(fh, Qh)
            tot += time.perf_counter() - t0
        out["e2e"] = {"value": world * evals * rec["steps"] / tot, "unit": UNIT,
                      "h2d_bytes_per_step": int(fh.numel() * es), "d2h_bytes_per_step": int(Qh.numel() * es)}

    # 256 uneven homogeneous relaxation problems (N in {24, 32, 48}, 2 or 3
    # species, M in {6, 12}, N_rho in {8, 16}): one collision call plus one
    # relaxation step of every problem per pass, run as separate calls, as a
    # graph of those calls, and as the batched work list (eager and captured)
    if not args.no_batch and main != "fp64" and world == 1:
        try:
            out["uneven_batch"] = uneven_batch(B, W, torch, np, main, dev, flush, stream, plan, rec)
        except (B.DgfsError, ValueError, RuntimeError) as e:  # reported; the headline line still prints
            out["uneven_batch"] = {"error": str(e)}
            torch.cuda.synchronize()

    # per-form throughput and error vs the oracle on a sampled subset of points
    sample_pts = [i for i in (0, 7, 15, 23) if i < P] if not args.quick else [0]
    Qo = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        cores = len(os.sched_getaffinity(0))
        O.set_threads(cores)
        prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
        t0 = time.perf_counter()
        Qo = prob.collide_all(pb["f"], points=sample_pts)
        dt = time.perf_counter() - t0
        n_ev = len(sample_pts) * S * S
        # one evaluation on one core: the single-thread figure
        O.set_threads(1)
        t1 = time.perf_counter()
        prob.pair(0, 1).collide(pb["f"][0, 0], pb["f"][0, 1])
        dt1 = time.perf_counter() - t1
        O.set_threads(cores)
        out["cpu_baseline"] = {"value": n_ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "%d points x %d pairs of the same workload (points %s), FP64, "
                                         "tables excluded" % (len(sample_pts), S * S, sample_pts),
                               "single_thread_value": 1.0 / dt1,
                               "single_thread_sample": "pair (0, 1) at point 0 on one core"}
    Qoh = None
    if Qo is not None and any(k.endswith("_hermitian") and "value" in r for k, r in forms.items()):
        Qoh = prob.collide_all_hermitian(pb["f"], points=sample_pts)
    out["forms"] = {}
    for form, r in forms.items():
        if "value" not in r:
            out["forms"][form] = r
            continue
        d = {"value": r["value"], "ms_per_step": r["ms_per_step"]}
        ref = Qoh if form.endswith("_hermitian") else Qo
        if ref is not None:
            Qg = r["Q"][sample_pts].double().cpu().numpy()
            d["rel_err_vs_oracle"] = float(np.abs(Qg - ref).max() / np.abs(ref).max())
            d["err_sample_points"] = sample_pts
            if form.endswith("_hermitian"):
                d["oracle"] = ("the oracle's declared Hermitian variant (Algorithm 2 with the Nyquist planes "
                               "removed); differs from the literal operator by the Nyquist content")
        out["forms"][form] = d
    return out


def alu_peaks(torch):
    """FP64 and FP32 (CUDA-core) GEMM throughput of the GPU through cuBLAS, as
    the measured reference points for the SIMT passes (TF32 tensor cores off
    for the FP32 figure).  Library kernels, reported beside the result only."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp64_gemm_tflops", torch.float64, 4096), ("fp32_simt_gemm_tflops", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record()
            for _ in range(reps):
                torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            out[name] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    out["source"] = "torch.matmul (cuBLAS) on this GPU, TF32 off"
    return out


def uneven_plans(B, W, torch, np, prec, dev, count=256):
    """The uneven relaxation workload as plans: problems with equal parameters
    share one plan as its points.  Returns (groups, plans, fs, Qs), groups[i]
    being the list of problems (dicts of workloads.relaxation_batch) whose
    data fs[i] holds, in order."""
    import collections

    inst = W.relaxation_batch(count)
    groups = collections.OrderedDict()
    for x in inst:
        groups.setdefault((x["N"], tuple(x["masses"]), x["M"], x["Nrho"], x["alpha"]), []).append(x)
    plans, fs, Qs = [], [], []
    for xs in groups.values():
        x = xs[0]
        pl = B.Plan(x["N"], x["L"], x["M"], x["Nrho"], x["masses"], x["pairs"], prec, len(xs), dev)
        fs.append(torch.from_numpy(np.concatenate([y["f"] for y in xs])).to("cuda", pl.dtype).contiguous())
        Qs.append(torch.empty(len(xs), pl.S, pl.S, pl.N, pl.N, pl.N, dtype=pl.dtype, device="cuda"))
        plans.append(pl)
    return list(groups.values()), plans, fs, Qs


def uneven_batch(B, W, torch, np, prec, dev, flush, stream, plan, rec, count=256, reps=5):
    """Timings of the batched work list on the uneven relaxation workload, and
    the work list's own device cost on the benchmark call (one instance)."""
    _, plans, fs, Qs = uneven_plans(B, W, torch, np, prec, dev, count)
    evals = sum(f.shape[0] * pl.S * pl.S for pl, f in zip(plans, fs))
    # algorithmic FLOPs of one pass (each problem at its own N, S, M, N_rho)
    aflops = sum(step_algorithmic_flops(pl.N, f.shape[0], pl.S, pl.M * pl.N_rho) for pl, f in zip(plans, fs))
    dt = 1e-3

    def timed(fn, reps=reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / reps

    def separate():
        for pl, f, Q in zip(plans, fs, Qs):
            pl.collide(f, Q)
            pl.relax_step(f, Q, dt)

    def launches(fn):
        n0 = sum(pl.launch_count() for pl in plans)
        fn()
        torch.cuda.synchronize()
        return sum(pl.launch_count() for pl in plans) - n0

    res = {"workload": "relaxation_batch: %d homogeneous problems, N in {24, 32, 48} with L = N/3.2, 2 or 3 "
                       "species (masses from {1, 2, 4}), M in {6, 12}, N_rho in {8, 16}, VHS or VSS, seeded "
                       "two-Maxwellian data (seed 5); one collision call + one relaxation step per problem "
                       "per pass" % count,
           "instances": count, "plans": len(plans), "evals_per_pass": evals, "precision": prec}
    t = timed(separate)
    res["algorithmic_flops_per_pass"] = aflops
    res["separate_calls"] = {"ms_per_pass": t, "evals_per_s": evals / (t / 1e3),
                             "alg_tflops": aflops / (t / 1e3) / 1e12, "launches": launches(separate)}
    g = B.dgfs_graph_capture([pl._h for pl in plans], [f.shape[0] for f in fs], fs, Qs, dt=dt)
    try:
        t = timed(lambda: B.dgfs_graph_launch(g, stream))
        res["graph_of_calls"] = {"ms_per_pass": t, "evals_per_s": evals / (t / 1e3),
                                 "alg_tflops": aflops / (t / 1e3) / 1e12, "launches": B.dgfs_graph_kernel_count(g)}
    finally:
        B.dgfs_graph_destroy(g)
    bt = B.Batch(plans, fs, Qs, dt)
    try:
        bt.set_schedule(1)
        t = timed(lambda: bt.launch(stream))
        res["batch_work_list"] = {"ms_per_pass": t, "evals_per_s": evals / (t / 1e3),
                                  "alg_tflops": aflops / (t / 1e3) / 1e12,
                                  "launches": launches(lambda: bt.launch(stream))}
        bt.set_schedule(0)
        t = timed(lambda: bt.launch(stream))
        res["batch"] = {"ms_per_pass": t, "evals_per_s": evals / (t / 1e3), "alg_tflops": aflops / (t / 1e3) / 1e12,
                        "launches": launches(lambda: bt.launch(stream))}
        cg = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.graph(cg, stream=cs):
            bt.launch(cs)
        t = timed(cg.replay)
        res["batch_graph"] = {"ms_per_pass": t, "evals_per_s": evals / (t / 1e3),
                              "alg_tflops": aflops / (t / 1e3) / 1e12}
        del cg
    finally:
        bt.close()
    for pl in plans:
        pl.check()
    del plans, fs, Qs
    # device cost of the work list itself: the benchmark call as a batch of one
    # instance against its plain launches (same kernels, default stage A variant)
    plan.set_kernel_variant(0)
    f, Q = rec["f"], rec["Q"]
    t_plain = timed(lambda: plan.collide(f, Q), reps=2 * reps)
    b1 = B.Batch([plan], [f], [Q])
    try:
        t_b1 = timed(lambda: b1.launch(stream), reps=2 * reps)
    finally:
        b1.close()
    res["one_instance"] = {"plain_ms": t_plain, "batch_ms": t_b1, "overhead": t_b1 / t_plain - 1.0}
    return res


def tc_executed_flops(name, info, P, S, RS, sigma=None):
    """Tensor-core FLOPs a kernel class executes per step (2 M N K per issued
    MMA, padded rows included): M = 128 data rows per CTA, N = 2N outputs,
    K = N (real input) or 2N (complex input), times the split products.
    Translates along an axis where the design direction has no component are
    the identity and are not issued (sigma: [M][3] design directions)."""
    N = int(info["N"])
    nt = int(info.get("nterms", 3)) or 3
    G = 128 // N
    NO, KR, KC = 2 * N, N, 2 * N
    gem = lambda K: 2.0 * 128 * NO * K * nt
    planes = -(-N // G)
    if sigma is None:
        live = [1.0, 1.0, 1.0]
    else:
        sg = [list(map(float, v)) for v in sigma]
        live = [sum(1 for v in sg if v[d] != 0.0) / len(sg) for d in range(3)]
        if N > 32:  # stage A skips the z-pass only where a row's z-pencil fits its prefetch registers
            live[2] = 1.0
    # translate sides stage A computes per step: same-species pairs compute the
    # A side only (their B side is the A side at the reflected direction)
    sides = 2 * S * S - S
    if name == "tc_stage_a":
        return sides * P * planes * RS * (live[2] * gem(KR) + live[1] * gem(KC))
    if name == "tc_stage_b":
        return S * S * P * (-(-N * N // 128)) * RS * (2 * live[0] + 1) * gem(KC)
    if name == "tc_stage_c":
        return S * S * P * planes * RS * 2 * gem(KC)
    if name == "tc_worklist":  # one launch runs all three stages
        return sum(tc_executed_flops(k, info, P, S, RS, sigma) for k in ("tc_stage_a", "tc_stage_b", "tc_stage_c"))
    return None


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the stage kernels of the
# 3xTF32 form on the slab workload, averaged over the four species-pair launches of one
# call, from a one-pass ncu capture at 24 points per launch (profiles/launches_c2_slab_n32_fp32_tc.md;
# stage A and B launches of the same-species pairs move about half of the others).
# A', B' and H are per point, so a launch over fewer points moves proportionally less.
NCU_TRAFFIC_24PT = {"tc_stage_a": 0.858e9, "tc_stage_b": 1.488e9, "tc_stage_c": 0.700e9}


def ncu_traffic(name, P, points_per_launch=None):
    """(bytes per launch, where the figure comes from), or (None, reason)."""
    if WORKLOAD != "c2_slab_n32" or name not in NCU_TRAFFIC_24PT:
        return None, "no ncu capture of this kernel"
    E = min(P, 24) if points_per_launch is None else points_per_launch
    return (NCU_TRAFFIC_24PT[name] * E / 24.0,
            "not measured in this run: one-pass ncu dram__bytes_read.sum + dram__bytes_write.sum at 24 points "
            "per launch, averaged over the species pairs%s" % ("" if E == 24 else ", scaled by %d/24 points" % E))


def step_algorithmic_bytes(N, P, S, RS, es=4):
    """Algorithmic HBM bytes of one step: f_p and f_q in and Q out per evaluation
    (es bytes per value) and each pair's b table (complex) read once."""
    n = N ** 3
    return S * S * P * 3.0 * n * es + S * S * RS * n * 2.0 * es


def alg_axis_flops(N):
    """One length-N pass of a 3-D transform over an N^3 grid: N^2 transforms of
    5 N log2 N flops (the radix-2 count the paper's FFTs would take)."""
    return 5.0 * N ** 3 * math.log2(N)


def tc_algorithmic_flops(name, N, P, S, RS):
    """Algorithmic FLOPs of one step's launches of a tensor-core stage kernel:
    per (point, pair, r, s), stage A does the z and y passes of both translates
    (4 axis passes), stage B the two x passes, the complex product and the
    forward x pass (3 passes + 6 N^3), stage C the forward y and z passes and the
    multiply-accumulate with w b (2 passes + 8 N^3); the 9 passes are the 3 x 3-D
    transforms of the (r, s) step of Algorithm 2."""
    a = alg_axis_flops(N)
    per = {"tc_stage_a": 4 * a, "tc_stage_b": 3 * a + 6.0 * N ** 3, "tc_stage_c": 2 * a + 8.0 * N ** 3,
           "tc_worklist": 9 * a + 14.0 * N ** 3}.get(name)
    return None if per is None else S * S * P * RS * per


def step_algorithmic_flops(N, P, S, RS):
    """The whole operator per step: (3 M N_rho + 2) 3-D transforms per evaluation,
    S forward transforms per point, ~28 flops per grid point per (r, s)."""
    t = 3 * alg_axis_flops(N)
    return S * S * P * ((3 * RS + 2) * t + 28.0 * RS * N ** 3) + S * P * t


def tc_roofline(name, info, P, S, RS, avg_s, peak, peak_src, launches_per_step, sigma=None):
    N = int(info["N"])
    alg = tc_algorithmic_flops(name, N, P, S, RS)
    exe = tc_executed_flops(name, info, P, S, RS, sigma)
    r = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak, "peak_source": peak_src,
         "achieved": alg / launches_per_step / avg_s / 1e12 if alg else None,
         "work_per_launch": alg / launches_per_step if alg else None,
         "work_unit": "algorithmic FLOPs: 5 N^3 log2 N per axis pass of a 3-D transform plus the method's "
                      "elementwise work (per (point, pair, r, s): stage A 4 passes, stage B 3 passes + 6 N^3, "
                      "stage C 2 passes + 8 N^3)"}
    if exe:
        ach = exe / launches_per_step / avg_s / 1e12
        r["executed_mma"] = {"achieved": ach, "frac": ach / peak, "work_per_launch": exe / launches_per_step,
                             "unit": "TFLOP/s",
                             "work_unit": "executed dense MMA FLOPs: every length-N pass as a 128 x 2N x K GEMM "
                                          "(K = N real or 2N complex input), all split products, identity "
                                          "translates not issued"}
    return r


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import numpy as np

    import oracle as O
    from paper_1903_04670_gb300 import workloads as W

    pb = W.make_problem(WORKLOAD)
    S = pb["f"].shape[1]
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    prob = O.Problem(pb["N"], pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    npts = max(1, cores // (S * S))
    pts = list(range(npts))
    for _ in range(args.warmup):
        prob.collide_all(pb["f"], points=pts[:1])
    t0 = time.perf_counter()
    for k in range(args.steps):
        prob.collide_all(pb["f"], points=pts)
    dt = time.perf_counter() - t0
    evals = args.steps * npts * S * S
    v = evals / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": v / PAPER_EVALS_PER_S,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "points": npts,
                       "evals_per_step": npts * S * S},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d points x %d pairs per step of the same workload, FP64, OpenMP "
                                       "over (point, pair)" % (npts, S * S)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _tc_adjoint(ap, Pa, S, dev, fa, ga, tev, df64, dw64):
    """The 3xTF32 plan's backward on the adjoint workload: its time against its
    forward, the per-kernel times of one profiled call, and (given the FP64
    plan's result) the relative differences of df and dL/d omega."""
    import torch
    from paper_1903_04670_gb300 import binding as B
    ptc = B.Plan(ap["N"], ap["L"], ap["M"], ap["Nrho"], ap["masses"], ap["pairs"], "fp32_tc", Pa, dev)
    fa32, ga32 = fa.float(), ga.float()
    Qt = ptc.collide(fa32)
    dft, dwt = ptc.backward(fa32, ga32)
    torch.cuda.synchronize()
    t_t = tev(lambda: ptc.collide(fa32, Qt), reps=5)
    t_tb = tev(lambda: ptc.backward(fa32, ga32), reps=3)
    # per-kernel-class times of one profiled backward call
    ptc.profile(True)
    ptc.backward(fa32, ga32)
    torch.cuda.synchronize()
    bprof = {k: round(v[1], 3) for k, v in ptc.profile_read().items()}
    ptc.profile(False)
    ne = Pa * S * S
    out = {"fp32_tc_forward_ms": t_t, "fp32_tc_backward_ms": t_tb, "fp32_tc_backward_over_forward": t_tb / t_t,
           "fp32_tc_backward_evals_per_s": ne / (t_tb / 1e3), "fp32_tc_backward_kernel_ms": bprof}
    if df64 is not None:
        out.update({"fp32_tc_vs_fp64_df_rel_err": float((dft.double() - df64).abs().max() / df64.abs().max()),
                    "fp32_tc_vs_fp64_domega_rel_err": float((dwt - dw64).abs().max() / dw64.abs().max()),
                    "note": "df and domega of both plans for the same seeded upstream gradient; the "
                            "tensor-core backward's inputs are the FP64 ones rounded to float32"})
    del ptc
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "fp32_tc", "tf32", "bf16x3"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-dg", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-peaks", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hermitian", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--points", type=int, default=None,
                    help="evaluate only the first POINTS spatial points (small cases for profiling)")
    ap.add_argument("--adjoint-points", type=int, default=None,
                    help="points of the adjoint workload (default: all 64; small cases for profiling)")
    ap.add_argument("--adjoint-forms", default="fp64,fp32_tc",
                    help="plans whose backward the adjoint section times: fp64, fp32_tc or both")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
