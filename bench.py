"""Benchmark: MW forward + inverse transforms/s at L = 2048, 16 maps (8 spin 0,
8 spin 2), complex Gaussian f_lm with E|f_lm|^2 = 1/(l+1)^2.

One step = the paper's round trip (Sec. V-D): the inverse transform of the
batch followed by the forward transform of its result, 2B transforms, each
call replayed as one captured CUDA graph.  Inputs (1.1 GB of f_lm, 2.1 GB of
maps) are larger than L2, so no flush is needed between steps.  value:
device-timed (CUDA events on the stream) with inputs resident in HBM.  Also
reported: separate forward and inverse rates, the fused forward + inverse of
independent batches that share one Delta recursion (mw_forward_inverse), and
e2e: the round trip through the C ABI with pinned host buffers, host<->device
copies inside the timed region.  The roofline entry
describes the dominant stage, timed live with the library's per-stage events.

--impl reference runs the FP64 CPU oracle (the only baseline this project has)
on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank transforms its own batch (weak scaling, no
data-path collective); value = all ranks' transforms / max rank time.
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

METRIC = "MW fwd+inv transforms/s at L=2048,B=16 (mixed vs FP64 GPU) at ≤1e-6 rel err"
L_BENCH, B_BENCH = 2048, 16
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# stage kernels in one round trip (inverse launches first), keyed by (L, B,
# precision, planes per launch, spin groups per contraction pass), from a
# 1-pass ncu capture of the headline round trip (bench.py --headline-only
# --tuning CHUNK,GROUPS,128) with the kernels as they are now; a stage or
# tuning absent here reports null.
TRAFFIC = {
    (2048, 16, "mixed", 512, 2): {
        "contract": [0.512e9, 2.808e9, 7.779e9, 13.679e9, 0.435e9, 2.507e9, 6.270e9, 11.810e9],
        "delta": [0.125e9, 1.220e9, 3.386e9, 6.624e9, 0.126e9, 1.220e9, 3.386e9, 6.624e9],
        "theta": [3.199e9, 2.101e9],
        "phi": [3.155e9, 3.247e9],
    },
}


def peaks():
    pk = {"hbm_gbs": 6794.8, "bf16_tflops": 1899.0, "bf16_tflops_sustained": 1700.8, "src": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            j = json.load(fh)
        pk.update({k: j[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained") if k in j})
        pk["src"] = "measured"
    except Exception:
        pass
    # FP64 peak: MEASURED_PEAKS.json has no FP64 entry; the figure is this
    # part's FP64 DFMA rate from an own microbenchmark, replaced by a DGEMM
    # measured in the same run when fp64_peak_live() succeeds.
    pk["fp64_tflops"] = 0.993
    pk["fp64_src"] = "own DFMA microbenchmark (constant)"
    return pk


def fp64_peak_live(dev):
    """FP64 throughput of torch.matmul (cuBLAS DGEMM, 4096^3, best of 3 after a
    warm-up) on this GPU, in TFLOP/s; None if it fails."""
    try:
        import torch
        n = 4096
        a = torch.randn(n, n, dtype=torch.float64, device=dev)
        b = torch.randn(n, n, dtype=torch.float64, device=dev)
        torch.matmul(a, b)
        torch.cuda.synchronize(dev)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    except Exception:
        return None


class ClockSampler:
    def __init__(self, gpu_index):
        self.idx, self.proc, self.lines = gpu_index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + CLOCK_Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_max(x, device=None):
    """Max of x over the ranks of the default process group (x itself when
    there is none): the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_value(world, batch, steps, seconds):
    """Transforms/s of the whole job: each of the `world` ranks runs `steps`
    steps of 2 * batch transforms (forward + inverse) in `seconds` (max over
    ranks).  Weak scaling: the per-rank work does not depend on world."""
    return world * 2 * batch * steps / seconds


def contraction_units(L, spins):
    """(l, m, m' >= 0, map) real-kernel x complex multiply-accumulates of one
    direction's Delta contraction (4 flops each)."""
    tot = 0
    for s in spins:
        for l in range(abs(s), L):
            tot += (2 * l + 1) * (l + 1)
    return tot


def risbo_units(L):
    """Stencil evaluations of one Risbo sweep that the pi/2 symmetries leave
    necessary: the lower triangle of the half-integer plane (l entries a side)
    and of the integer plane (l + 1) for every l = 1 .. L-1 (7 flops each:
    4 multiplies and 3 adds)."""
    tot = 0
    for l in range(1, L):
        tot += l * (l + 1) // 2 + (l + 1) * (l + 2) // 2
    return tot


def risbo_ff_instructions(L):
    """FP32 instructions of one float-float Risbo sweep (the mixed paths): per
    octant element of a half-step plane 4 float-float operations (one product
    at 7 FP32 instructions, three multiply-adds at 15) = 52, per integer-plane
    element 5 (two products, three multiply-adds) = 59."""
    tot = 0
    for l in range(1, L):
        tot += 52 * (l * (l + 1) // 2) + 59 * ((l + 1) * (l + 2) // 2)
    return tot


def error_report(x, ref, L, n_bands=8):
    """Relative errors of f_lm tensors [B][L*L] (any device): rel_max =
    max|x - ref| / max|ref|, rel_rms = ||x - ref|| / ||ref||, and rel_max per
    band of l (n_bands equal bands of l, each relative to the band's own
    max|ref|), as floats."""
    import torch
    d = (x - ref).abs().reshape(-1, L * L).to(torch.float64)
    r = ref.abs().reshape(-1, L * L).to(torch.float64)
    out = {"rel_max": float(d.max() / r.max().clamp_min(1e-300)),
           "rel_rms": float(d.norm() / r.norm().clamp_min(1e-300))}
    ell = torch.arange(L * L, device=d.device, dtype=torch.float64).sqrt().floor().to(torch.int64)
    edges = [round(k * L / n_bands) for k in range(n_bands + 1)]
    bands = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        if hi <= lo:
            continue
        sel = (ell >= lo) & (ell < hi)
        bands.append({"l": [lo, hi], "rel_max": float(d[:, sel].max() / r[:, sel].max().clamp_min(1e-300))})
    out["bands"] = bands
    return out


def tn_units(L):
    """Quarter-plane elements of one Trapani-Navaza pass over the planes
    l < L: every column m of plane l recurses over m' = l .. 0."""
    return sum((l + 1) ** 2 for l in range(L))


def contraction_bytes(L, B, precision):
    """Algorithmic HBM bytes of both contractions of one round trip: each
    staged plane read once per direction (FP32 quarter planes on the mixed
    paths, FP64 on the FP64 path), the forward's G+ read and f_lm written, the
    inverse's N_l f_lm read and F+ written."""
    M = 2 * L - 1
    plane_b = 4 if precision != "fp64" else 8
    planes = plane_b * tn_units(L)
    gp = B * M * L * (8 if precision != "fp64" else 16)
    flm_in = B * L * L * (8 if precision != "fp64" else 16)
    fplus = B * M * L * 16
    flm_out = B * L * L * 16
    return 2 * planes + gp + flm_out + flm_in + fplus


def delta_roofline(recursion, L, seconds, pk, fp32_issue, n_sm, mhz):
    """Roofline entry of the Wigner-plane stage (two recursions per round trip)
    for the recursion that ran: "risbo_f64" (double state, FP64 pipe),
    "risbo_ff" (float-float state, FP32 pipe) or "tn" (Trapani-Navaza,
    float-float, FP32 pipe and FP32 staging writes)."""
    sweeps = 2
    issue_src = f"{n_sm} SMs x 128 FP32 lanes x {mhz:.0f} MHz (median SM clock in the timed region)"
    if recursion == "tn":
        units = sweeps * tn_units(L)
        instr = 25 * units          # float-float: 2/b times the integer m (3), a product (7), a multiply-add (15)
        nbytes = 4 * units          # every quarter-plane element staged once in FP32
        t_i, t_b = instr / fp32_issue, nbytes / (pk["hbm_gbs"] * 1e9)
        issue = {"achieved": instr / seconds / 1e12, "peak": fp32_issue / 1e12, "unit": "T instr/s",
                 "frac": t_i / seconds, "work": "25 FP32 instructions per quarter-plane element",
                 "peak_src": issue_src}
        hbm = {"achieved": nbytes / seconds / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": t_b / seconds,
               "work": "4 bytes (FP32 staging) per quarter-plane element", "peak_src": pk["src"]}
        out = dict(issue, bound="alu") if t_i >= t_b else dict(hbm, bound="hbm")
        out.update(kernel="k_tn_planes", recursion="Trapani-Navaza", fp32_issue=issue, hbm=hbm,
                   floor_ms=1e3 * max(t_i, t_b))
        return out
    fl = sweeps * risbo_units(L) * 7
    a = fl / seconds / 1e12
    out = {"bound": "alu", "achieved": a, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
           "frac": a / pk["fp64_tflops"], "kernel": "k_risbo_sweep", "recursion": "Risbo",
           "peak_src": pk.get("fp64_src", "own FP64 DFMA microbenchmark"),
           "work": "7 flops per octant element of each half-step plane",
           "frac_quarter_plane_units": sweeps * 7.0 * L ** 3 / seconds / 1e12 / pk["fp64_tflops"],
           "floor_ms": 1e3 * fl / (pk["fp64_tflops"] * 1e12)}
    if recursion == "risbo_ff":
        instr = sweeps * risbo_ff_instructions(L)
        out["arith"] = "float-float on the FP32 pipe (FP64-equivalent flops above)"
        out["fp32_issue"] = {"achieved": instr / seconds / 1e12, "peak": fp32_issue / 1e12, "unit": "T instr/s",
                             "frac": instr / fp32_issue / seconds,
                             "work": "52 / 59 FP32 instructions per half / integer octant element",
                             "peak_src": issue_src}
        out["floor_ms"] = 1e3 * instr / fp32_issue
    return out


def fp64_rate_delta_stage(L, t_d, fp64_tflops, tc_flops, tc_peak, c_bytes, hbm_gbs):
    """The Delta stage (recursion + contractions, t_d seconds per round trip)
    against the formula that counts the recursion at the FP64 rate: max(7
    flops per element of two recursions / FP64 peak, products / tensor peak,
    bytes / HBM), with the recursion's elements counted as the octant that
    the pi/2 symmetries leave and, second, as L^3 per sweep (quarter plane)."""
    sweeps = 2
    rec_oct = sweeps * risbo_units(L) * 7 / (fp64_tflops * 1e12)
    rec_q = sweeps * 7.0 * L ** 3 / (fp64_tflops * 1e12)
    rest = max(tc_flops / (tc_peak * 1e12), c_bytes / (hbm_gbs * 1e9))
    return {"frac": max(rec_oct, rest) / t_d, "frac_quarter_plane_units": max(rec_q, rest) / t_d,
            "roofline_ms": 1e3 * max(rec_oct, rest), "roofline_ms_quarter_plane_units": 1e3 * max(rec_q, rest),
            "what": "recursion counted at the FP64 rate (7 flops per element) whatever arithmetic runs it"}


def fft_stage_bytes(L, B, precision):
    """Algorithmic HBM bytes of the FFT stages of one round trip (inverse +
    forward): every stage boundary written once and read once."""
    M = 2 * L - 1
    nmw = (L - 1) * M + 1
    cf = 16 if precision == "fp64" else 8       # G_m(theta_t) buffers
    gp_f = 16 if precision == "fp64" else 8     # G+ (forward contraction input)
    phi = B * (nmw * 16 + M * L * cf) * 2       # phi forward + phi inverse
    theta = B * (M * L * cf + M * L * gp_f) + B * (M * L * 16 + M * L * cf)  # theta forward + theta inverse
    return {"phi": phi, "theta": theta}


def timed_calls(fn, n, stream, dev):
    """n calls of fn bracketed by barriers and device syncs, CUDA events on the
    call stream around each; returns (total ms, max over ranks; per-call ms)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    rank_barrier()
    torch.cuda.synchronize(dev)
    for i in range(n):
        ev[i].record(stream)
        fn()
    ev[n].record(stream)
    torch.cuda.synchronize(dev)
    rank_barrier()
    each = [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
    return rank_max(ev[0].elapsed_time(ev[n]), dev), each


def rel_errors(x, ref):
    """rel_max = max|x - ref| / max|ref| and rel_rms = ||x - ref|| / ||ref||."""
    d = (x - ref).abs()
    return {"rel_max": float(d.max() / ref.abs().max().clamp_min(1e-300)),
            "rel_rms": float(d.norm() / ref.abs().norm().clamp_min(1e-300))}


def stage_breakdown(plan, call, n, dev):
    """Per-stage milliseconds per call (the library's stage events, graphs off)
    and kernel launches per call."""
    import torch
    plan.set_timing(True)
    plan.stage_times(reset=True)
    nl = 0
    for _ in range(n):
        nl = call()
    torch.cuda.synchronize(dev)
    st = {k: v[0] / n for k, v in plan.stage_times(reset=True).items()}
    plan.set_timing(False)
    return st, nl


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1110_6298_gb300 import build as lib_build
    from paper_1110_6298_gb300 import mw, workloads as wl

    if rank == 0 or world == 1:
        lib_build.build()
    rank_barrier()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = wl.workload_l2048_b16(L=args.L)
    L, spins = w["L"], w["spins"]
    B = len(spins)
    nmw = mw.map_size(L)
    flm_h = torch.from_numpy(np.stack(w["flm"]))
    flm = flm_h.to(dev)
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    timed = lambda fn, n: timed_calls(fn, n, stream, dev)  # noqa: E731

    def roundtrip_arm(plan, out_maps, out_flm):
        """Warm up, then time K graph-replayed round trips (inverse of the
        batch, forward of the result) of `plan`."""
        def rt():
            plan.inverse(flm, out=out_maps)
            plan.forward(out_maps, out=out_flm)
        for _ in range(W):
            rt()
        torch.cuda.synchronize(dev)
        plan.sync()
        return timed(rt, K)

    def breakdown(plan, out_maps, out_flm):
        def call():
            plan.inverse(flm, out=out_maps)
            n = plan.last_launches
            plan.forward(out_maps, out=out_flm)
            return n + plan.last_launches
        return stage_breakdown(plan, call, 2, dev)

    # ---- the headline: mixed precision, whole calls replayed as CUDA graphs,
    # the plan's launch cuts chosen by the library's autotuner (a search over
    # planes per launch, spin groups per contraction pass and Trapani-Navaza
    # block size, timed on this GPU before the timed region)
    t_tune = time.perf_counter()
    plan = mw.Plan(L, spins, precision=args.precision, graph=True,
                   autotune=not (args.no_autotune or args.tuning))
    if args.tuning:
        plan.set_tuning(*[int(x) for x in args.tuning.split(",")])
    t_tune = time.perf_counter() - t_tune
    tuning = plan.tuning
    maps = torch.empty((B, nmw), dtype=torch.complex128, device=dev)
    out = torch.empty_like(flm)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, each = roundtrip_arm(plan, maps, out)
    ck = clocks.stop()
    value = whole_job_value(world, B, K, ms / 1e3)
    err_report = error_report(out, flm, L)
    stages, launches_per_step = breakdown(plan, maps, out)

    # ---- the plain FP64 GPU path on the identical workload and protocol
    fp64_line = None
    acc = {}
    if args.precision != "fp64" and not args.no_fp64_arm and not args.headline_only:
        p64 = mw.Plan(L, spins, precision="fp64", graph=True)
        maps64 = torch.empty_like(maps)
        out64 = torch.empty_like(out)
        ms64, each64 = roundtrip_arm(p64, maps64, out64)
        st64, _ = breakdown(p64, maps64, out64)
        v64 = whole_job_value(world, B, K, ms64 / 1e3)
        # the mixed path against the FP64 path (itself pinned to the FP64
        # oracle at 1e-12) on every output: the inverse of the batch, and the
        # forward of the FP64 maps, per band of l
        plan.inverse(flm, out=maps)
        acc["inverse_vs_fp64"] = rel_errors(maps, maps64)
        fm = torch.empty_like(out)
        plan.forward(maps64, out=fm)
        p64.forward(maps64, out=out64)
        acc["forward_vs_fp64"] = error_report(fm, out64, L)
        p64.inverse(flm, out=maps64)
        p64.forward(maps64, out=out64)
        rt64 = error_report(out64, flm, L)
        p64.close()
        del p64, maps64, out64, fm
        fp64_line = {"value": v64, "unit": "transforms/s", "ms_per_step": ms64 / K,
                     "ms_per_step_median": statistics.median(each64), "steps": K, "warmup": W,
                     "roundtrip_rel_max": rt64["rel_max"], "roundtrip_rel_rms": rt64["rel_rms"],
                     "stage_ms_per_step": st64,
                     "what": "the same round trip on an MW_PREC_FP64 plan (FP64 FFTs, FP64 Risbo sweep, "
                             "DMMA contraction), graph-replayed, CUDA events, same steps"}
    torch.cuda.synchronize(dev)

    if args.headline_only:
        return headline_only_result(args, world, value, ms, K, W, L, B, stages, launches_per_step, ck, err_report,
                                    tuning)

    # ---- separate forward and inverse rates
    inv_ms, _ = timed(lambda: plan.inverse(flm, out=maps), K)
    fwd_ms, _ = timed(lambda: plan.forward(maps, out=out), K)
    plan.forward(maps, out=out)

    # ---- fused forward + inverse of independent batches (one shared recursion)
    flm2 = torch.from_numpy(np.stack(wl.workload_l2048_b16(L=args.L, seed=14)["flm"])).to(dev)
    maps_in = plan.inverse(flm2)
    fu_flm, fu_map = torch.empty_like(flm), torch.empty_like(maps)
    plan.forward_inverse(maps_in, flm, fu_flm, fu_map)
    fu_ms, _ = timed(lambda: plan.forward_inverse(maps_in, flm, fu_flm, fu_map), K)
    fu_err = float((fu_flm - flm2).abs().max().item() / flm2.abs().max().item())
    del flm2, maps_in, fu_flm, fu_map

    # ---- quadrature rule (Sec. IV-F): integrals of B maps in the quadrature layout
    gq = torch.Generator(device=dev)
    gq.manual_seed(11106298)
    mq = torch.randn((B, mw.quadrature_size(L)), dtype=torch.complex128, device=dev, generator=gq)
    qout = torch.empty(B, dtype=torch.complex128, device=dev)
    plan.quadrature(mq, out=qout)
    q_ms, _ = timed(lambda: plan.quadrature(mq, out=qout), K)
    q_gbs = mq.numel() * 16 * K / (q_ms / 1e3) / 1e9
    del mq

    # ---- real signals (Sec. IV-G): B real spin-0 maps, two per complex transform
    rplan = mw.RealPlan(L, B, precision=args.precision, graph=True)
    cr = torch.from_numpy(np.stack([wl.uniform_flm_real(wl.rng(3300 + b), L) for b in range(B)])).to(dev)
    rmap = torch.empty((B, nmw), dtype=torch.float64, device=dev)
    rout = torch.empty_like(cr)

    def real_roundtrip():
        rplan.inverse(cr, out=rmap)
        rplan.forward(rmap, out=rout)

    for _ in range(2):
        real_roundtrip()
    rplan.sync()
    r_err = float((rout - cr).abs().max().item() / cr.abs().max().item())
    r_ms, _ = timed(real_roundtrip, K)
    rplan.close()
    del rplan, cr, rmap, rout

    # ---- the same round trip with Risbo's recursion for the Wigner planes
    rb_line = None
    if args.precision != "fp64":
        rb = mw.Plan(L, spins, precision=args.precision, graph=True, delta="risbo")
        rb_out = torch.empty_like(flm)
        rb_ms, _ = roundtrip_arm(rb, maps, rb_out)
        rb_err = float((rb_out - flm).abs().max().item() / flm.abs().max().item())
        rb_stages, _ = breakdown(rb, maps, rb_out)
        rb.close()
        del rb, rb_out
        rb_line = {"value": whole_job_value(world, B, K, rb_ms / 1e3), "unit": "transforms/s",
                   "ms_per_step": rb_ms / K, "rel_err": rb_err, "stage_ms_per_step": rb_stages,
                   "what": "the same round trip with Risbo's recursion (MW_FLAG_DELTA_RISBO)"}

    # ---- a batch of one spin: B spin-0 maps with the headline's tuning; with
    # two spin groups per contraction pass the two groups of 8 maps share one
    # A operand (one N = 64 MMA per split product)
    os_line = None
    if args.precision != "fp64" and not args.no_configs:
        g1 = wl.rng(41)
        f1 = torch.from_numpy(np.stack([wl.gaussian_flm(g1, L, 0, wl.cl_red) for _ in range(B)])).to(dev)
        p1 = mw.Plan(L, [0] * B, precision=args.precision, graph=True)
        p1.set_tuning(tuning["chunk"], tuning["groups"], tuning["tn_threads"])
        o1 = torch.empty_like(f1)

        def rt_1():
            p1.inverse(f1, out=maps)
            p1.forward(maps, out=o1)
        for _ in range(W):
            rt_1()
        torch.cuda.synchronize(dev)
        p1.sync()
        os_ms, _ = timed(rt_1, K)
        os_err = float((o1 - f1).abs().max().item() / f1.abs().max().item())

        def call_1():
            p1.inverse(f1, out=maps)
            n = p1.last_launches
            p1.forward(maps, out=o1)
            return n + p1.last_launches
        os_stages, _ = stage_breakdown(p1, call_1, 2, dev)
        p1.close()
        del p1, f1, o1
        os_line = {"value": whole_job_value(world, B, K, os_ms / 1e3), "unit": "transforms/s",
                   "ms_per_step": os_ms / K, "rel_err": os_err, "stage_ms_per_step": os_stages,
                   "what": f"the same round trip on {B} spin-0 maps (one spin: the two spin groups of a "
                           "contraction pass share one A operand), the headline's tuning"}

    # ---- a prime 2L-1: L = 2047 (4093) runs its ring and theta DFTs by
    # Bluestein's convolution; its phi + theta time against L = 2048's
    pr_line = None
    if L == 2048 and not args.no_configs:
        wp = wl.workload_l2048_b16(L=2047)
        fp = torch.from_numpy(np.stack(wp["flm"])).to(dev)
        pp = mw.Plan(2047, spins, precision=args.precision, graph=True)
        mp = torch.empty((B, mw.map_size(2047)), dtype=torch.complex128, device=dev)
        op = torch.empty_like(fp)

        def rt_p():
            pp.inverse(fp, out=mp)
            pp.forward(mp, out=op)
        for _ in range(W):
            rt_p()
        torch.cuda.synchronize(dev)
        pr_ms, _ = timed(rt_p, K)
        pr_err = float((op - fp).abs().max().item() / fp.abs().max().item())
        pp.set_timing(True)
        pp.stage_times(reset=True)
        for _ in range(2):
            pp.inverse(fp, out=mp)
            pp.forward(mp, out=op)
        torch.cuda.synchronize(dev)
        pr_st = {k: v[0] / 2 for k, v in pp.stage_times(reset=True).items()}
        pr_line = {"value": whole_job_value(world, B, K, pr_ms / 1e3), "unit": "transforms/s",
                   "ms_per_step": pr_ms / K, "rel_err": pr_err, "bluestein": pp.fft_bluestein,
                   "stage_ms_per_step": pr_st,
                   "phi_theta_ms_vs_l2048": (pr_st["phi"] + pr_st["theta"]) / (stages["phi"] + stages["theta"]),
                   "what": "the same round trip at L=2047, whose 2L-1 = 4093 is prime: ring and theta DFTs by "
                           "Bluestein's convolution of length 8192"}
        pp.close()
        del pp, fp, mp, op

    # ---- end to end: the round trip through the C ABI with pinned host
    # buffers, host<->device copies inside the timed region, every step
    flm_pin = flm_h.pin_memory()
    map_pin = torch.empty((B, nmw), dtype=torch.complex128).pin_memory()
    out_pin = torch.empty_like(flm_pin).pin_memory()
    plan.inverse(flm_pin, out=map_pin)
    plan.forward(map_pin, out=out_pin)
    rank_barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_each = []
    for _ in range(K):
        ts = time.perf_counter()
        plan.inverse(flm_pin, out=map_pin)
        plan.forward(map_pin, out=out_pin)
        e2e_each.append(1e3 * (time.perf_counter() - ts))
    torch.cuda.synchronize(dev)
    t_e2e = rank_max(time.perf_counter() - t0, dev)
    e2e_value = whole_job_value(world, B, K, t_e2e)
    bytes_flm = B * L * L * 16
    bytes_map = B * nmw * 16
    e2e_err = float((out_pin - flm_h).abs().max() / flm_h.abs().max())
    del flm_pin, map_pin, out_pin

    # ---- the other configurations and the paper's accuracy protocol
    configs = None if args.no_configs or L != 2048 else config_lines(args, mw, wl, dev, stream, world)
    sweep = None if args.no_configs or L != 2048 else accuracy_sweep(args, mw, wl, dev, acc)

    # ---- rooflines per round trip: every stage against its own bound
    pk = peaks()
    f64 = fp64_peak_live(dev)
    if f64:
        pk["fp64_tflops"], pk["fp64_src"] = f64, "torch.matmul float64 4096^3 (cuBLAS DGEMM), this run"
    pk_hbm = pk["hbm_gbs"]
    fb = fft_stage_bytes(L, B, args.precision)
    t = {k: v / 1e3 for k, v in stages.items()}  # seconds per round trip
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (ck or {}).get("sm_mhz") or 2070.0
    fp32_issue = n_sm * 128 * mhz * 1e6  # FP32 instructions per second
    recursion = "risbo_f64" if args.precision == "fp64" else "tn"
    stage_roof = {}
    if t["delta"] > 0:
        stage_roof["delta"] = delta_roofline(recursion, L, t["delta"], pk, fp32_issue, n_sm, mhz)
    tc_flops = 2 * contraction_units(L, spins) * 4
    c_bytes = contraction_bytes(L, B, args.precision)
    tc_peak = {"mixed": pk["bf16_tflops"], "mixed_tf32": pk["bf16_tflops"] * 0.5}.get(args.precision,
                                                                                       pk["fp64_tflops"])
    if t["contract"] > 0:
        a_t = tc_flops / t["contract"] / 1e12
        a_b = c_bytes / t["contract"] / 1e9
        t_tensor, t_hbm = tc_flops / (tc_peak * 1e12), c_bytes / (pk_hbm * 1e9)
        kern = {"mixed": "k_tc2 (BF16x3 pipeline, both directions)",
                "mixed_tf32": "k_tc_forward/k_tc_inverse (TF32x3)"}.get(args.precision, "k_dmma_forward/k_dmma_inverse")
        tensor = {"achieved": a_t, "peak": tc_peak, "unit": "TFLOP/s", "frac": a_t / tc_peak,
                  "work": "4 flops per (l, m, m' >= 0, map) multiply-add, both directions",
                  "peak_src": {"mixed": "measured (MEASURED_PEAKS.json bf16 dense burst)",
                               "mixed_tf32": "measured BF16 peak x nominal TF32/BF16 ratio"}.get(
                      args.precision, pk["fp64_src"])}
        hbm = {"achieved": a_b, "peak": pk_hbm, "unit": "GB/s", "frac": a_b / pk_hbm,
               "work": "staged planes read once per direction, G+ / N_l f_lm read, f_lm / F+ written",
               "peak_src": pk["src"]}
        if t_hbm >= t_tensor:
            stage_roof["contract"] = dict(hbm, bound="hbm", kernel=kern, tensor=tensor)
        else:
            stage_roof["contract"] = dict(tensor, bound="tensor", kernel=kern, hbm=hbm)
    for k in ("theta", "phi"):
        if t[k] > 0:
            a = fb[k] / t[k] / 1e9
            stage_roof[k] = {"bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                             "frac": a / pk["hbm_gbs"], "peak_src": pk["src"]}
    # the Delta stage (recursion + contractions) against the largest of its floors
    t_d = t["delta"] + t["contract"]
    rec_floor = stage_roof["delta"]["floor_ms"] / 1e3 if "delta" in stage_roof else 0.0
    bounds = (rec_floor, tc_flops / (tc_peak * 1e12), c_bytes / (pk_hbm * 1e9))
    delta_stage = {"ms": 1e3 * t_d, "roofline_ms": 1e3 * max(bounds), "frac": max(bounds) / t_d,
                   "recursion": recursion,
                   "bounds_ms": {"recursion": 1e3 * bounds[0], "contraction_tensor": 1e3 * bounds[1],
                                 "contraction_hbm": 1e3 * bounds[2]},
                   "fp64_rate_formula": fp64_rate_delta_stage(L, t_d, pk["fp64_tflops"], tc_flops, tc_peak, c_bytes,
                                                           pk_hbm)}
    if rb_line is not None:
        rb_line["delta_roofline"] = delta_roofline("risbo_ff", L, rb_line["stage_ms_per_step"]["delta"] / 1e3, pk,
                                                   fp32_issue, n_sm, mhz)
    dom = max(("delta", "contract", "theta", "phi"), key=lambda k: stages[k])
    traffic = TRAFFIC.get((L, B, args.precision, tuning["chunk"], tuning["groups"])) if recursion == "tn" else None
    for k, v in (traffic or {}).items():
        if k in stage_roof and v:
            stage_roof[k]["traffic"] = sum(v) / len(v)  # DRAM bytes per launch, averaged over the launches
            stage_roof[k]["traffic_per_step"] = sum(v)
    roof = dict(stage_roof[dom])
    roof["stage"] = dom
    roof.setdefault("traffic", None)
    err = err_report["rel_max"]
    meets = err <= 1e-6 and all(v["rel_max"] <= 1e-6 for v in acc.values())
    result = {
        "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f64+f32+bf16", "mixed_tf32": "f64+f32+tf32"}[args.precision],
        "data": "synthetic (seeded complex Gaussian f_lm, C_l=1/(l+1)^2)",
        "config": {"workload": f"MW round trip (inverse then forward) L={L}, B={B} (8 maps s=0, 8 maps s=2)",
                   "L": L, "batch": B, "precision": args.precision,
                   "l2_flush": "inputs larger than L2", "graph": True, "parallelism": f"replicas x{world}",
                   "tuning": dict(tuning, autotuned=not (args.no_autotune or args.tuning),
                                  search_s=round(t_tune, 2))},
        "gpu_launches": launches_per_step * K,
        "e2e": {"value": e2e_value, "unit": "transforms/s", "h2d_bytes_per_step": bytes_flm + bytes_map,
                "d2h_bytes_per_step": bytes_map + bytes_flm, "steps": K, "rel_err": e2e_err,
                "ms_each_step": [round(x, 1) for x in e2e_each]},
        "roofline": roof,
        "clocks": ck,
        "stage_roofline": stage_roof,
        "delta_stage": delta_stage,
        "quadrature": {"value": world * B * K / (q_ms / 1e3), "unit": "integrals/s", "ms_per_call": q_ms / K,
                       "what": f"MW quadrature rule, {B} maps of L(L-1)+1 samples per call",
                       "roofline": {"bound": "hbm", "achieved": q_gbs, "peak": pk_hbm, "unit": "GB/s",
                                    "frac": q_gbs / pk_hbm, "kernel": "k_quad_partial"}},
        "real": {"value": whole_job_value(world, B, K, r_ms / 1e3), "unit": "transforms/s",
                 "ms_per_step": r_ms / K, "rel_err": r_err,
                 "what": f"round trip of {B} real spin-0 maps (Sec. IV-G), uniform[-1,1] coefficients"},
        "risbo": rb_line,
        "one_spin": os_line,
        "prime_l2047": pr_line,
        "fused": {"value": whole_job_value(world, B, K, fu_ms / 1e3), "unit": "transforms/s",
                  "ms_per_step": fu_ms / K, "rel_err": fu_err,
                  "what": "mw_forward_inverse: forward of B maps and inverse of B independent f_lm, one recursion"},
        "forward_rate": whole_job_value(world, B, K, fwd_ms / 1e3) / 2,
        "inverse_rate": whole_job_value(world, B, K, inv_ms / 1e3) / 2,
        "configs": configs,
        "paper_accuracy_protocol": sweep,
        "stage_ms_per_step": stages,
        "ms_per_step_median": statistics.median(each),
        "roundtrip_errors": err_report,
        "mixed_vs_fp64_errors": acc or None,
        "fp64_gpu": fp64_line,
        "speedup_mixed_over_fp64": (value / fp64_line["value"]) if fp64_line else None,
        "roundtrip_rel_err": err,
        "meets_1e-6": meets,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, quick=False)
        result = {**{k: v for k, v in result.items() if k in HEAD_KEYS}, "cpu_baseline": cb,
                  **{k: v for k, v in result.items() if k not in HEAD_KEYS}}
    return result


def headline_only_result(args, world, value, ms, K, W, L, B, stages, launches_per_step, ck, err_report, tuning):
    """The line of a --headline-only run (for profiling: the headline round
    trips and the per-stage breakdown, no secondary arms)."""
    return {"metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f64+f32+bf16", "mixed_tf32": "f64+f32+tf32"}[args.precision],
            "data": "synthetic (seeded complex Gaussian f_lm, C_l=1/(l+1)^2)",
            "config": {"workload": f"MW round trip (inverse then forward) L={L}, B={B} (8 maps s=0, 8 maps s=2)",
                       "L": L, "batch": B, "precision": args.precision, "graph": True,
                       "tuning": dict(tuning, autotuned=not (args.no_autotune or args.tuning)),
                       "headline_only": True},
            "gpu_launches": launches_per_step * K, "clocks": ck, "stage_ms_per_step": stages,
            "roundtrip_rel_err": err_report["rel_max"]}


HEAD_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "gpu_launches", "e2e", "roofline", "clocks")


def config_lines(args, mw, wl, dev, stream, world):
    """The other workloads as secondary lines: FP64-path and mixed-path
    transforms/s (graph-replayed round trips, or forward + adjoint for the
    gradient workload) and errors against the FP64 oracle (on every map, or on
    the maps named in `oracle_maps`) and of the mixed path against the FP64
    path on every output."""
    import numpy as np
    import torch

    import oracle
    n_t = max(3, min(args.steps, 10))
    out = {}

    def rate(fn, n_transforms):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        ms, _ = timed_calls(fn, n_t, stream, dev)
        return world * n_transforms * n_t / (ms / 1e3)

    # configs 1 and 2: one map, FP64 inverse + forward against the oracle
    for name, wk in (("c1_L32_s0", wl.workload_small()), ("c2_L256_s2", wl.workload_l256_s2())):
        L, s = wk["L"], wk["spins"][0]
        f = torch.from_numpy(np.stack(wk["flm"])).to(dev)
        ref_map = oracle.inverse(wk["flm"][0], L, s)
        line = {}
        for prec in ("fp64", "mixed"):
            p = mw.Plan(L, [s], precision=prec, graph=True)
            m = torch.empty((1, mw.map_size(L)), dtype=torch.complex128, device=dev)
            b = torch.empty_like(f)

            def rt():
                p.inverse(f, out=m)
                p.forward(m, out=b)
            r = rate(rt, 2)
            mm = m.cpu().numpy()[0]
            ref_back = oracle.forward(mm, L, s)
            line[prec] = {"transforms_per_s": r,
                          "inverse_vs_oracle": rel_np(mm, ref_map),
                          "forward_vs_oracle": rel_np(b.cpu().numpy()[0], ref_back),
                          "roundtrip_max_abs": float(np.max(np.abs(b.cpu().numpy()[0] - wk["flm"][0])))}
            p.close()
        out[name] = line

    # config 3: 64 maps of uneven L and spin in one ragged plan, one graph launch per call
    wk = wl.workload_ragged()
    Ls, ss = wk["Ls"], wk["spins"]
    f = torch.from_numpy(np.concatenate(wk["flm"])).to(dev)
    line, maps_by = {}, {}
    for prec in ("fp64", "mixed"):
        p = mw.RaggedPlan(Ls, ss, precision=prec, graph=True)
        m = torch.empty(p._nmap, dtype=torch.complex128, device=dev)
        b = torch.empty_like(f)

        def rt():
            p.inverse(f, out=m)
            p.forward(m, out=b)
        line[prec] = {"transforms_per_s": rate(rt, 2 * len(Ls)),
                      "roundtrip": rel_errors(b, f)}
        maps_by[prec] = (m.clone(), p.map_offsets)
        p.close()
    line["mixed"]["inverse_vs_fp64"] = rel_errors(maps_by["mixed"][0], maps_by["fp64"][0])
    seen, worst = set(), 0.0
    mm, mo = maps_by["mixed"][0].cpu().numpy(), maps_by["mixed"][1]
    for b, (L, s) in enumerate(zip(Ls, ss)):
        if L in seen:
            continue
        seen.add(L)
        worst = max(worst, rel_np(mm[mo[b]:mo[b] + mw.map_size(L)], oracle.inverse(wk["flm"][b], L, s))["rel_max"])
    line["mixed"]["inverse_vs_oracle_rel_max"] = worst
    line["oracle_maps"] = "one map of each band limit"
    out["c3_ragged_64"] = line

    # config 5: L = 512, 32 spin-0 maps of i.i.d. samples; the gradient step
    # forward + forward adjoint (the backward of the loss)
    wk = wl.workload_grad_l512_b32()
    L = wk["L"]
    x = torch.from_numpy(np.stack(wk["maps"])).to(dev)
    tg = torch.from_numpy(np.stack(wk["targets"])).to(dev)
    line, fwd_by = {}, {}
    for prec in ("fp64", "mixed"):
        p = mw.Plan(L, wk["spins"], precision=prec, graph=True)
        y = torch.empty_like(tg)
        gmap = torch.empty_like(x)

        def step():
            p.forward(x, out=y)
            p.forward_adjoint(2 * (y - tg), out=gmap)
        line[prec] = {"transforms_per_s": rate(step, 2 * len(wk["maps"]))}
        p.forward(x, out=y)
        fwd_by[prec] = y.clone()
        p.close()
    line["mixed"]["forward_vs_fp64"] = rel_errors(fwd_by["mixed"], fwd_by["fp64"])
    ref = oracle.forward(wk["maps"][0], L, 0)
    line["fp64"]["forward_vs_oracle"] = rel_np(fwd_by["fp64"][0].cpu().numpy(), ref)
    line["mixed"]["forward_vs_oracle"] = rel_np(fwd_by["mixed"][0].cpu().numpy(), ref)
    line["oracle_maps"] = "map 0"
    out["c5_L512_B32_grad"] = line
    return out


def rel_np(x, ref):
    import numpy as np
    d = np.abs(np.asarray(x) - np.asarray(ref))
    r = np.abs(np.asarray(ref))
    return {"rel_max": float(d.max() / max(r.max(), 1e-300)),
            "rel_rms": float(np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300))}


def accuracy_sweep(args, mw, wl, dev, acc):
    """The paper's accuracy protocol (Sec. V-D): five signals per spin with Re,
    Im uniform in [-1, 1], spins 0, 2 and 10, inverse then forward; the mean
    over the five signals of the max-abs round-trip error per L, for the FP64
    path and the mixed path.  At L = 2048 the mixed forward is also compared
    with the FP64 forward per band of l (white coefficients put every band at
    the same amplitude, so the per-band figures are not hidden by the global
    normalisation)."""
    import numpy as np
    import torch
    spins = [0] * 5 + [2] * 5 + [10] * 5
    res = []
    for L in (32, 64, 128, 256, 512, 1024, 2048):
        g = wl.rng(7000 + L)
        f = torch.from_numpy(np.stack([wl.uniform_flm(g, L, s) for s in spins])).to(dev)
        row = {"L": L}
        maps = {}
        for prec in ("fp64", "mixed"):
            p = mw.Plan(L, spins, precision=prec)
            m = p.inverse(f)
            b = p.forward(m)
            e = (b - f).abs().amax(dim=1).cpu().numpy()
            row[prec] = {str(s): float(np.mean(e[5 * k:5 * k + 5])) for k, s in enumerate((0, 2, 10))}
            maps[prec] = (p, m)
        if L == 2048:
            p64, m64 = maps["fp64"]
            fm = maps["mixed"][0].forward(m64)
            f64 = p64.forward(m64)
            rep = error_report(fm, f64, L)
            acc["forward_vs_fp64_white"] = rep
            acc["inverse_vs_fp64_white"] = rel_errors(maps["mixed"][1], m64)
        for p, _ in maps.values():
            p.close()
        del maps
        res.append(row)
        torch.cuda.synchronize(dev)
    return {"what": "mean over 5 signals of max|f_lm round trip - f_lm| (Re, Im uniform[-1,1]), by spin",
            "rows": res}


def cpu_baseline(w, quick=False):
    """FP64 oracle round trip of one map of the workload on the host cores."""
    import numpy as np

    import oracle
    L, s = w["L"], w["spins"][0]
    f = np.asarray(w["flm"][0])
    t0 = time.perf_counter()
    m = oracle.inverse(f, L, s)
    oracle.forward(m, L, s)
    t = time.perf_counter() - t0
    return {"value": 2.0 / t, "unit": "transforms/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one map (spin {s}) of the L={L} workload: oracle inverse + forward, {t:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_1110_6298_gb300 import workloads as wl
    w = wl.workload_l2048_b16(n_maps=2, L=args.L)
    for _ in range(args.warmup):
        cpu_baseline(w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(w)
    t = time.perf_counter() - t0
    value = 2.0 * args.steps / t
    cb["value"] = value
    cb["sample"] = f"each step: one map of the L={args.L} workload, oracle inverse + forward"
    return {"metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"MW round trip L={args.L}, one map per step (oracle sample)"},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_tf32", "fp64"])
    ap.add_argument("--L", type=int, default=L_BENCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the FP64-path round trip")
    ap.add_argument("--no-autotune", action="store_true", help="use the fixed default tuning")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads' lines and the paper's accuracy protocol")
    ap.add_argument("--tuning", default=None, metavar="CHUNK,GROUPS,TN_THREADS",
                    help="apply this tuning to the headline plan instead of autotuning it")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the headline round trip and its stage breakdown (profiling runs)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
