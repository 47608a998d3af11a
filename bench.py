#!/usr/bin/env python
"""Benchmark of the overlap hot path on one GB300 (or N independent replicas).

Workload (the 24^3 x 48 lattice the headline metric is quoted on):
  links U = exp(i 0.3 H) seeded (synthetic stand-in for the paper's smeared
  ensembles), 40 deflated eigenpairs of K from ov_eigs, Chebyshev order 256 on
  [|lambda_41|, lambda_max], Gaussian source.  One step = one sign(K) psi
  application through the C ABI (deflation projection, 2N+1 fused stencil
  launches, deflation correction), inputs resident in HBM; the working set
  (links, eigenvectors, recurrence vectors: several GB) is far larger than L2.

Also reported: the stencil's achieved HBM bandwidth (algorithmic bytes over
its CUDA-event-timed launches inside the timed region), the same metric end
to end through host buffers, sign(K) applies/s in every precision, the time
to a 1e-10 solve of D^dagger D in mixed precision and in plain FP64 (both
measured; --quick skips the FP64 solve and the batched ones), the 12 point
sources solved in one call by CG and by GMRESR, the chiral-sector solve of a
point source, the GMRESR solve of D x = b, 3 steps of over-improved stout
smearing, the 16^3 x 32 FP32-operator solve and the gradient.  The field
(plaquette, spectral interval) and the host running the CPU baseline (nproc,
CPU model, nproc and 1 BLAS/OpenMP threads) are described in the line.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sign(K)ψ applies/s & dslash HBM GB/s at 24^3×48, mixed vs FP64 at 1e-10"
DIMS = (24, 24, 24, 48)
ORDER = 256
N_EV = 40
MU = 0.02
SEED_LINKS = 1003
SEED_SRC = 2003
FALLBACK_HBM_GBS = 6800.0

# bytes per site of one stored object, per precision
LINK_B = {"fp64": 4 * 144, "fp32": 4 * 48, "fp16": 4 * 24, "bf16": 4 * 24}
SPIN_B = {"fp64": 192, "fp32": 96, "fp16": 48, "bf16": 48}
VEC_B = {"fp64": 192, "fp32": 96, "fp16": 96, "bf16": 96}
# bytes per site of one D_W / K application when each link is read once and the
# spinor once in and once out (the stored layouts: FP64 18-real links, the others
# reconstruct-12)
MIN_B = {p: LINK_B[p] + 2 * SPIN_B[p] for p in LINK_B}
# the no-reuse convention quoted for the paper's era (1440 B/site in FP32: the 8
# neighbour spinors and links, the output and the diagonal term, no cache reuse),
# scaled by the storage width
NO_REUSE_B = {"fp64": 2880, "fp32": 1440, "fp16": 720, "bf16": 720}


def stencil_metrics(prec, vol, launch_s, peak_gbs):
    """The metric triple of one stencil launch of launch_s seconds: ncu DRAM GB/s
    (committed capture, when it matches the sources), t_min / t at MIN_B, and the
    effective GB/s under the no-reuse convention."""
    traffic = ncu_traffic(prec)
    t_min = MIN_B[prec] * vol / (peak_gbs * 1e9)
    out = {"t_min_over_t": t_min / launch_s, "min_bytes_per_site": MIN_B[prec],
           "effective_GBps_no_reuse": NO_REUSE_B[prec] * vol / launch_s / 1e9,
           "no_reuse_bytes_per_site": NO_REUSE_B[prec]}
    if traffic is not None:
        out["dram_GBps_ncu_traffic"] = traffic * vol / launch_s / 1e9
        out["dram_frac_ncu_traffic"] = out["dram_GBps_ncu_traffic"] / peak_gbs
    return out


def recurrence_bytes(prec, order, vol):
    """Algorithmic HBM bytes of the 2N back-to-back stencil launches of the
    Chebyshev recurrence (the launches bracketed by profiling mode 2)."""
    l, s = LINK_B[prec], SPIN_B[prec]
    k_steps = order * (l + 2 * s)                          # t = K b_{k+1}
    clenshaw = (l + 3 * s) + (order - 1) * (l + 5 * s)     # first step reads psi_perp once
    return vol * (k_steps + clenshaw)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def ncu_traffic(prec):
    """DRAM bytes per site per stencil launch from the committed ncu summary,
    if it was taken on the current stencil source (else None)."""
    csrc = os.path.join(ROOT, "paper_1510_06897_gb300", "csrc")
    path = os.path.join(ROOT, "profiles", "dslash_24x24x24x48.md")
    try:
        h = hashlib.sha256()
        for name in ("dslash_kernel.cuh", "spin.cuh", "common.cuh"):  # everything the stencil is built from
            h.update(open(os.path.join(csrc, name), "rb").read())
        sha = h.hexdigest()[:16]
        text = open(path).read()
    except OSError:
        return None
    if f"source_sha256_16: {sha}" not in text:
        return None
    for line in text.splitlines():
        line = line.strip()
        if line.startswith(f"traffic_bytes_per_site_{prec}:"):
            return float(line.split(":")[1])
    return None


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_sample(a, b, order, sample_terms=2, sample_vecs=4):
    """The FP64 oracle timed on the host: sample_terms Chebyshev terms and a
    projection onto sample_vecs vectors, extrapolated to one full sign(K)
    apply (order terms, one final K, N_EV-vector deflation).  The projection's
    cost does not depend on the vectors, so seeded Gaussian stand-ins of the
    eigenvectors' size are used."""
    from oracle import chebyshev, overlap, wilson
    from paper_1510_06897_gb300 import inputs

    links = inputs.gauge_links(DIMS, seed=SEED_LINKS)
    psi = inputs.gaussian_source(DIMS, seed=SEED_SRC)[0]
    vecs = inputs.gaussian_source(DIMS, seed=SEED_SRC + 50, nrhs=sample_vecs)
    c = chebyshev.coefficients(sample_terms, a, b)

    def kop(w):
        return wilson.kernel_k(links, w)

    t0 = time.perf_counter()
    chebyshev.apply_fn(kop, c, a, b, psi)
    t_terms = time.perf_counter() - t0
    t0 = time.perf_counter()
    kop(psi)
    t_k = time.perf_counter() - t0
    t0 = time.perf_counter()
    coeffs = overlap.project(vecs, psi)
    perp = psi.copy()
    for i in range(sample_vecs):
        perp = perp - coeffs[i] * vecs[i]
    t_defl = time.perf_counter() - t0
    per_apply = t_terms / sample_terms * order + t_k + 2 * t_defl * N_EV / sample_vecs
    return {"per_apply_s": per_apply, "sample_seconds": t_terms + t_k + t_defl,
            "sample": (f"FP64 NumPy oracle on 24^3x48: {sample_terms} Chebyshev terms ({2 * sample_terms} K), "
                       f"1 K, projection onto {sample_vecs} vectors; extrapolated to {order} terms + "
                       f"{N_EV}-vector deflation")}


def host_description():
    """nproc and the CPU model (lscpu) of the machine running the bench."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def cpu_baseline(a, b, order):
    """The oracle sample run in fresh interpreters (no GPU use) with the BLAS /
    OpenMP thread count set to nproc and to 1; the headline value is the nproc
    run, labelled extrapolated (a full sign(K) apply takes hours on the host)."""
    host = host_description()
    runs = {}
    for threads in sorted({host["nproc"] or 1, 1}, reverse=True):
        env = dict(os.environ)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[var] = str(threads)
        env["CUDA_VISIBLE_DEVICES"] = ""
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", f"{a!r},{b!r},{order}"],
                             capture_output=True, text=True, env=env, timeout=900)
        if res.returncode != 0:
            runs[threads] = {"error": res.stderr.strip().splitlines()[-1:] or ["cpu sample failed"]}
            continue
        runs[threads] = json.loads(res.stdout.strip().splitlines()[-1])
    top = max(runs)
    main_run = runs[top]
    if "per_apply_s" not in main_run:
        return {"value": None, "unit": "applies/s", "cores": top, "kind": "oracle (extrapolated)",
                "sample": str(main_run), **host}
    out = {"value": 1.0 / main_run["per_apply_s"], "unit": "applies/s", "cores": top,
           "kind": "oracle (extrapolated)", "sample": main_run["sample"],
           "sample_seconds": main_run["sample_seconds"], "threads": "BLAS/OpenMP threads = nproc", **host}
    if 1 in runs and top != 1 and "per_apply_s" in runs[1]:
        out["single_thread"] = {"value": 1.0 / runs[1]["per_apply_s"], "unit": "applies/s", "cores": 1,
                                "sample_seconds": runs[1]["sample_seconds"]}
    return out


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, each step a bounded sample of the
    workload (one application of K; a sign(K) apply needs 2N+1 of them plus the
    vector algebra and the deflation, which this sample leaves out)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import wilson
    from paper_1510_06897_gb300 import inputs

    links = inputs.gauge_links(DIMS, seed=SEED_LINKS)
    psi = inputs.gaussian_source(DIMS, seed=SEED_SRC)[0]

    def step():
        wilson.kernel_k(links, psi)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    per_k = (time.perf_counter() - t0) / args.steps
    per_apply = per_k * (2 * ORDER + 1)
    value = 1.0 / per_apply
    sample = (f"one K application of the FP64 NumPy oracle at 24^3x48 per step ({per_k:.2f} s), "
              f"x {2 * ORDER + 1} per sign(K) apply; vector algebra and deflation not included")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_k * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"24^3x48 sign(K) psi, Chebyshev order {ORDER} (oracle sample: one K per step)",
                       "lattice": "24x24x24x48"},
            "cpu_baseline": {"value": value, "unit": "applies/s", "kind": "oracle (extrapolated)", "cores": 1,
                             "sample": sample, **host_description()},
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_over_ranks(elapsed_ms, steps, world, dist=None, device=None):
    """Max of the timed region over ranks (replicas) and the whole-job rate."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, world * steps / (elapsed_ms * 1e-3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp16", choices=["fp16", "bf16", "fp32", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="headline only")
    ap.add_argument("--quick", action="store_true",
                    help="skip the minutes-long solves (plain FP64 solve, the 12 point sources by CG and GMRESR)")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--eigs-cache", default=None,
                    help="checkpoint file of the set-up eigenpairs: loaded when it matches this workload, "
                         "else computed and written there")
    args = ap.parse_args()
    if args.cpu_sample:
        a, b, order = args.cpu_sample.split(",")
        print(json.dumps(cpu_sample(float(a), float(b), int(order))), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_1510_06897_gb300 import inputs
    from paper_1510_06897_gb300.binding import (OV_ERR_NOT_CONVERGED, Ctx, OverlapError, ov_eigs, ov_get_stats,
                                                ov_reset_stats, ov_set_profiling, ov_sign_apply, ov_solve)

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vol = inputs.volume(DIMS)
    t_setup = time.perf_counter()
    links = inputs.gauge_links(DIMS, seed=SEED_LINKS)
    links_d = torch.from_numpy(links).cuda()
    fshape = (DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)

    # S0 setup (not timed): eigenpairs of K from an FP32 context, or from a
    # checkpoint of exactly this workload
    t_eigs = time.perf_counter()
    eigs_source = "ov_eigs"
    cached = None
    if args.eigs_cache and os.path.exists(args.eigs_cache):
        from paper_1510_06897_gb300 import checkpoint
        try:
            cached = checkpoint.load_eigenpairs(args.eigs_cache, DIMS, n_ev=N_EV + 1, links_seed=SEED_LINKS,
                                                tol=2e-5)
        except checkpoint.CheckpointError as e:
            print(f"eigenpair cache not used: {e}", file=sys.stderr)
    if cached is not None:
        evals, ev_h, meta = cached
        evecs = torch.from_numpy(ev_h).cuda()
        lmax = meta["lambda_max"]
        eigs_source = "checkpoint"
    else:
        evecs = torch.zeros((N_EV + 1,) + fshape, dtype=torch.complex128, device="cuda")
        with Ctx(DIMS, links_d, "fp32") as c32:
            try:
                evals, lmax = ov_eigs(c32.handle, N_EV + 1, 2e-5, 300, evecs)
            except OverlapError as e:  # keep the measurement: more sweeps, then the best pairs found
                if e.status != OV_ERR_NOT_CONVERGED:
                    raise
                evals, lmax = ov_eigs(c32.handle, N_EV + 1, 2e-5, 600, evecs, allow_not_converged=True)
                eigs_source = "ov_eigs (best pairs after 300 + 600 sweeps; 2e-5 not reached)"
        if args.eigs_cache:
            from paper_1510_06897_gb300 import checkpoint
            checkpoint.save_eigenpairs(args.eigs_cache, DIMS, evals, evecs, lambda_max=lmax, links_seed=SEED_LINKS,
                                       tol=2e-5)
    t_eigs = time.perf_counter() - t_eigs
    a, b = float(abs(evals[N_EV])), float(lmax)
    evals40, evecs40 = evals[:N_EV].copy(), evecs[:N_EV].contiguous()
    del evecs

    psi = torch.from_numpy(inputs.gaussian_source(DIMS, seed=SEED_SRC)).cuda()
    out = torch.empty_like(psi)
    ctx = Ctx(DIMS, links_d, args.prec)
    ctx.sign_config(ORDER, a, b, evals40, evecs40)
    setup_s = time.perf_counter() - t_setup

    for _ in range(args.warmup):
        ov_sign_apply(ctx.handle, psi, out, 1)
    torch.cuda.synchronize()
    ov_reset_stats(ctx.handle)
    ov_set_profiling(ctx.handle, 2)  # one event pair around each recurrence (2N stencil launches)
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ov_sign_apply(ctx.handle, psi, out, 1)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ov_set_profiling(ctx.handle, False)
    elapsed_ms = e0.elapsed_time(e1)
    st = ov_get_stats(ctx.handle)
    elapsed_ms, value = aggregate_over_ranks(elapsed_ms, args.steps, world, dist, device="cuda")
    ms_per_step = elapsed_ms / args.steps

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    bytes_launch = recurrence_bytes(args.prec, ORDER, vol) / (2 * ORDER)
    dslash_ms_avg = st["dslash_ms"] / max(1, st["dslash_timed"])
    achieved = bytes_launch / (dslash_ms_avg * 1e-3) / 1e9
    traffic_site = ncu_traffic(args.prec)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": (traffic_site * vol if traffic_site is not None else None),
                "kernel": f"k_dslash ({args.prec} storage), average over the 2N back-to-back launches of the "
                          f"Chebyshev recurrence (one CUDA event pair around them per apply, gaps included)",
                "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_us": dslash_ms_avg * 1e3, "peak_source": f"hbm_gbs of {peak_kind}",
                "variant": {k: st[k] for k in ("stencil_tpb", "stencil_minb", "stencil_lrec", "stencil_async",
                                               "stencil_brick", "stencil_slab")},
                "stencil_share_of_step": st["dslash_ms"] / elapsed_ms if world == 1 else None}
    roofline.update(stencil_metrics(args.prec, vol, dslash_ms_avg * 1e-3, hbm))

    # end to end through the C ABI with host (pinned) buffers
    psi_h = psi.cpu().pin_memory()
    out_h = torch.empty_like(psi_h).pin_memory()
    n_e2e = max(3, min(args.steps, 10))
    ov_sign_apply(ctx.handle, psi_h, out_h, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ov_sign_apply(ctx.handle, psi_h, out_h, 1)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    iface = vol * 12 * 16
    e2e = {"value": world / e2e_s, "unit": "applies/s", "h2d_bytes_per_step": iface, "d2h_bytes_per_step": iface}

    line = {"metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec != "fp64" else "f64",
            "data": "synthetic (seeded exp(i 0.3 H) links, Gaussian source)",
            "config": {"workload": f"24^3x48 sign(K) psi, Chebyshev order {ORDER}, {N_EV} deflated eigenpairs, "
                                   f"{args.prec} storage",
                       "lattice": "24x24x24x48", "order": ORDER, "n_ev": N_EV, "storage": args.prec,
                       "interval": [a, b], "l2": "inputs larger than L2 (links + eigenvectors + vectors, GBs)",
                       "parallelism": "replicas" if world > 1 else "1 GPU", "setup_s": setup_s,
                       "eigs_s": t_eigs, "eigs_source": eigs_source,
                       "field": field_description(links_d, evals, a, b)},
            "roofline": roofline, "e2e": e2e, "gpu_launches": st["kernel_launches"], "clocks": clk}

    if rank == 0 and not args.no_extras:
        try:
            line["extras"] = extras(args, ctx, links_d, a, b, evals40, evecs40, psi, vol)
        except Exception as e:  # a failing extra must not cost the headline line
            line["extras"] = {"error": f"{type(e).__name__}: {e}"}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(a, b, ORDER)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def field_description(links_d, evals, a, b):
    """The synthetic field's average plaquette and the spectral interval of
    the sign function: |lambda_min(K)|, |lambda_{n_ev+1}| (the interval's
    lower end a) and the upper end b (ov_eigs' bound on lambda_max)."""
    return {"plaquette": _plaquette(links_d), "abs_lambda_min": float(abs(evals[0])),
            f"abs_lambda_{N_EV + 1}": float(a), "lambda_max_bound": float(b),
            "links": "U = exp(i 0.3 H), H seeded Gaussian traceless Hermitian (stand-in for the paper's "
                     "stout-smeared ensembles)"}


def extras(args, ctx, links_d, a, b, evals, evecs, psi, vol):
    """Per-precision sign(K) rates and stencil bandwidth; solves to 1e-10."""
    import torch
    from paper_1510_06897_gb300.binding import (Ctx, ov_get_stats, ov_reset_stats, ov_set_profiling,
                                                ov_sign_apply, ov_solve)
    peaks, _ = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    res = {"precisions": {}}
    out = torch.empty_like(psi)
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        reps = 2 if prec == "fp64" else 8
        with Ctx(DIMS, links_d, prec) as c:
            c.sign_config(ORDER, a, b, evals, evecs)
            ov_sign_apply(c.handle, psi, out, 1)
            torch.cuda.synchronize()
            ov_reset_stats(c.handle)
            ov_set_profiling(c.handle, 2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ov_sign_apply(c.handle, psi, out, 1)
            e1.record()
            torch.cuda.synchronize()
            ov_set_profiling(c.handle, False)
            st = ov_get_stats(c.handle)
        ms = e0.elapsed_time(e1) / reps
        avg = st["dslash_ms"] / max(1, st["dslash_timed"])
        gbs = recurrence_bytes(prec, ORDER, vol) / (2 * ORDER) / (avg * 1e-3) / 1e9
        res["precisions"][prec] = {"applies_per_s": 1e3 / ms, "ms_per_apply": ms, "stencil_avg_us": avg * 1e3,
                                   "stencil_GBps": gbs, "stencil_frac_of_hbm": gbs / hbm}
        res["precisions"][prec].update(stencil_metrics(prec, vol, avg * 1e-3, hbm))
    # batched: the 12 spin-colour point sources in one call (config of the
    # batched workload), per-RHS rate against the single-RHS rate above
    from paper_1510_06897_gb300 import inputs as _inp
    src = torch.from_numpy(_inp.point_sources(DIMS)).cuda()
    outb = torch.empty_like(src)
    batched = {}
    for prec in ("fp16", "fp32"):
        with Ctx(DIMS, links_d, prec) as c:
            c.sign_config(ORDER, a, b, evals, evecs)
            ov_sign_apply(c.handle, src, outb, 12)          # tunes the 12-RHS stencil shape
            torch.cuda.synchronize()
            ov_reset_stats(c.handle)
            ov_set_profiling(c.handle, 2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ov_sign_apply(c.handle, src, outb, 12)
            e1.record()
            torch.cuda.synchronize()
            ov_set_profiling(c.handle, False)
            st = ov_get_stats(c.handle)
        ms = e0.elapsed_time(e1)
        single = res["precisions"][prec]["ms_per_apply"]
        batched[prec] = {"rhs_applies_per_s": 12e3 / ms, "ms_per_12rhs_apply": ms,
                         "speedup_vs_12_single": 12 * single / ms,
                         "stencil_share": st["dslash_ms"] / ms}
    res["batched_12_point_sources"] = batched
    # time to solution, D^dagger D x = D^dagger b to 1e-10 (true residual, FP64 operator)
    solves = {}
    precs = [args.prec] + ([] if args.quick or args.prec == "fp64" else ["fp64"])
    for prec in precs:
        with Ctx(DIMS, links_d, prec) as c:
            c.sign_config(ORDER, a, b, evals, evecs)
            x = torch.empty_like(psi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, r = ov_solve(c.handle, MU, 1e-10, 20000, psi, x, 1, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = ov_get_stats(c.handle)
        if prec == args.prec:
            x_cg = x
        solves[prec] = {"seconds": dt, "iterations": it, "outer": st["outer_iterations"], "true_rel_resid": r,
                        "mu": MU}
    if "fp64" in solves:
        solves["speedup_mixed_vs_fp64"] = solves["fp64"]["seconds"] / solves[args.prec]["seconds"]
    if not args.quick:
        with Ctx(DIMS, links_d, args.prec) as c:
            c.sign_config(ORDER, a, b, evals, evecs)
            x = torch.empty_like(src)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, r = ov_solve(c.handle, MU, 1e-10, 200000, src, x, 12, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = ov_get_stats(c.handle)
        batched_cg = {"precision": args.prec, "method": "CG on D^dagger D, 12 right-hand sides per launch",
                      "seconds": dt, "iterations": it, "outer": st["outer_iterations"], "true_rel_resid": r}
        if "fp64" in solves:
            fp64_12 = 12 * solves["fp64"]["seconds"]
            batched_cg["fp64_single_rhs_path_x12_seconds"] = fp64_12
            batched_cg["fp64_single_rhs_path_x12_basis"] = (
                "12 x the measured plain-FP64 single-RHS CG solve of the Gaussian source above "
                "(the FP64 path solves one right-hand side per call)")
            batched_cg["speedup_vs_fp64_single_rhs_path_x12"] = fp64_12 / dt
        solves["batched_12_point_sources"] = batched_cg
        gm = _guarded(gmresr_batched_timing, links_d, a, b, evals, evecs, src, args.prec)
        if "fp64" in solves and "seconds" in gm:
            gm["speedup_vs_fp64_single_rhs_path_x12"] = 12 * solves["fp64"]["seconds"] / gm["seconds"]
        solves["batched_12_point_sources_gmresr"] = gm
    # chiral point source (spin 0, colour 0 at the origin: chirality +1): D^-1 b
    # from the chiral-sector solve (one sign apply per iteration) + one D^dagger,
    # against the D^dagger D solve of the same source
    from paper_1510_06897_gb300.binding import ov_overlap, ov_solve_chiral
    src0 = src[0:1].contiguous()
    chiral = {}
    with Ctx(DIMS, links_d, args.prec) as c:
        c.sign_config(ORDER, a, b, evals, evecs)
        x = torch.empty_like(src0)
        y = torch.empty_like(src0)
        for name in ("chiral_sector", "normal_equations"):
            ov_reset_stats(c.handle)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "chiral_sector":
                it, r = ov_solve_chiral(c.handle, MU, 1, 1e-10, 20000, src0, y, 1, allow_not_converged=True)
                ov_overlap(c.handle, MU, 1, y, x, 1)            # D^-1 b = D^dagger A^-1 P b
            else:
                it, r = ov_solve(c.handle, MU, 1e-10, 20000, src0, x, 1, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = ov_get_stats(c.handle)
            chiral[name] = {"seconds": dt, "iterations": it, "outer": st["outer_iterations"],
                            "sign_applies": st["sign_applies"], "true_rel_resid": r}
    chiral["speedup"] = chiral["normal_equations"]["seconds"] / chiral["chiral_sector"]["seconds"]
    solves["chiral_point_source"] = chiral
    solves["gmresr"] = _guarded(gmresr_timing, links_d, a, b, evals, evecs, psi, args.prec,
                                solves[args.prec]["seconds"], x_cg=x_cg)
    res["solve_1e-10"] = solves
    res["launch_gaps"] = _guarded(launch_gap_timing, ctx, psi, args.prec)
    res["stout_smearing"] = _guarded(smear_timing, links_d)
    res["paper_lattices_wilson"] = _guarded(paper_wilson_timing)
    res["solve_16x16x16x32_fp32"] = _guarded(solve_16_timing)
    res["gradient"] = _guarded(gradient_timing)
    return res


def _guarded(fn, *args, **kwargs):
    """fn's result, or the error it raised (independent extras do not take
    the others down with them)."""
    try:
        return fn(*args, **kwargs)
    except Exception as e:
        return {"error": f"{type(e).__name__}: {e}"}


def gmresr_timing(links_d, a, b, evals, evecs, psi, prec, cg_seconds=None, x_cg=None):
    """D[mu] x = psi to 1e-10 (||psi - D x|| / ||psi||, FP64 operator) by
    GMRESR: GCR on D (FP32 copy of the operator for 16-bit storage, the
    default), inner SUMR in the storage precision with a relaxed (automatic,
    sign error <= 1e-2) sign, FP64 defect correction; the FP32 copy is made
    before the timed solve and its set-up reported apart.  For 16-bit storage
    also the same solve with GCR in the storage precision.  x_cg: the CG
    (normal equations) solution of the same system, whose ||psi - D x|| / ||psi||
    and distance to the GMRESR solution are reported (the CG stops on the
    normal-equation residual instead)."""
    import torch
    from paper_1510_06897_gb300.binding import (Ctx, ov_enable_fp32_operator, ov_get_stats, ov_overlap,
                                                ov_reset_stats, ov_set_gmresr_fp32_level, ov_solve_gmresr)
    out = {}
    if x_cg is not None:
        with Ctx(DIMS, links_d, "fp64") as c64:
            c64.sign_config(ORDER, a, b, evals, evecs)
            dx = torch.empty_like(psi)
            ov_overlap(c64.handle, MU, 0, x_cg, dx, 1)
            out["cg_true_rel_resid_D"] = (torch.linalg.vector_norm(psi - dx) / torch.linalg.vector_norm(psi)).item()
    levels = [("default", True)] + ([("storage_precision_gcr", False)] if prec in ("fp16", "bf16") else [])
    for name, fp32_level in levels:
        with Ctx(DIMS, links_d, prec) as c:
            t0 = time.perf_counter()
            if fp32_level:
                ov_enable_fp32_operator(c.handle, links_d)
            else:
                ov_set_gmresr_fp32_level(c.handle, 0)
            c.sign_config(ORDER, a, b, evals, evecs)
            setup = time.perf_counter() - t0
            x = torch.empty_like(psi)
            ov_reset_stats(c.handle)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, r = ov_solve_gmresr(c.handle, MU, 1e-10, 100000, psi, x, 1, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = ov_get_stats(c.handle)
        gcr = ("fp32" if (fp32_level and prec in ("fp16", "bf16")) else prec)
        out[name] = {
            "precision": f"{prec} SUMR, {gcr} GCR", "seconds": dt, "setup_s": setup, "sumr_iterations": it,
            "relaxed_order": st["gmresr_order"], "gcr_steps": st["gcr_iterations"],
            "fp64_passes": st["outer_iterations"], "sign_applies": st["sign_applies"],
            "dslash_launches": st["dslash_launches"], "true_rel_resid_D": r, "mu": MU,
            "speedup_vs_cg_normal_equations": (cg_seconds / dt) if cg_seconds else None,
            "rel_diff_to_cg_solution": ((torch.linalg.vector_norm(x - x_cg) / torch.linalg.vector_norm(x_cg)).item()
                                        if x_cg is not None else None)}
    return out


def gmresr_batched_timing(links_d, a, b, evals, evecs, src, prec):
    """D[mu] x = src for all right-hand sides of src in one ov_solve_gmresr
    call (batched stencil launches), to 1e-10 in ||b - D x|| / ||b||."""
    import torch
    from paper_1510_06897_gb300.binding import Ctx, ov_get_stats, ov_solve_gmresr
    with Ctx(DIMS, links_d, prec) as c:
        c.sign_config(ORDER, a, b, evals, evecs)
        x = torch.empty_like(src)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, r = ov_solve_gmresr(c.handle, MU, 1e-10, 200000, src, x, src.shape[0], allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = ov_get_stats(c.handle)
    return {"precision": prec, "nrhs": int(src.shape[0]), "seconds": dt, "sumr_iterations": it,
            "relaxed_order": st["gmresr_order"], "gcr_steps": st["gcr_iterations"],
            "fp64_passes": st["outer_iterations"], "true_rel_resid_D": r}


# The paper's Wilson-matrix times on its own lattices (Table 4, one GTX Titan,
# precision not stated), quoted beside ours for context only.
PAPER_WILSON_MS = {"8x8x8x32": 0.248, "20x20x20x64": 6.759}


def paper_wilson_timing():
    """D_W (ov_wilson's stencil launch, CUDA events around each launch) on the
    paper's two lattices, FP64 / FP32 / FP16 storage, seeded synthetic links."""
    import torch
    from paper_1510_06897_gb300 import inputs
    from paper_1510_06897_gb300.binding import Ctx, ov_get_stats, ov_reset_stats, ov_set_profiling, ov_wilson
    out = {}
    for dims in ((8, 8, 8, 32), (20, 20, 20, 64)):
        key = "x".join(str(d) for d in dims)
        links = torch.from_numpy(inputs.gauge_links(dims, seed=SEED_LINKS)).cuda()
        psi = torch.from_numpy(inputs.gaussian_source(dims, seed=SEED_SRC)).cuda()
        res = {"paper_gtx_titan_ms": PAPER_WILSON_MS[key]}
        for prec in ("fp64", "fp32", "fp16"):
            with Ctx(dims, links, prec) as c:
                y = torch.empty_like(psi)
                for _ in range(3):
                    ov_wilson(c.handle, psi, y, 1)
                torch.cuda.synchronize()
                ov_reset_stats(c.handle)
                ov_set_profiling(c.handle, 1)
                for _ in range(20):
                    ov_wilson(c.handle, psi, y, 1)
                torch.cuda.synchronize()
                ov_set_profiling(c.handle, 0)
                st = ov_get_stats(c.handle)
            res[f"{prec}_stencil_ms"] = st["dslash_ms"] / max(1, st["dslash_timed"])
        out[key] = res
        del links, psi
    return out


def launch_gap_timing(ctx, psi, prec, reps=4):
    """Stencil time per launch of the recurrence measured two ways on the
    headline context: one event pair around every launch (kernel time; the
    extra event records between launches slow the apply itself) and one pair
    around the 2N back-to-back launches (kernel time plus the gaps between
    launches).  Their difference bounds what overlapping consecutive
    launches could save."""
    import torch
    from paper_1510_06897_gb300.binding import ov_get_stats, ov_reset_stats, ov_set_profiling, ov_sign_apply
    out = torch.empty_like(psi)
    per = {}
    for mode in (1, 2):
        ov_reset_stats(ctx.handle)
        ov_set_profiling(ctx.handle, mode)
        for _ in range(reps):
            ov_sign_apply(ctx.handle, psi, out, 1)
        torch.cuda.synchronize()
        ov_set_profiling(ctx.handle, 0)
        st = ov_get_stats(ctx.handle)
        per[mode] = st["dslash_ms"] / max(1, st["dslash_timed"]) * 1e3
    return {"precision": prec, "us_per_launch_events_around_each": per[1],
            "us_per_launch_bracketed_recurrence": per[2], "gap_us_per_launch": per[2] - per[1]}


def _plaquette(u):
    """Average (1/3) Re tr of the plaquettes of device links (4, Lt, Lz, Ly, Lx, 3, 3)."""
    import torch
    axis = (3, 2, 1, 0)
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = (u[mu] @ torch.roll(u[nu], -1, axis[mu])
                 @ torch.roll(u[mu], -1, axis[nu]).conj().transpose(-1, -2) @ u[nu].conj().transpose(-1, -2))
            tot += (p.diagonal(dim1=-2, dim2=-1).sum(-1).real.mean() / 3).item()
    return tot / 6


def smear_timing(links_d):
    """3 steps of over-improved stout smearing (rho = 0.1, eps = -0.25) of the
    24^3 x 48 field: time (CUDA events) and the average plaquette before and
    after each step."""
    import torch
    from paper_1510_06897_gb300.binding import ov_stout_smear
    out = torch.empty_like(links_d)
    ov_stout_smear(DIMS, links_d, out, 0.1, -0.25, 3)  # warm-up
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    ov_stout_smear(DIMS, links_d, out, 0.1, -0.25, 3)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    plaq = [_plaquette(links_d)]
    cur = links_d.clone()
    for _ in range(3):
        ov_stout_smear(DIMS, cur, cur, 0.1, -0.25, 1)
        plaq.append(_plaquette(cur))
    del cur
    vol = 1
    for d in DIMS:
        vol *= d
    return {"ms_3_steps": ms, "links_per_s": 3 * 4 * vol / (ms * 1e-3), "plaquette_per_step": plaq,
            "rho": 0.1, "eps": -0.25, "precision": "fp64"}


def solve_16_timing():
    """The 16^3 x 32 FP32-operator workload: 20 eigenpairs from ov_eigs,
    Chebyshev order 200, CG on D^dagger D at mu = 0.05 to a 1e-10 true residual
    (time to solution, iterations, stencil launches; eigensolver timed apart)."""
    import torch
    from paper_1510_06897_gb300 import inputs
    from paper_1510_06897_gb300.binding import Ctx, ov_eigs, ov_get_stats, ov_reset_stats, ov_solve
    dims, n_ev, order, mu = (16, 16, 16, 32), 20, 200, 0.05
    links = torch.from_numpy(inputs.gauge_links(dims, seed=1002)).cuda()
    b_src = torch.from_numpy(inputs.gaussian_source(dims, seed=2002)).cuda()
    evecs = torch.zeros((n_ev + 1, dims[3], dims[2], dims[1], dims[0], 4, 3), dtype=torch.complex128, device="cuda")
    with Ctx(dims, links, "fp32") as c:
        t0 = time.perf_counter()
        evals, lmax = ov_eigs(c.handle, n_ev + 1, 2e-5, 3000, evecs)  # dense low band, |lambda| 0.531..0.536
        torch.cuda.synchronize()
        t_eigs = time.perf_counter() - t0
        a, b = float(abs(evals[n_ev])), float(lmax)
        c.sign_config(order, a, b, evals[:n_ev], evecs[:n_ev].contiguous())
        x = torch.empty_like(b_src)
        ov_reset_stats(c.handle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, r = ov_solve(c.handle, mu, 1e-10, 20000, b_src, x, 1, allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = ov_get_stats(c.handle)
    return {"seconds": dt, "iterations": it, "outer": st["outer_iterations"], "true_rel_resid": r,
            "stencil_launches": st["dslash_launches"], "mu": mu, "order": order, "n_ev": n_ev,
            "interval": [a, b], "eigs_seconds": t_eigs}


def gradient_timing():
    """Adjoint of chi^dagger P(K) chi at 16^3 x 32, order 128, complex64 chi, FP32
    context: time of ov_sign_poly_grad against one forward P(K) chi apply, with
    every recurrence term kept on the device (the default) and with
    checkpoints every 16 terms and recomputation (allowance 0)."""
    import torch
    from paper_1510_06897_gb300 import inputs
    from paper_1510_06897_gb300.binding import (Ctx, ov_get_stats, ov_set_grad_memory, ov_sign_apply,
                                                ov_sign_poly_grad)
    dims = (16, 16, 16, 32)
    links = torch.from_numpy(inputs.gauge_links(dims, seed=1005)).cuda()
    chi = torch.from_numpy(inputs.gaussian_source(dims, seed=2005).astype(np.complex64)).cuda()
    grad = torch.empty((4, 32, 16, 16, 16, 3, 3), dtype=torch.complex128, device="cuda")
    a, b, order = 0.45, 6.5, 128
    with Ctx(dims, links, "fp32") as c:
        c.sign_config(order, a, b)
        out = torch.empty_like(chi)
        ov_sign_apply(c.handle, chi, out, 1)
        ov_sign_poly_grad(c.handle, order, a, b, chi, grad)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            ov_sign_apply(c.handle, chi, out, 1)
        torch.cuda.synchronize()
        t_fwd = (time.perf_counter() - t0) / 3
        t_grad = {}
        for name, allowance in (("kept", -1), ("recompute", 0)):
            ov_set_grad_memory(c.handle, allowance)
            ov_sign_poly_grad(c.handle, order, a, b, chi, grad)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                ov_sign_poly_grad(c.handle, order, a, b, chi, grad)
            torch.cuda.synchronize()
            t_grad[name] = ((time.perf_counter() - t0) / 3, ov_get_stats(c.handle)["grad_kept_terms"])
        ov_set_grad_memory(c.handle, -1)
    return {"lattice": "16x16x16x32", "order": order, "forward_ms": t_fwd * 1e3,
            "gradient_ms": t_grad["kept"][0] * 1e3, "ratio": t_grad["kept"][0] / t_fwd,
            "kept_terms": t_grad["kept"][1],
            "recompute": {"gradient_ms": t_grad["recompute"][0] * 1e3, "ratio": t_grad["recompute"][0] / t_fwd,
                          "kept_terms": t_grad["recompute"][1]}}


if __name__ == "__main__":
    main()
