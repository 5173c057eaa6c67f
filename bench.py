#!/usr/bin/env python
"""Benchmark: encrypted quadratic-gradient NAG logistic-regression training.

One step = one full-batch QG-NAG iteration (gradient over every encrypted data
block, quadratic gradient, NAG update, refresh of W and V) on synthetic data
shaped like the paper's Financial workload: 422,108 samples x 200 features,
N = 2^16, 9 ciphertext primes (one 60-bit, eight 40-bit) and a 60-bit special
prime, scale 2^40, 128 x 256 packing (3,298 blocks).  Data blocks are resident
in HBM (29 GiB, far larger than L2) before timing starts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank trains an independent
replica of the job on its GPU (the method shards into independent jobs; no
collective on the data path); value = max-over-ranks time / (N * K).
"""
import argparse
import ctypes
import hashlib
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "enc. QG-NAG sec/iter at 422,108x200 (N=2^16); keyswitch/s; batched vs plain GPU"
N_SAMPLES, N_FEAT, LOGN, NQ, LOG_SCALE = 422108, 200, 16, 9, 40.0
ITER_LEVEL = 6  # fresh ciphertexts sit at the depth of one iteration
PAPER_CONTEXT = {"paper_full_batch_update_s": 60.0, "paper_full_batch_iter_s": 90.0,
                 "paper_hardware": "8 vCPUs, HEAAN (non-RNS), Q=2^275, Delta=2^30"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=0, help="data blocks per launch (0 = library default)")
    ap.add_argument("--rows", type=int, default=N_SAMPLES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-twin", action="store_true")
    ap.add_argument("--no-mini", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-first-order", action="store_true")
    ap.add_argument("--no-bbar", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the compact primitive sweep and the tensor-core floor")
    ap.add_argument("--no-images", action="store_true", help="skip the MNIST-shaped workload")
    ap.add_argument("--no-train", action="store_true", help="skip the whole-training call (he_lr_train)")
    ap.add_argument("--no-boot", action="store_true", help="skip the workload refreshed by bootstrapping")
    ap.add_argument("--no-autotune", action="store_true", help="default key-switch waves (profiling runs)")
    ap.add_argument("--rot-radix", type=int, default=0,
                    help="log2 of the hoisted rotation group (0 = library default)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--sweep-point", default="", help="log_n,limbs,batch: run only this NTT sweep point")
    ap.add_argument("--ks-point", default="",
                    help="level,items,kind (kind relin, rot7, or rot7tc with the inner product on the tensor "
                         "cores): one batched key switch or hoisted rotation sum at N=2^16, the full chain, timed "
                         "(profiling entry)")
    ap.add_argument("--sweep", action="store_true",
                    help="HE primitive sweep: batched NTT and key switching vs N, limbs and batch (JSON line per point)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(dev):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(dev), "--query-gpu=" + CLOCK_Q, "--format=csv,noheader,nounits",
                              "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def clocks_stop(handle):
    p, path = handle
    if p is not None:
        p.send_signal(signal.SIGTERM)
        try:
            p.wait(5)
        except subprocess.TimeoutExpired:
            p.kill()
    rows = []
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(path)
    except OSError:
        pass
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
    sm = sorted(float(r[1]) for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons, "samples": len(rows),
            "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ------------------------------------------------------------------ roofline inputs
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def kernel_sources_hash():
    """sha256 (12 hex digits) of the transform and key-switch sources with
    comments and whitespace removed: it changes with the code, not the prose."""
    import re
    src = "".join(open(os.path.join(ROOT, "paper_2406_13221_gb300", "csrc", f)).read()
                  for f in ("ntt_core.cuh", "ks.cu", "ntt.cu"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return hashlib.sha256("".join(src.split()).encode()).hexdigest()[:12]


def recorded_traffic(kernel):
    """DRAM traffic over algorithmic bytes of one ncu-captured launch of `kernel`
    (profiles/traffic.txt), valid while the kernel's sources are unchanged (else
    None); bench.py scales it to its own average launch."""
    h = kernel_sources_hash()
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            p = line.split()
            if len(p) >= 3 and not line.startswith("#") and p[0] == kernel and p[1] == h:
                return float(p[2])  # measured / algorithmic DRAM bytes of the captured launch
    except OSError:
        pass
    return None


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world):
    import torch
    from paper_2406_13221_gb300 import binding, build, synth

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.cuda.current_device()
    t0 = time.time()
    X, y = synth.financial(seed=1, n=args.rows)
    ctx = binding.Context(LOGN, NQ)
    if args.rot_radix:
        ctx.set_rotation_radix(args.rot_radix)
    # key-switch wave per level from the library's autotuner (the relinearisation
    # key it times with comes from the same seed the job uses for its keys)
    ta = time.time()
    ctx.keygen(2)
    tuned_levels = 0 if args.no_autotune else ctx.autotune(None, 256)
    autotune = {"ks_wave_by_level": [ctx.ks_wave(lv) for lv in range(NQ)],
                "ks_tile_by_level": [ctx.ks_tile(lv) for lv in range(NQ)],
                "hoist_form_by_level": [ctx.hoist_form(lv) for lv in range(NQ)], "levels_measured": tuned_levels,
                "s": round(time.time() - ta, 2)}
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, LOG_SCALE, enc_seed=3, key_seed=2,
                      batch_blocks=args.chunk)
    info = job.stats()
    chunk_used = info_chunk(job, args)
    setup_s = time.time() - t0
    sched = (2.0, 1.0, 81.0, 2.5)
    t = 0
    for _ in range(args.warmup):
        job.step(t, sched)
        t += 1
    # ---------------- timed region (device-resident inputs)
    ctx.prof_enable(True)
    l0 = binding.launch_count()
    clk = clocks_start(dev)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_range:
        torch.cuda.cudart().cudaProfilerStart()
    e0.record()
    for _ in range(args.steps):
        job.step(t, sched)
        t += 1
    e1.record()
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.cudart().cudaProfilerStop()
    barrier(world)
    clocks = clocks_stop(clk)
    launches = binding.launch_count() - l0
    ms = e0.elapsed_time(e1)
    prof = {name: ctx.prof_read(i) for i, name in enumerate(CLASSES)}
    ks_prof = ctx.prof_read(4)
    ks_by_limbs = ctx.prof_keyswitches()
    ctx.prof_enable(False)
    st = job.stats()
    ks_per_iter = int(st.keyswitches)
    ms_max, sec_iter, rates = replica_rates(ms, args.steps, world,
                                            {"ks": ks_per_iter, "limbs": transform_limbs(prof) / args.steps})
    # decrypted weights (on the device) for the FP64-twin check of the CPU leg
    main_w = {"iters": t, "sched": sched, "rows": {r: job.weights(r) for r in (0, 127)}}
    # ---------------- batched vs plain one-ciphertext-per-launch
    plain = None
    if not args.no_plain:
        job.set_batch(1)
        job.step(t, sched)
        t += 1
        torch.cuda.synchronize()
        p0 = time.time()
        job.step(t, sched)
        t += 1
        torch.cuda.synchronize()
        plain = time.time() - p0
        job.set_batch(chunk_used)
    # ---------------- end to end through the public API with host state
    e2e = None
    if not args.no_e2e:
        ctw = 2 * (ITER_LEVEL + 1) * (1 << LOGN)
        sin = pinned_u64(2 * ctw)
        sout = pinned_u64(2 * ctw)
        job.step_io(t, None, sout, sched)
        t += 1
        sin[:] = sout
        torch.cuda.synchronize()
        h0 = time.time()
        for _ in range(args.steps):
            job.step_io(t, sin, sout, sched)
            sin[:] = sout
            t += 1
        torch.cuda.synchronize()
        e2e_s = allreduce_max(time.time() - h0, world) / (args.steps * world)
        e2e = {"value": round(e2e_s, 5), "unit": "s/iter", "h2d_bytes_per_step": int(sin.nbytes),
               "d2h_bytes_per_step": int(sout.nbytes)}
    mini = None
    if not args.no_mini:
        mini = minibatch_time(ctx, X, y, args)
    bbar = None
    if world == 1 and not args.no_bbar:
        bbar = bbar_time(ctx, X, y)
    # the oracle on a sample of the job's own ciphertexts, before the job is released
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(X, y, samples=1, job=job, ctx=ctx)
    multi = first = None
    if world == 1 and not (args.no_multi and args.no_first_order):
        job.close()
        del job
        if not args.no_first_order:
            first = first_order_time(ctx, X, y, args)
        if not args.no_multi:
            multi = multijob_time(ctx)
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks.get("sm_max_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    roof = roofline(prof, ks_prof, ks_by_limbs, args.steps, ms_max / 1000.0 / args.steps, props.multi_processor_count,
                    sm_mhz)
    trained = None
    if world == 1 and not args.no_train:
        trained = whole_training(ctx, X, y)
    ntt = standalone_ntt(ctx)
    psweep = k4 = hoist_tc = images = None
    if not args.no_sweep:
        psweep = primitive_sweep(ctx)
        k4 = k4_tensor_floor(ctx)
        hoist_tc = hoist_forms(ctx)
    if world == 1 and not args.no_images:
        images = image_pair_time(ctx, args)
    booted = None
    if world == 1 and not args.no_boot:
        ctx.close()
        booted = boot_refresh_time(X, y, args)
    # the CPU leg (rank 0 of a single-GPU run): FP64-twin checks of the decrypted weights
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_twin:
        err = twin_checks(X, y, main_w, images, booted, trained)
    else:
        for name in ("full_batch", "mini_batch"):
            if images:
                images[name].pop("_w", None)
        for extra in (booted, trained):
            if extra:
                extra.pop("_w", None)
    out = {
        "metric": METRIC, "value": round(sec_iter, 5), "unit": "s/iter", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "full-batch QG-NAG, %d x %d synthetic Financial-shaped data, N=2^16, "
                               "chain 60+8x40 bits + 60-bit P, scale 2^40, 128x256 packing, g8 sigmoid" % (args.rows, N_FEAT),
                   "blocks": int(info.n_blocks), "blocks_per_launch": chunk_used,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "no flush: %.1f GiB of encrypted data blocks > 129 MB L2" % (info.n_blocks * ctw_bytes() / 2 ** 30)},
        "keyswitch_per_s": round(rates["ks"], 1) if sec_iter else None,
        "keyswitches_per_iter": ks_per_iter,
        "ntt_limbs_per_s": round(rates["limbs"], 1) if sec_iter else None,
        "keyswitch_hbm_frac": roof["keyswitch_hbm_frac_of_iteration"],
        "ntt_standalone": ntt,
        "ntt_hbm_frac": ntt["hbm_frac"],
        "primitive_sweep": psweep,
        "k4_tensor_ntt": k4,
        "hoist_ip_tensor_cores": hoist_tc,
        "image_pair_g16": images,
        "bootstrapped_refresh": booted,
        "whole_training": trained,
        "plain_one_ct_per_launch_s_per_iter": round(plain, 4) if plain else None,
        "mini_batch": mini,
        "multi_job": multi,
        "first_order_nag": first,
        "client_bbar": bbar,
        "batched_speedup_vs_plain": round(plain / sec_iter / world, 2) if plain else None,
        "setup_s": round(setup_s, 1),
        "autotune": autotune,
        "max_abs_err_vs_fp64_twin": err,
        "clocks": clocks, "gpu_launches": int(launches), "roofline": roof, "e2e": e2e,
        "context": PAPER_CONTEXT,
    }
    if cb is not None:
        out["cpu_baseline"] = cb
    return out


def minibatch_time(ctx, X, y, args):
    """Mini-batch QG-NAG (Algorithm 1) on the same data: 1,024-sample batches
    (8 blocks), the job's own schedule; seconds per iteration over 8 iterations
    after 3 warm-up iterations, batched and plain (one block per launch)."""
    import torch
    from paper_2406_13221_gb300 import binding
    job = binding.Job(ctx, X, y, binding.MINI_BATCH, 1024, binding.G8, LOG_SCALE, enc_seed=3, key_seed=2)
    sched = (1.0, 0.1, 413.0, 2.5)
    out = {}
    t = 0
    for mode, bpl, graph in (("batched", 8, False), ("batched_graph", 8, True), ("plain", 1, False)):
        job.set_batch(bpl)
        job.set_graph(graph)
        for _ in range(3):
            job.step(t, sched)
            t += 1
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(8):
            job.step(t, sched)
            t += 1
        e1.record()
        torch.cuda.synchronize()
        out[mode + "_s_per_iter"] = round(e0.elapsed_time(e1) / 8 / 1000.0, 5)
    out["keyswitches_per_iter"] = int(job.stats().keyswitches)
    out["batched_speedup_vs_plain"] = round(out["plain_s_per_iter"] / out["batched_s_per_iter"], 2)
    out["batched_graph_speedup_vs_plain"] = round(out["plain_s_per_iter"] / out["batched_graph_s_per_iter"], 2)
    job.close()
    return out


def bbar_time(ctx, X, y):
    """Client precompute of Bbar_k for every 1,024-row mini-batch (Sec. 3.1):
    on the device (host arrays in, host array out, transfers included) against
    the host routine on one thread (8 batches, extrapolated)."""
    from paper_2406_13221_gb300 import binding
    nb = -(-X.shape[0] // 1024)
    binding.lr_bbar_batches(ctx, X[:4096], y[:4096], 1024, 256)  # first-call set-up
    t0 = time.time()
    binding.lr_bbar_batches(ctx, X, y, 1024, 256)
    gpu = time.time() - t0
    t0 = time.time()
    for k in range(8):
        binding.lr_bbar(X, y, 1024 * k, 1024, 256)
    host = (time.time() - t0) * nb / 8
    return {"batches": nb, "device_s": round(gpu, 4), "host_one_thread_s": round(host, 3),
            "host_sample": "8 of %d batches, extrapolated" % nb}


def first_order_time(ctx, X, y, args):
    """The first-order NAG baseline (Sec. 2.3: no Bbar product, one level less)
    on the same full-batch workload at the rate of the paper's first-order
    Financial run (0.01, constant): seconds per iteration over 2 iterations
    after one warm-up iteration."""
    import torch
    from paper_2406_13221_gb300 import binding
    job = binding.Job(ctx, X, y, binding.FULL_BATCH | binding.FIRST_ORDER, 1024, binding.G8, LOG_SCALE, enc_seed=3,
                      key_seed=2, batch_blocks=args.chunk)
    sched = (0.01, 0.01, 81.0, 2.5)
    job.step(0, sched)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(1, 3):
        job.step(t, sched)
    e1.record()
    torch.cuda.synchronize()
    out = {"s_per_iter": round(e0.elapsed_time(e1) / 2 / 1000.0, 5), "keyswitches_per_iter": int(job.stats().keyswitches),
           "start_level": 5, "rate": 0.01}
    job.close()
    return out


def multijob_time(ctx):
    """16 independent full-batch jobs, n_j log-uniform in [5,000, 100,000],
    f_j uniform in {32, 64, 128, 200}: seconds per iteration with all jobs
    stepped together (key switches batched across jobs) against each job alone."""
    import torch
    from paper_2406_13221_gb300 import binding, synth
    shapes = synth.multijob_shapes(seed=5)
    jobs, alone = [], []
    for i, (n, f) in enumerate(shapes):
        X, y = synth.job(seed=100 + i, n=n, f=f)
        jobs.append(binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, LOG_SCALE, enc_seed=1000 + i,
                                key_seed=2, batch_blocks=16))
    multi = binding.Multi(ctx, jobs, blocks_per_launch=64)
    sched = (2.0, 1.0, 81.0, 2.5)
    multi.step(0, sched)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in (1, 2):
        multi.step(t, sched)
    e1.record()
    torch.cuda.synchronize()
    agg = e0.elapsed_time(e1) / 2 / 1000.0
    per = []
    for i, j in enumerate(jobs):
        j.step(3, sched)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        j.step(4, sched)
        a1.record()
        torch.cuda.synchronize()
        st = j.stats()
        per.append({"n": shapes[i][0], "f": shapes[i][1], "g": st.g, "blocks": st.n_blocks,
                    "s_per_iter_alone": round(a0.elapsed_time(a1) / 1000.0, 4)})
    multi.close()
    for j in jobs:
        j.close()
    tot = sum(p["s_per_iter_alone"] for p in per)
    return {"jobs": len(jobs), "blocks": sum(p["blocks"] for p in per), "samples": sum(p["n"] for p in per),
            "aggregate_s_per_iter": round(agg, 4), "sum_of_jobs_alone_s_per_iter": round(tot, 4),
            "batched_speedup": round(tot / agg, 3), "per_job": per}


def sweep(args):
    """Batched NTT limbs/s and key switches/s on GB300 (uniform random residues)."""
    import torch
    from paper_2406_13221_gb300 import binding, build
    build.build()
    point = tuple(int(x) for x in args.sweep_point.split(",")) if args.sweep_point else None
    for logn in (14, 15, 16):
        n = 1 << logn
        if point and logn != point[0]:
            continue
        for limbs in (8, 16, 24, 32, 40):
            if point and limbs != point[1]:
                continue
            nq = min(limbs, 38)
            ctx = binding.Context(logn, nq)
            for batch in (1, 8, 64, 512):
                if point and batch != point[2]:
                    continue
                nl = batch * limbs
                if nl * n * 8 > 8 << 30:
                    continue
                buf = torch.randint(0, 1 << 30, (nl * n,), dtype=torch.int64, device="cuda")
                prime_of = list(range(nq))
                for _ in range(2):
                    ctx.ntt_forward(buf.data_ptr(), nl, prime_of)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = max(2, min(50, 4096 // nl))
                e0.record()
                for _ in range(reps):
                    ctx.ntt_forward(buf.data_ptr(), nl, prime_of)
                    ctx.ntt_inverse(buf.data_ptr(), nl, prime_of)
                e1.record()
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) / 1000.0
                print(json.dumps({"sweep": "ntt", "log_n": logn, "limbs": limbs, "ciphertexts_per_launch": batch,
                                  "ntt_limbs_per_s": round(2 * reps * nl / sec, 1),
                                  "hbm_frac_of_alg_bytes": round(2 * reps * nl * 16 * n / sec / 1e9 /
                                                                 measured_peaks().get("hbm_gbs", 6800.0), 4)}), flush=True)
                del buf
            if not point:
                sweep_ct_ops(ctx, logn, limbs)
            ctx.close()
    if point:
        return
    # key switching at the bench chain (N = 2^16, 9 primes + P), relinearisation key
    ctx = binding.Context(LOGN, NQ)
    ctx.keygen(2, [])
    n = 1 << LOGN
    for level in (7, 4):
        nl = level + 1
        for batch in (1, 8, 32, 128, 256):
            din = torch.randint(0, 1 << 30, (batch * nl * n,), dtype=torch.int64, device="cuda")
            dout = torch.zeros(batch * 2 * nl * n, dtype=torch.int64, device="cuda")
            ctx.keyswitch_batch(din.data_ptr(), dout.data_ptr(), batch, level, 0)
            torch.cuda.synchronize()
            reps = max(2, 256 // batch)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ctx.keyswitch_batch(din.data_ptr(), dout.data_ptr(), batch, level, 0)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0
            print(json.dumps({"sweep": "keyswitch", "log_n": LOGN, "limbs": nl, "batch": batch,
                              "keyswitch_per_s": round(reps * batch / sec, 1)}), flush=True)
            del din, dout


def sweep_ct_ops(ctx, logn, limbs, rot=4):
    """The ciphertext operations of the primitive sweep at the full chain of
    `limbs` primes: ct x ct multiply with relinearisation, rotation by `rot`
    slots and rescale, each batched over 1, 8, 64 and 512 ciphertexts
    (he_mul_relin_batch, he_rotate_batch, he_rescale_batch) on uniform random
    residues.  Algorithmic bytes at L limbs (8N bytes a limb, keys once per
    call): Mul 2 ciphertexts in and 1 out plus the 2L(L+1) key limbs; rotation
    1 in, 1 out plus the key; rescale 2L limbs in, 2(L-1) out.  Points whose
    working set (operands, evaluator and key-switch scratch) would pass
    120 GB are skipped."""
    import torch
    nl = min(limbs, 38)  # the sweep's contexts hold at most 38 ciphertext primes
    n, level = 1 << logn, nl - 1
    ctx.keygen(2, [rot])
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    for batch in (1, 8, 64, 512):
        words = batch * nl * n * (6 + 8 + 4) + min(128, batch) * nl * (nl + 1) * n
        if words * 8 > 120 << 30:
            continue
        a = torch.randint(0, 1 << 30, (batch * 2 * nl * n,), dtype=torch.int64, device="cuda")
        b = torch.randint(0, 1 << 30, (batch * 2 * nl * n,), dtype=torch.int64, device="cuda")
        o = torch.zeros_like(a)
        keyb = 2 * nl * (nl + 1)
        ops = (("mul_relin", lambda: ctx.mul_relin_batch(a.data_ptr(), b.data_ptr(), o.data_ptr(), batch, level),
                batch * 6 * nl + keyb),
               ("rotate", lambda: ctx.rotate_batch(a.data_ptr(), o.data_ptr(), batch, level, rot),
                batch * 4 * nl + keyb),
               ("rescale", lambda: ctx.rescale_batch(a.data_ptr(), o.data_ptr(), batch, level),
                batch * (4 * nl - 2)))
        for name, call, limbs_moved in ops:
            call()
            torch.cuda.synchronize()
            reps = max(2, min(20, 256 // batch))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0 / reps
            print(json.dumps({"sweep": name, "log_n": logn, "limbs": nl, "ciphertexts_per_launch": batch,
                              "ciphertexts_per_s": round(batch / sec, 1),
                              "hbm_frac_of_alg_bytes": round(limbs_moved * 8 * n / sec / 1e9 / hbm, 4)}), flush=True)
        del a, b, o


def ks_primitive(ctx, level, items, kind, reps=3):
    """Seconds per call and key switches per second of one batched primitive at
    N = 2^16: a relinearisation key switch of `items` polynomials (relin) or a
    hoisted sum of the seven rotations 1..7 of `items` ciphertexts (rot7),
    uniformly random residues in evaluation form."""
    import torch
    n, nl = 1 << LOGN, level + 1
    if kind == "relin":
        din = torch.randint(0, 1 << 30, (items * nl * n,), dtype=torch.int64, device="cuda")
        dout = torch.zeros(items * 2 * nl * n, dtype=torch.int64, device="cuda")
        call = lambda: ctx.keyswitch_batch(din.data_ptr(), dout.data_ptr(), items, level, 0)  # noqa: E731
        ks = items
    else:
        din = torch.randint(0, 1 << 30, (items * 2 * nl * n,), dtype=torch.int64, device="cuda")
        dout = torch.zeros_like(din)
        call = lambda: ctx.rotsum_batch(din.data_ptr(), dout.data_ptr(), items, level, list(range(1, 8)))  # noqa: E731
        ks = 7 * items
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0 / reps
    del din, dout
    return sec, ks / sec


def ks_point(args):
    """One primitive point (profiling entry): prints its JSON line."""
    from paper_2406_13221_gb300 import binding, build
    build.build()
    level, items, kind = args.ks_point.split(",")
    level, items = int(level), int(items)
    ctx = binding.Context(LOGN, NQ)
    ctx.keygen(2, list(range(1, 8)))
    if kind.endswith("tc"):  # hoisted inner product on the tensor cores
        kind = kind[:-2]
        ctx.set_hoist_form(1)
    sec, rate = ks_primitive(ctx, level, items, kind)
    ctx.check_device()
    print(json.dumps({"ks_point": kind, "log_n": LOGN, "limbs": level + 1, "items": items, "s_per_call": round(sec, 6),
                      "keyswitch_per_s": round(rate, 1)}), flush=True)
    ctx.close()


def k4_tensor_floor(ctx, limbs=64, reps=5):
    """The tensor pipe's share of an exact four-step NTT at N = 2^16 = 256 x 256,
    measured against the butterfly transforms of the same limbs.

    Each pass of a four-step NTT multiplies every limb, as a 256 x 256 matrix,
    by the 256 x 256 DFT matrix modulo q.  With 40-bit words cut into five
    byte slices the exact product needs the 25 slice-by-slice GEMMs (each sum
    of 256 products of bytes stays below 2^24, so FP32 accumulation is exact);
    the twiddle product between the passes and the carry/modular recombination
    come on top.  The GEMMs alone therefore bound a tensor-core pass from
    below.  They are timed here with cuBLAS (the measured peak reference) as
    one GEMM per pass over all limbs: [5*256 x 256] slices of the DFT matrix
    times [256 x 5*256*limbs] slices of the data, for each exact input type
    the installed PyTorch offers (INT8 -> INT32, FP16 -> FP32, TF32 -> FP32),
    after checking one product against an integer matmul.  sm_103a has no
    INT8 tcgen05.mma (ptxas: ".kind::i8 not supported on .target sm_103a"),
    so cuBLAS's INT8 rate is whatever the part offers without it."""
    import torch
    n = 1 << LOGN
    side = 256
    out = {"n": n, "limbs": limbs, "slices_per_word": 5, "slice_gemms_per_pass": 25,
           "tcgen05_kind_i8_on_sm_103a": "unsupported (ptxas: Feature '.kind::i8' not supported on .target 'sm_103a')"}
    # butterfly reference: forward + inverse = four passes per limb
    buf = torch.randint(0, 1 << 30, (limbs * n,), dtype=torch.int64, device="cuda")
    prime_of = list(range(NQ))
    for _ in range(2):
        ctx.ntt_forward(buf.data_ptr(), limbs, prime_of)
        ctx.ntt_inverse(buf.data_ptr(), limbs, prime_of)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.ntt_forward(buf.data_ptr(), limbs, prime_of)
        ctx.ntt_inverse(buf.data_ptr(), limbs, prime_of)
    e1.record()
    torch.cuda.synchronize()
    bfly_pass_us = e0.elapsed_time(e1) * 1000.0 / (reps * 4 * limbs)
    out["butterfly_us_per_limb_pass"] = round(bfly_pass_us, 4)
    del buf
    g = torch.Generator(device="cuda").manual_seed(5)
    M, K, Ncols = 5 * side, side, 5 * side * limbs
    flops = 2.0 * M * K * Ncols
    candidates = []
    if hasattr(torch, "_int_mm"):
        candidates.append(("int8_to_int32", lambda a, b: torch._int_mm(a, b), torch.int8, -128, 128))
    try:
        a = torch.ones(16, 16, dtype=torch.float16, device="cuda")
        torch.mm(a, a, out_dtype=torch.float32)
        candidates.append(("fp16_to_fp32", lambda a, b: torch.mm(a, b, out_dtype=torch.float32), torch.float16, 0, 256))
    except (TypeError, RuntimeError):
        out["fp16_to_fp32"] = "torch.mm has no out_dtype in this PyTorch"
    candidates.append(("tf32_to_fp32", None, torch.float32, 0, 256))
    for name, fn, dt, lo, hi in candidates:
        A = torch.randint(lo, hi, (M, K), generator=g, device="cuda", dtype=torch.int32)
        B = torch.randint(lo, hi, (K, Ncols), generator=g, device="cuda", dtype=torch.int32)
        Ad, Bd = A.to(dt), B.to(dt)
        if fn is None:
            prev = torch.backends.cuda.matmul.allow_tf32
            torch.backends.cuda.matmul.allow_tf32 = True
            fn = lambda a, b: torch.mm(a, b)  # noqa: E731
        try:
            C = fn(Ad, Bd)
            torch.cuda.synchronize()
            cols = slice(0, 512)
            ref = A.cpu().numpy().astype(np.int64) @ B[:, cols].cpu().numpy().astype(np.int64)
            exact = bool(np.array_equal(C[:, cols].double().cpu().numpy().astype(np.int64), ref))
            for _ in range(2):
                fn(Ad, Bd)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                fn(Ad, Bd)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0 / reps
            out[name] = {"exact": exact, "tops": round(flops / sec / 1e12, 1),
                         "gemm_us_per_limb_pass": round(sec * 1e6 / limbs, 4),
                         "vs_butterfly_pass": round(sec * 1e6 / limbs / bfly_pass_us, 2)}
        except RuntimeError as e:
            out[name] = "unavailable: %s" % str(e).splitlines()[0][:120]
        finally:
            if name == "tf32_to_fp32":
                torch.backends.cuda.matmul.allow_tf32 = prev
        del A, B, Ad, Bd
    return out


def whole_training(ctx, X, y, iters=3):
    """The paper's whole problem through one C-ABI call, he_lr_train, on the
    headline data.  The call generates the keys, encodes and encrypts the data
    blocks and Enc(n Bbar) from the host arrays, runs `iters` full-batch
    iterations and decrypts the weights into a host array.  Reported:
    wall-clock seconds of the call, with the device idle on both sides."""
    import time
    import torch
    from paper_2406_13221_gb300 import binding
    sched = (2.0, 1.0, 81.0, 2.5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w, st = binding.lr_train(ctx, X, y, iters, sched=sched, enc_seed=7, key_seed=2)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return {"call": "he_lr_train", "iterations": iters, "seconds": round(sec, 3),
            "blocks": int(st.n_blocks), "keyswitches": int(st.keyswitches),
            "includes": "keygen, encoding and encryption of the data from host arrays, the iterations, decryption",
            "_w": (w, iters, sched)}


def hoist_forms(ctx, items=128, reps=5):
    """The two forms of the hoisted inner product on the bench's rotation
    groups: he_rotsum_batch of `items` ciphertexts with the 7 rotations of one
    hoisted group (1..7) at 6 and at 4 limbs, with the inner product on the CUDA
    cores (the default) and on the tensor cores (he_set_hoist_form(1):
    tcgen05.mma on FP16 byte slices of digits and keys, exact, for the 40-bit
    targets).  Seconds per call of each, whether their output words are equal,
    and whether the tensor-core kernel ran."""
    import torch
    n = 1 << LOGN
    rots = list(range(1, 8))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for level in (5, 3):
        nl = level + 1
        din = torch.randint(0, 1 << 30, (items * 2 * nl * n,), dtype=torch.int64, device="cuda")
        rec = {"limbs": nl, "items": items, "rotations": len(rots)}
        res = []
        for form, name in ((0, "cuda_cores"), (1, "tensor_cores")):
            dout = torch.zeros_like(din)
            ctx.set_hoist_form(form)
            try:
                n0 = ctx.hoist_tensor_launches()
                ctx.rotsum_batch(din.data_ptr(), dout.data_ptr(), items, level, rots)
                torch.cuda.synchronize()
                ran = ctx.hoist_tensor_launches() > n0
                e0.record()
                for _ in range(reps):
                    ctx.rotsum_batch(din.data_ptr(), dout.data_ptr(), items, level, rots)
                e1.record()
                torch.cuda.synchronize()
            finally:
                ctx.set_hoist_form(-1)
            ctx.check_device()
            rec[name + "_s_per_call"] = round(e0.elapsed_time(e1) / 1000.0 / reps, 6)
            if form == 1:
                rec["tensor_kernel_ran"] = bool(ran)
            res.append(dout)
        rec["words_equal"] = bool(torch.equal(res[0], res[1]))
        rec["tensor_vs_cuda_cores"] = round(rec["tensor_cores_s_per_call"] / rec["cuda_cores_s_per_call"], 3)
        out.append(rec)
        del din, res
    return out


def primitive_sweep(ctx):
    """A compact HE primitive sweep (N = 2^14..2^16 transforms, key switching
    and hoisted rotation sums at two limb counts), each point with its HBM
    fraction at the algorithmic bytes of the survey's measurement table: a
    transform of one limb reads and writes it once (16N bytes); a key switch
    at L limbs reads its input and writes two polynomials (3L limbs) and reads
    its 2L(L+1) key limbs once per call; a hoisted sum of r rotations reads
    and writes its ciphertext once and r keys."""
    import torch
    from paper_2406_13221_gb300 import binding
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    out = {"ntt": [], "keyswitch": []}
    for logn in (14, 15, 16):
        n = 1 << logn
        c = ctx if logn == LOGN else binding.Context(logn, 8)
        limbs = 512  # 64 ciphertexts of 8 limbs
        buf = torch.randint(0, 1 << 30, (limbs * n,), dtype=torch.int64, device="cuda")
        prime_of = list(range(8))
        for _ in range(2):
            c.ntt_forward(buf.data_ptr(), limbs, prime_of)
            c.ntt_inverse(buf.data_ptr(), limbs, prime_of)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 4
        e0.record()
        for _ in range(reps):
            c.ntt_forward(buf.data_ptr(), limbs, prime_of)
            c.ntt_inverse(buf.data_ptr(), limbs, prime_of)
        e1.record()
        torch.cuda.synchronize()
        rate = 2 * reps * limbs / (e0.elapsed_time(e1) / 1000.0)
        out["ntt"].append({"log_n": logn, "limbs_per_launch": limbs, "ntt_limbs_per_s": round(rate, 1),
                           "hbm_frac": round(rate * 16 * n / 1e9 / hbm, 4)})
        del buf
        if c is not ctx:
            c.close()
    n = 1 << LOGN
    for kind, level in (("relin", 6), ("relin", 3), ("rot7", 5), ("rot7", 3)):
        items, nl = 128, level + 1
        sec, rate = ks_primitive(ctx, level, items, kind)
        r = 1 if kind == "relin" else 7
        alg = (3.0 * nl * items + r * 2.0 * nl * (nl + 1)) * 8 * n  # per call
        out["keyswitch"].append({"kind": kind, "log_n": LOGN, "limbs": nl, "items": items,
                                 "keyswitch_per_s": round(rate, 1), "hbm_frac": round(alg / sec / 1e9 / hbm, 4)})
    return out


def image_pair_time(ctx, args):
    """The MNIST-shaped workload (Sec. 5.2, Table 2: 11,982 x 196, sigmoid
    polynomial g16) on synthetic images: full batch and mini-batch (1,024
    samples) seconds per iteration over 2 iterations after one warm-up, and
    the decrypted weights against the FP64 twin."""
    import torch
    from paper_2406_13221_gb300 import binding, synth
    X, y = synth.image_pair()
    out = {"workload": "11,982 x 196 synthetic two-class images, g16, N=2^16, 128 x 256 packing"}
    for mode, name, sched in ((binding.FULL_BATCH, "full_batch", (2.0, 1.0, 81.0, 2.5)),
                              (binding.MINI_BATCH, "mini_batch", (1.0, 0.1, 81.0, 2.5))):
        job = binding.Job(ctx, X, y, mode, 1024, binding.G16, LOG_SCALE, enc_seed=21, key_seed=2)
        job.step(0, sched)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for t in (1, 2):
            job.step(t, sched)
        e1.record()
        torch.cuda.synchronize()
        res = {"s_per_iter": round(e0.elapsed_time(e1) / 2 / 1000.0, 5), "blocks": int(job.stats().n_blocks),
               "keyswitches_per_iter": int(job.stats().keyswitches)}
        res["_w"] = (job.weights(0), "full" if mode == binding.FULL_BATCH else "mini", sched)
        out[name] = res
        job.close()
    return out


BOOT_BITS = [50] + [40] * 6 + [55] * 14  # q0, the iteration's six levels, the bootstrap's fourteen
BOOT_PARAMS = dict(slots=256, K=16, r=6, deg=19, scale_out=2.0 ** LOG_SCALE, level_out=ITER_LEVEL)


def boot_refresh_time(X, y, args, iters=2):
    """The full-batch workload with W and V refreshed by bootstrapping (Sec. 4.3
    Step 7 as the paper runs it, no client round trip) on the bootstrappable
    chain (q0 50 bits, six 40-bit levels for the iteration, fourteen 55-bit
    levels for the bootstrap; a secret of 64 nonzero coefficients): seconds per
    iteration over `iters` iterations after one warm-up, the bootstrap's share,
    and the decrypted weights for the FP64-twin check of the CPU leg."""
    import torch
    from paper_2406_13221_gb300 import binding
    t0 = time.time()
    ctx = binding.Context(LOGN, len(BOOT_BITS), bits=BOOT_BITS, secret_weight=64)
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, LOG_SCALE, enc_seed=3, key_seed=2,
                      batch_blocks=args.chunk)
    job.set_refresh(BOOT_PARAMS)
    setup = time.time() - t0
    sched = (2.0, 1.0, 81.0, 2.5)
    job.step(0, sched)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(1, 1 + iters):
        job.step(t, sched)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0 / iters
    st = job.stats()
    # a bootstrap of W and V alone (the refresh), timed on its own
    n = 1 << LOGN
    din = torch.randint(0, 1 << 30, (2 * 2 * n,), dtype=torch.int64, device="cuda")
    dout = torch.zeros(2 * 2 * (ITER_LEVEL + 1) * n, dtype=torch.int64, device="cuda")
    ctx.bootstrap_batch(din.data_ptr(), 0, dout.data_ptr(), 2, **BOOT_PARAMS)
    torch.cuda.synchronize()
    e0.record()
    ctx.bootstrap_batch(din.data_ptr(), 0, dout.data_ptr(), 2, **BOOT_PARAMS)
    e1.record()
    torch.cuda.synchronize()
    boot_s = e0.elapsed_time(e1) / 1000.0
    out = {"workload": "full-batch QG-NAG at %d x %d, W and V refreshed by bootstrapping" % X.shape,
           "chain_bits": BOOT_BITS, "secret_nonzeros": 64, "bootstrap": BOOT_PARAMS,
           "s_per_iter": round(sec, 5), "bootstrap_of_w_and_v_s": round(boot_s, 5),
           "update_share": round(st.sec_update_avg / st.sec_iter_avg, 3) if st.sec_iter_avg else None,
           "setup_s": round(setup, 1), "_w": (job.weights(0), 1 + iters, sched)}
    job.close()
    ctx.close()
    return out


def ctw_bytes():
    return 2 * (ITER_LEVEL + 1) * (1 << LOGN) * 8


def info_chunk(job, args):
    return min(args.chunk if args.chunk else 256, int(job.info.n_blocks))


_PINNED = []


def pinned_u64(n):
    import torch
    t = torch.empty(n, dtype=torch.int64, pin_memory=True)
    _PINNED.append(t)  # keep the pinned storage alive
    return t.numpy().view(np.uint64)


# The integer multiply pipe (fmaheavy: every IMAD and 32x32 -> 64 product)
# issues 16 lanes per clock in each of the 4 sub-partitions of an SM.
FMAHEAVY_LANES_PER_SM = 64
CLASSES = ["ntt_fwd", "ntt_inv", "modup", "ks_inner"]  # timing classes 0-3; class 4 = whole key switches
KERNEL_OF_CLASS = {"ks_inner": "k_ks_inner_rows", "modup": "k_ks_modup_cols",
                   "ntt_fwd": "k_ks_down_rows+k_ntt_fwd_*", "ntt_inv": "k_ntt_inv_*"}


def transform_limbs(prof):
    """Limb transforms (forward and inverse, standalone or fused into key
    switching) counted as whole transforms: the fused kernels report the
    column or row halves they run."""
    return (prof["ntt_fwd"][1] + prof["ntt_inv"][1]
            + 0.5 * (prof["modup"][1] + prof["modup"][3] + prof["ks_inner"][1]))


def class_butterflies(name, units, units2):
    """Butterflies a timing class executed, from its work counts: a column or
    row half of a transform is (log N / 2) stages of N/2 butterflies."""
    n = 1 << LOGN
    half = (LOGN // 2) * (n / 2)
    if name.startswith("ntt"):  # whole-limb transform equivalents
        return units * 2 * half
    if name == "modup":         # forward column halves + inverse column halves
        return (units + units2) * half
    return units * half         # ks_inner: row halves


def recorded_keyswitch_traffic(by_limbs):
    """Measured DRAM bytes per key switch (ncu, profiles/traffic.txt lines
    `keyswitch <code-sha> nl=<L> <bytes per key switch>`), valid for the
    current kernel sources only.  A record `nl=all` (the DRAM bytes of every
    kernel of a whole iteration over the key switches it issued) serves any
    mix; otherwise the per-limb-count records are weighted by the key
    switches of each limb count, and None unless every limb count has one."""
    h = kernel_sources_hash()
    rec = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            p = line.split()
            if len(p) >= 4 and not line.startswith("#") and p[0] == "keyswitch" and p[1] == h and p[2].startswith("nl="):
                rec[p[2][3:]] = float(p[3])
    except OSError:
        return None
    tot = sum(by_limbs.values())
    if not tot:
        return None
    if "all" in rec:
        return rec["all"]
    if any(str(nl) not in rec for nl in by_limbs):
        return None
    return sum(rec[str(nl)] * k for nl, k in by_limbs.items()) / tot


def recorded_fmaheavy(kernel):
    """Integer-multiply-pipe (fmaheavy) warp instructions per warp-wide step of
    32 butterflies of `kernel`, from an ncu capture (profiles/traffic.txt lines
    `fmaheavy <kernel> <code-sha> <value>`: the pipe's busy cycles x 2 warp
    instructions per SM cycle over the butterflies / 32), valid for the
    current kernel sources only."""
    h = kernel_sources_hash()
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            p = line.split()
            if len(p) >= 4 and not line.startswith("#") and p[0] == "fmaheavy" and p[1] == kernel and p[2] == h:
                return float(p[3])
    except OSError:
        pass
    return None


def roofline(prof, ks, ks_by_limbs, steps, sec_iter, sms, sm_mhz):
    """The key switch as the unit of work (the fused kernels of one key switch
    run as one pipeline): algorithmic bytes of every key switch the timed steps
    issued (3L limbs per item, 2L(L+1) key limbs per wave) over the time spent
    inside key switches, against the measured HBM copy bandwidth.  Beside it:
    the same bytes over the whole iteration, and the column kernel of ModUp and
    ModDown (k_ks_modup_cols, the kernel with the largest share) on the
    integer multiply pipe: its butterflies per second times the measured
    instructions per 32 butterflies, against SMs x 2 warp instructions per
    clock (16 lanes per sub-partition)."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n = 1 << LOGN
    ks_ms, ks_n, _, ks_limbs, ks_alg_limbs = ks
    alg = ks_alg_limbs * 8.0 * n
    sec = ks_ms / 1000.0
    achieved = alg / sec / 1e9 if sec else 0.0
    traffic = recorded_keyswitch_traffic(ks_by_limbs)
    best = max(CLASSES, key=lambda k: prof[k][0])
    ms, units, launches, units2, _ = prof["modup"]
    bf = class_butterflies("modup", units, units2)
    ipb = recorded_fmaheavy("k_ks_modup_cols")
    pipe_peak = sms * FMAHEAVY_LANES_PER_SM * sm_mhz * 1e6 / 32.0  # warp instructions per second
    issue = None
    if ipb is not None and ms:
        ach = bf / 32.0 * ipb / (ms / 1000.0)
        issue = {"kernel": "k_ks_modup_cols", "pipe": "fmaheavy (integer multiply)",
                 "warp_instr_per_32_butterflies": ipb, "achieved": round(ach / 1e12, 4),
                 "peak": round(pipe_peak / 1e12, 4), "unit": "T warp-instr/s", "frac": round(ach / pipe_peak, 4),
                 "sms": sms, "sm_mhz": sm_mhz}
    ts = sum(prof[k][0] for k in CLASSES)
    return {"kernel": "key switch (k_ntt_inv_rows + k_ks_modup_cols + k_ks_inner_rows + k_ks_down_rows)",
            "unit_of_work": "one key switch", "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": round(traffic) if traffic is not None else None,
            "traffic_scope": "DRAM bytes of every kernel of an iteration per key switch issued (ncu, 256-block "
                             "iteration scaled per key switch)",
            "alg_bytes_per_unit": round(alg / ks_n) if ks_n else None, "units": int(ks_n),
            "avg_unit_us": round(1000.0 * ks_ms / ks_n, 3) if ks_n else None,
            "keyswitches_by_limbs": {str(k): int(v / steps) for k, v in sorted(ks_by_limbs.items())},
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "fallback" not in peaks else "fallback 6.8 TB/s",
            "share_of_step": round(sec / (sec_iter * steps), 3) if sec_iter else None,
            "keyswitch_hbm_frac_of_iteration": round(alg / steps / sec_iter / 1e9 / hbm, 4) if sec_iter else None,
            "dominant_class": best, "dominant_share": round(ms / ts, 3) if ts else None,
            "issue_view": issue,
            "classes_ms_per_step": {k: round(prof[k][0] / steps, 2) for k in CLASSES}}


def standalone_ntt(ctx, limbs=256, reps=10):
    """Batched forward + inverse transforms of `limbs` limbs at N = 2^16 (256
    MiB, beyond L2) outside key switching: limbs per second and the HBM
    fraction at 16N algorithmic bytes per limb transform (read + write once)."""
    import torch
    n = 1 << LOGN
    buf = torch.randint(0, 1 << 30, (limbs * n,), dtype=torch.int64, device="cuda")
    prime_of = list(range(NQ))
    for _ in range(2):
        ctx.ntt_forward(buf.data_ptr(), limbs, prime_of)
        ctx.ntt_inverse(buf.data_ptr(), limbs, prime_of)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.ntt_forward(buf.data_ptr(), limbs, prime_of)
        ctx.ntt_inverse(buf.data_ptr(), limbs, prime_of)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0
    rate = 2 * reps * limbs / sec
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    del buf
    return {"limbs_per_launch": limbs, "log_n": LOGN, "ntt_limbs_per_s": round(rate, 1),
            "achieved_gbs": round(rate * 16 * n / 1e9, 1), "peak_gbs": hbm,
            "hbm_frac": round(rate * 16 * n / 1e9 / hbm, 4)}


def twin_checks(X, y, main_w, images, booted=None, trained=None):
    """Part of the CPU leg: the decrypted weights the GPU jobs produced (rows 0
    and m-1 of the full-batch job; row 0 of each MNIST-shaped job) against the
    FP64 plaintext run of the same iterations (oracle/plain.py); fills in the
    image jobs' errors and returns the full-batch job's."""
    from oracle import plain, qgnag
    data = qgnag.TrainData(X, y, g=256, m=128, batch_rows=1024)
    wp = plain.train(data, main_w["iters"], sched=main_w["sched"])
    err = max(float(np.abs(w - wp).max()) for w in main_w["rows"].values())
    if images:
        from paper_2406_13221_gb300 import synth
        Xi, yi = synth.image_pair()
        di = qgnag.TrainData(Xi, yi, g=256, m=128, batch_rows=1024)
        for name in ("full_batch", "mini_batch"):
            w, mode, sched = images[name].pop("_w")
            wpi = plain.train(di, 3, mode=mode, sched=sched, poly=qgnag.G16)
            images[name]["max_abs_err_vs_fp64_twin"] = float(np.abs(w - wpi).max())
    if booted:
        w, iters, sched = booted.pop("_w")
        booted["max_abs_err_vs_fp64_twin"] = float(np.abs(w - plain.train(data, iters, sched=sched)).max())
    if trained:
        w, iters, sched = trained.pop("_w")
        trained["max_abs_err_vs_fp64_twin"] = float(np.abs(w - plain.train(data, iters, sched=sched)).max())
    return err


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, world):
    """Maximum of v over the ranks (NCCL on the GPU run, gloo on the CPU tests)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rates(ms_local, steps, world, per_iter):
    """Whole-job figures of `world` independent replicas that each ran `steps`
    iterations: the slowest rank's time bounds the job, so seconds per
    iteration = max-over-ranks ms / (steps * world); every per-iteration count
    in `per_iter` becomes a whole-job rate (count / seconds per iteration)."""
    ms_max = allreduce_max(ms_local, world)
    sec_iter = ms_max / 1000.0 / (steps * world)
    rates = {k: (v / sec_iter if sec_iter else None) for k, v in per_iter.items()}
    return ms_max, sec_iter, rates


# ------------------------------------------------------------------ CPU oracle
def cpu_baseline(X, y, samples=1, steps=1, warmup=0, job=None, ctx=None):
    """The CPU oracle on a bounded sample of the same workload: Steps 1-6 on
    `samples` data blocks plus Steps 7-9 and the refresh once, at N = 2^16;
    sec/iter extrapolated linearly to all blocks (key generation untimed).
    With the GPU job at hand the oracle takes the job's own ciphertexts (its
    first blocks, Enc(n Bbar), its current W and V), and the GPU's iteration on
    the same inputs (he_lr_iteration) is compared with the oracle's W', V' word
    for word; the small configuration then runs in full on both sides."""
    from oracle import qgnag
    from oracle.ckks import Ckks, Ct as OCt
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    data = qgnag.TrainData(X, y, g=256, m=128, batch_rows=1024)
    he = Ckks(LOGN, NQ)
    circ = qgnag.Circuit(he, 256, 128, 2.0 ** LOG_SCALE)
    k0 = time.time()
    he.keygen(2, circ.rotations())
    keygen_s = time.time() - k0
    L, D = circ.L, 2.0 ** LOG_SCALE
    if job is not None:
        Z = [OCt(job.input(0, b).export(), L, D) for b in range(samples)]
        B = OCt(job.input(1, 0).export(), L, D)
        (Ww, lw, sw), (Vw, lv, sv) = job.state_words()
        W, V = OCt(Ww, lw, sw), OCt(Vw, lv, sv)
    else:
        Z = [he.encrypt(he.encode(data.blocks[b], L, D), qgnag.obj_seed(3, 1, b)) for b in range(samples)]
        B = he.encrypt(he.encode(np.tile(data.n * data.bbar_full, 128), L, D), qgnag.obj_seed(3, 2, 0))
        W = he.encrypt(he.encode(np.zeros(he.nslots), L, D), 5)
        V = he.encrypt(he.encode(np.zeros(he.nslots), L, D), 6)
    alpha, eta = 2.0, 0.99
    vals, first = [], None
    for i in range(warmup + steps):
        t0 = time.time()
        acc = None
        for z in Z:
            g = circ.block_grad(z, W)
            acc = g if acc is None else he.add(acc, g)
        t1 = time.time()
        Wn, Vn = circ.finish(acc, B, W, V, alpha, eta, 1.0 / data.n)
        circ.refresh(Wn, 7)
        circ.refresh(Vn, 8)
        t2 = time.time()
        first = first or (Wn, Vn)
        est = (t1 - t0) / samples * data.blocks.shape[0] + (t2 - t1)
        if i >= warmup:
            vals.append(est)
    out = {"value": round(float(np.mean(vals)), 1), "unit": "s/iter", "cores": cores, "kind": "oracle",
           "sample": "Steps 1-6 on %d of %d blocks + Steps 7-9 and refresh once, N=2^16, extrapolated "
                     "linearly to all blocks; keygen (%.0f s) untimed" % (samples, data.blocks.shape[0], keygen_s)}
    if job is not None:
        from paper_2406_13221_gb300 import binding
        imp = lambda c: ctx.import_ct(c.data, c.level, c.scale)  # noqa: E731
        gW, gV = binding.lr_iteration(ctx, [imp(z) for z in Z], imp(B), imp(W), imp(V), 256, 128, alpha, eta,
                                      1.0 / data.n, qgnag.G8)
        out["bitwise_equal_gpu"] = bool(np.array_equal(gW.export(), first[0].data) and
                                        np.array_equal(gV.export(), first[1].data))
        out["check"] = ("the sample's W', V' (Steps 1-9 on the job's own block, Enc(n Bbar), W and V) "
                        "against he_lr_iteration on the same ciphertexts, word for word")
        out["small_config"] = small_config_run()
    return out


def small_config_run(iters=2):
    """The small configuration in full (1,024 x 15 + bias, N=2^13, 4 blocks of
    256 x 16, 2 full-batch iterations): the GPU job and the oracle from the
    job's own encrypted inputs, state compared word for word after every
    iteration; seconds per iteration of each (refresh included)."""
    import torch
    from oracle import qgnag
    from oracle.ckks import Ckks, Ct as OCt
    from paper_2406_13221_gb300 import binding, synth
    Xs, ys = synth.small()
    ctx = binding.Context(13, NQ)
    job = binding.Job(ctx, Xs, ys, binding.FULL_BATCH, 1024, binding.G8, LOG_SCALE, enc_seed=3, key_seed=2)
    he = Ckks(13, NQ)
    data = qgnag.TrainData(Xs, ys, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, 2.0 ** LOG_SCALE)
    he.keygen(2, circ.rotations())
    L, D = circ.L, 2.0 ** LOG_SCALE
    nb = data.blocks.shape[0]
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(nb)]
    B = OCt(job.input(1, 0).export(), L, D)
    (Ww, _, _), (Vw, _, _) = job.state_words()
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    etas = qgnag.nag_scalars(iters)
    gpu, orc, equal = [], [], True
    for t in range(iters):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        job.step(t)
        e1.record()
        torch.cuda.synchronize()
        gpu.append(e0.elapsed_time(e1) / 1e3)
        t0 = time.time()
        Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(t), etas[t], 1.0 / data.n)
        W = circ.refresh(Wn, qgnag.obj_seed(3, qgnag.SEED_WREF, t))
        V = circ.refresh(Vn, qgnag.obj_seed(3, qgnag.SEED_VREF, t))
        orc.append(time.time() - t0)
        (Ww, _, _), (Vw, _, _) = job.state_words()
        equal = equal and np.array_equal(Ww, W.data) and np.array_equal(Vw, V.data)
    job.close()
    ctx.close()
    return {"workload": "1,024 x 15 (+bias) synthetic, N=2^13, %d blocks of 256 x 16, %d full-batch iterations"
                        % (nb, iters),
            "gpu_s_per_iter": round(float(np.mean(gpu)), 5), "oracle_s_per_iter": round(float(np.mean(orc)), 3),
            "bitwise_equal": bool(equal)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2406_13221_gb300 import synth
    X, y = synth.financial(seed=1, n=args.rows)
    cb = cpu_baseline(X, y, samples=1, steps=args.steps, warmup=args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "s/iter", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "full-batch QG-NAG, %d x %d synthetic Financial-shaped data, N=2^16, "
                                   "chain 60+8x40 bits + 60-bit P, scale 2^40, 128x256 packing, g8 sigmoid" % (args.rows, N_FEAT)},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "s/iter", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.ks_point:
        ks_point(args)
        return
    if args.sweep or args.sweep_point:
        sweep(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
