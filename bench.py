#!/usr/bin/env python
"""Benchmark: LUCJ forward + VJP layers/s at norb = 16, nelec = (8, 8).

Workload (one step = one pass of the whole path): the 10-layer LUCJ circuit
of the N=16 (8,8) workload (Haar-random orbital rotations, diagonal-Coulomb
couplings ~ N(0, 0.5) at t = 0.3, random normalised initial state,
1.66e8 amplitudes), forward pass then VJP by uncomputation, complex64 state
and FP32 arithmetic.  value = 10 layers / step time.  The same workload runs
once in complex128 for the c64-vs-c128 figure.

Prints one JSON line on rank 0.  `--impl reference` times the oracle (plain
CPU NumPy) on a bounded sample of the same workload instead.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NORB, NELEC, NLAYERS = 16, (8, 8), 10
WORKLOAD = "lucj_fwd_vjp_norb16_nelec8_8_10layers"
METRIC = "LUCJ fwd+VJP layers/s at norb=16 (8,8)"


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    import hashlib
    src = os.path.join(ROOT, "paper_2605_03123_gb300", "csrc", "fs_sweep_kern.cuh")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = [x.strip() for x in line.strip().strip("|").split("|")]
        if len(parts) >= 4 and parts[0] == kernel and parts[3] == h:
            try:
                return float(parts[1])
            except ValueError:
                return None
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- workload
def workload(args=None):
    from paper_2605_03123_gb300 import inputs
    if args is not None and args.norb:
        return inputs.lucj_layers(args.norb, (args.nalpha, args.nbeta), args.layers, 0.5, 0.3,
                                  2000 + 99)
    return inputs.plain_at_scale()


def algorithmic_bytes(kernel, S, n_layers):
    """Bytes the method itself must move per launch of each kernel kind:
    a sweep reads and writes its state(s) once; the reverse alpha sweep also
    writes W (real, half a state) for the layers that have a gate to undo."""
    if kernel.startswith("sweep_vjp_alpha"):
        return 4 * S + 0.5 * S * n_layers / (n_layers + 1)
    if kernel.startswith("sweep_vjp"):
        return 4 * S
    if kernel.startswith("sweep"):
        return 2 * S
    if kernel.startswith("phase"):
        return 2 * S
    return None


FLOPS_PER_ELEMENT_GIVENS = 10


def algorithmic_flops(kernel, norb, nelec, amplitudes):
    """FP32 (or FP64) flops the method needs per launch of a sweep: 10 real
    flops per element-Givens (x' = c x + s y: 2 for c x, 6 for the complex
    product s y, 2 for the sum), N(N-1)/2 rotations each touching the
    fraction 2 C(N-2, n-1) / C(N, n) of the strings; the reverse sweep
    rotates two states and adds the transition reduction, n(N-n) + n
    complex multiply-adds (8 flops) per amplitude and spin."""
    spin = 0 if "alpha" in kernel else 1
    n = nelec[spin]
    N = norb
    if not kernel.startswith("sweep") or n < 1 or N < 2:
        return None
    eg = N * (N - 1) / 2 * 2 * math.comb(N - 2, n - 1) / math.comb(N, n)
    per = FLOPS_PER_ELEMENT_GIVENS * eg
    if "vjp" in kernel:
        per = 2 * per + 8 * (n * (N - n) + n)
    return per * amplitudes


def max_over_ranks(ms, dist=None, device="cpu"):
    """The job's time: the largest of the ranks' times (ms).  Each rank runs
    its own replica; the job ends when the slowest rank ends."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / (ms / 1e3)


def run_gpu(args):
    import torch
    from paper_2605_03123_gb300 import fsgpu

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fsgpu.load_library()
    ctx = fsgpu.context(local)
    global NORB, NELEC, NLAYERS, WORKLOAD
    if args.norb:
        NORB, NELEC, NLAYERS = args.norb, (args.nalpha, args.nbeta), args.layers
        WORKLOAD = "lucj_fwd_vjp_norb%d_nelec%d_%d_%dlayers" % (NORB, NELEC[0], NELEC[1], NLAYERS)
    da, db = math.comb(NORB, NELEC[0]), math.comb(NORB, NELEC[1])
    # pinned host buffers of the end-to-end leg, allocated before the
    # multi-GB host workload arrays exist (pinned pages placed later copied
    # at a fraction of the link rate on the GB300 host)
    if args.e2e_steps > 0:
        hv = torch.empty((da, db), dtype=torch.complex64, pin_memory=True)
        hc = torch.empty((da, db), dtype=torch.complex64, pin_memory=True)
        hout = torch.empty((da, db), dtype=torch.complex64, pin_memory=True)
    w = workload(args)
    K, Jaa, Jab = w["K"], w["J_aa"], w["J_ab"]
    S = 8 * da * db
    vec0 = torch.from_numpy(w["vec"].astype(np.complex64)).cuda()
    cot0 = torch.from_numpy(w["cot"].astype(np.complex64)).cuda()
    vec = vec0.clone()
    cot = torch.empty_like(cot0)

    def step():
        cot.copy_(cot0)
        fsgpu.lucj_forward_(vec, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        return fsgpu.lucj_vjp_(vec, cot, K, Jaa, Jab, NORB, NELEC, ctx=ctx)

    # the FP32 FMA pipe's measured rate (library probe kernel), before the
    # workload so that it runs on a cool GPU either way
    fma_probe = None
    try:
        fma_probe = fsgpu.measure_fp32_fma(local)[0]
    except fsgpu.FsError:
        pass
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ctx.profile_start()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile_stop()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_per_step = ms / args.steps
    value = job_throughput(world, NLAYERS * args.steps, ms)
    launches = sum(v[2] for v in prof.values())

    # parity at full size, properties: recovered input and dL/dpsi_in identities
    rec_err = float((vec - vec0).abs().max().item())

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hv.copy_(torch.from_numpy(w["vec"].astype(np.complex64)))
        hc.copy_(torch.from_numpy(w["cot"].astype(np.complex64)))
        main = torch.cuda.current_stream()
        copy_s = torch.cuda.Stream()
        # two device buffer pairs: the inputs of step k+1 are copied on the
        # copy stream while step k computes, and the result of step k is
        # read back while step k+1 computes (every step's copies stay inside
        # the timed region)
        dv = [torch.empty_like(vec0) for _ in range(2)]
        dc = [torch.empty_like(cot0) for _ in range(2)]
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        used = [False, False]

        def load(b):
            with torch.cuda.stream(copy_s):
                if used[b]:
                    copy_s.wait_event(done[b])
                dv[b].copy_(hv, non_blocking=True)
                dc[b].copy_(hc, non_blocking=True)
                ready[b].record(copy_s)

        def run(b):
            main.wait_event(ready[b])
            fsgpu.lucj_forward_(dv[b], K, Jaa, Jab, NORB, NELEC, ctx=ctx)
            g = fsgpu.lucj_vjp_(dv[b], dc[b], K, Jaa, Jab, NORB, NELEC, ctx=ctx)
            done[b].record(main)
            used[b] = True
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(done[b])
                hout.copy_(dc[b], non_blocking=True)
            return g

        def pipelined(nsteps, evs=None):
            copy_s.wait_stream(main)
            load(0)
            for k in range(nsteps):
                if k + 1 < nsteps:
                    load((k + 1) % 2)
                run(k % 2)
                if evs:
                    evs[k + 1].record(main)
            main.wait_stream(copy_s)

        pipelined(2)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
        ctx.profile_start()
        evs[0].record(main)
        pipelined(args.e2e_steps, evs)
        end = torch.cuda.Event(enable_timing=True)
        end.record(main)
        torch.cuda.synchronize()
        eprof = ctx.profile_stop()
        each = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.e2e_steps)]
        ems = max_over_ranks(evs[0].elapsed_time(end) / args.e2e_steps, dist, "cuda")

        # one more step without overlap, instrumented phase by phase
        # (outside the timed steps): where the time of an unpipelined step goes
        phases = ("h2d", "forward", "vjp", "d2h")
        pe = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        pe[0].record(main)
        dv[0].copy_(hv, non_blocking=True)
        dc[0].copy_(hc, non_blocking=True)
        pe[1].record(main)
        fsgpu.lucj_forward_(dv[0], K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        pe[2].record(main)
        fsgpu.lucj_vjp_(dv[0], dc[0], K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        pe[3].record(main)
        hout.copy_(dc[0], non_blocking=True)
        pe[4].record(main)
        torch.cuda.synchronize()
        breakdown = {ph: pe[i].elapsed_time(pe[i + 1]) for i, ph in enumerate(phases)}
        grad_bytes = K.size * 16 + Jaa.size * 8 + Jab.size * 8
        e2e = {"value": job_throughput(world, NLAYERS, ems), "unit": "layers/s",
               "h2d_bytes_per_step": 2 * S, "d2h_bytes_per_step": S + grad_bytes,
               "ms_per_step": ems, "ms_each_step": each,
               "pipelined": "inputs of step k+1 copied and result of step k-1 read back "
                            "on a copy stream while step k computes; first copy and "
                            "last read-back exposed",
               "phase_ms_one_unpipelined_step": breakdown,
               "kernel_ms_per_step": sum(v[1] for v in eprof.values()) / args.e2e_steps,
               "device_timed_kernel_ms_per_step": sum(v[1] for v in prof.values()) / args.steps}

    # complex128, same workload, plain path on the same GPU
    c128 = None
    if args.c128_steps > 0:
        v2 = torch.from_numpy(w["vec"]).cuda()
        c2 = torch.from_numpy(w["cot"]).cuda()
        cm = c2.clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fsgpu.lucj_forward_(v2, K, Jaa, Jab, NORB, NELEC, ctx=ctx)  # warm-up
        out128 = v2.clone()
        g128 = fsgpu.lucj_vjp_(v2, cm, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.c128_steps):
            cm.copy_(c2)
            fsgpu.lucj_forward_(v2, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
            fsgpu.lucj_vjp_(v2, cm, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        b.record()
        torch.cuda.synchronize()
        cms = a.elapsed_time(b) / args.c128_steps
        # c64 against c128 on the same inputs: forward output and gradients
        v64 = vec0.clone()
        fsgpu.lucj_forward_(v64, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        fwd_err = float((v64.to(torch.complex128) - out128).abs().max().item())
        c64 = cot0.clone()
        g64 = fsgpu.lucj_vjp_(v64, c64, K, Jaa, Jab, NORB, NELEC, ctx=ctx)
        rel = max(float(np.linalg.norm(x - y) / np.linalg.norm(y)) for x, y in zip(g64, g128))
        c128 = {"layers_per_s": NLAYERS / (cms / 1e3), "ms_per_step": cms,
                "c64_speedup": (NLAYERS / (cms / 1e3)) and value / world / (NLAYERS / (cms / 1e3)),
                "c64_vs_c128_fwd_max_abs": fwd_err, "c64_vs_c128_grad_rel": rel}
        del v2, c2, cm, out128, v64, c64

    # roofline of the dominant kernel
    peak, peak_kind = peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (recs, tot_ms, kl) = top
    per_launch_ms = tot_ms / recs
    ab = algorithmic_bytes(name, S, NLAYERS)
    roof = None
    if ab is not None:
        ach = ab / (per_launch_ms / 1e3) / 1e9
        hbm = {"achieved": ach, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
               "frac": ach / peak, "algorithmic_bytes_per_launch": ab}
        tr = recorded_traffic(name)
        fl = algorithmic_flops(name, NORB, NELEC, da * db)
        csum = clk.summary()
        if fl is not None and csum:
            # The fused sweeps move each amplitude once per launch and are
            # bound by FP32 arithmetic: the roofline is the FP32 FMA peak from
            # the unit counts (SMs of this device x 128 FP32 lanes x 2 flops
            # per clock) at the SM clock sampled during the timed region; the
            # library's FMA-throughput probe and the HBM view are kept beside
            # it.
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            fpeak = sms * 128 * 2 * csum["sm_mhz"] * 1e6 / 1e12
            fach = fl / (per_launch_ms / 1e3) / 1e12
            roof = {"bound": "alu", "kernel": name, "achieved": fach, "peak": fpeak,
                    "peak_source": "unit counts x sampled SM clock (FP32 FMA), %d SMs" % sms,
                    "peak_fp32_fma_probe": fma_probe,
                    "frac_of_probe": fach / fma_probe if fma_probe else None,
                    "unit": "TFLOP/s", "frac": fach / fpeak, "traffic": tr,
                    "flops_per_element_givens": FLOPS_PER_ELEMENT_GIVENS,
                    "algorithmic_flops_per_launch": fl, "ms_per_launch": per_launch_ms,
                    "share_of_step": tot_ms / ms, "hbm": hbm}
        else:
            roof = {"bound": "hbm", "kernel": name, "traffic": tr,
                    "ms_per_launch": per_launch_ms, "share_of_step": tot_ms / ms, **hbm}

    out = {
        "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Haar rotations, N(0,0.5) couplings, random state)",
        "config": {"workload": WORKLOAD, "norb": NORB, "nelec": list(NELEC),
                   "layers": NLAYERS, "state": "complex64", "amplitudes": da * db,
                   "l2": "inputs larger than L2 (%.2f GB state, 129 MB L2)" % (S / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "recovered_input_max_abs_err": rec_err, "c128": c128},
        "roofline": roof, "e2e": e2e, "gpu_launches": launches,
        "kernels": {k: {"records": v[0], "ms": v[1], "launches": v[2]} for k, v in prof.items()},
        "clocks": clk.summary(),
    }
    if not args.norb:
        del vec, cot, vec0, cot0
        torch.cuda.empty_cache()
        if args.batch_steps > 0:
            out["batch"] = run_batch(args, ctx)
        if args.largest:
            out["largest"] = run_largest(args, ctx)
        if args.extras:
            out["dc_phase"] = run_dc_phase(args, ctx)
            out["small_rotation"] = run_small_rotation(args, ctx)
            out["trotter"] = run_trotter(args, ctx)
            out["operator_action"] = run_operator_action(args, ctx)
            out["sampling"] = run_sampling(args, ctx)
    if c128:
        out["c128_layers_per_s"] = c128["layers_per_s"]
        out["c64_speedup_vs_c128"] = c128["c64_speedup"]
    if out.get("batch"):
        b = out["batch"]
        out["batch_circuits_per_s"] = b["circuits_per_s"]
        out["batch_c64_speedup_vs_plain_c128"] = b["c64_batched_speedup_vs_plain_c128"]
        out["batch_speedup_vs_plain_c64"] = b["circuits_per_s"] / b["plain_c64_circuits_per_s_equiv"]
    if out.get("largest"):
        out["largest_fwd_vjp_ms"] = out["largest"]["fwd_vjp_ms"]
        out["largest_fwd_ms_c128"] = out["largest"]["fwd_ms_c128"]
    if rank == 0 and not args.no_cpu_baseline and not args.norb:
        out["cpu_baseline"] = cpu_baseline(w)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def _timed(fn, reset=None, steps=1):
    """CUDA-event time of `fn` per call (ms), `reset` run untimed before each."""
    import torch
    tot = 0.0
    for _ in range(steps):
        if reset:
            reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def run_batch(args, ctx):
    """512 LUCJ circuits (norb in {8,10,12,14}, half filling, 2 repetitions,
    from Hartree-Fock): forward + VJP of all of them as one batched call
    (complex64, one CUDA graph), against the plain complex128 path run
    circuit by circuit on a strided sample of the same circuits."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    cir = inputs.batch_circuits(512)
    amp = [math.comb(c["norb"], c["nelec"][0]) * math.comb(c["norb"], c["nelec"][1]) for c in cir]
    shape = [(math.comb(c["norb"], c["nelec"][0]), math.comb(c["norb"], c["nelec"][1]))
             for c in cir]
    cots0 = [inputs.device_state(c["norb"], c["nelec"], c["cot_seed"], torch.complex64)
             for c in cir]
    vecs = [torch.zeros_like(x) for x in cots0]
    cots = [x.clone() for x in cots0]
    cfg = [dict(c, from_hf=True) for c in cir]

    def reset():
        for x, y in zip(cots, cots0):
            x.copy_(y)

    fsgpu.lucj_batch_(vecs, cots, cfg, ctx=ctx)  # warm-up: plans, tables
    ctx.profile_start()
    ms = _timed(lambda: fsgpu.lucj_batch_(vecs, cots, cfg, ctx=ctx), reset, args.batch_steps)
    prof = ctx.profile_stop()
    reset()
    grads64 = fsgpu.lucj_batch_(vecs, cots, cfg, ctx=ctx)
    del cots
    fwd64 = vecs
    fsgpu.lucj_batch_(fwd64, None, cfg, do_vjp=False, ctx=ctx)
    # plain paths, circuit by circuit, on every k-th circuit
    sample = list(range(0, len(cir), args.batch_stride))
    famp = sum(amp[i] for i in sample) / sum(amp)

    def plain(dtype, keep=None):
        vs = [torch.zeros(shape[i], dtype=dtype, device="cuda") for i in sample]
        c0 = [cots0[i].to(dtype) for i in sample]
        cs = [x.clone() for x in c0]
        res = []

        def run():
            res.clear()
            for v, c, x, i in zip(vs, cs, c0, sample):
                C = cir[i]
                c.copy_(x)
                fsgpu.lucj_forward_(v, C["K"], C["J_aa"], C["J_ab"], C["norb"], C["nelec"],
                                    from_hf=True, ctx=ctx)
                if keep is not None:
                    keep.append(v.clone())
                res.append(fsgpu.lucj_vjp_(v, c, C["K"], C["J_aa"], C["J_ab"], C["norb"],
                                           C["nelec"], from_hf=True, ctx=ctx))
        return run, res

    run128, _ = plain(torch.complex128)
    run128()  # warm-up
    ms128 = _timed(run128)
    del run128
    out128 = []
    run128k, g128 = plain(torch.complex128, out128)
    run128k()
    run64, _ = plain(torch.complex64)
    run64()
    ms64p = _timed(run64)
    fwd_err = max(float((fwd64[i].to(torch.complex128) - o).abs().max().item())
                  for i, o in zip(sample, out128))
    grad_rel = max(float(np.linalg.norm(a - b) / np.linalg.norm(b))
                   for i, g in zip(sample, g128) for a, b in zip(grads64[i], g))
    n = len(cir)
    rate = n / (ms / 1e3)
    # plain-path rates scaled to the whole batch by the sample's share of
    # the amplitudes
    rate128 = n * famp / (ms128 / 1e3)
    return {"workload": "lucj_batch_512_circuits_norb8-14_half_filling_2reps",
            "circuits": n, "amplitudes_total": sum(amp), "state": "complex64",
            "circuits_per_s": rate, "ms_per_step": ms, "steps": args.batch_steps,
            "graph_launches_per_step": 1,
            "kernels": {k: {"records": v[0], "ms": v[1], "launches": v[2]}
                        for k, v in prof.items()},
            "plain_sample": "every %d-th circuit (%d circuits, %.3f of the amplitudes)"
                            % (args.batch_stride, len(sample), famp),
            "plain_c128_circuits_per_s_equiv": rate128,
            "plain_c64_circuits_per_s_equiv": n * famp / (ms64p / 1e3),
            "c64_batched_speedup_vs_plain_c128": rate / rate128,
            "autotuned_slab_widths": ctx.tuning_report(),
            "c64_vs_c128_fwd_max_abs": fwd_err, "c64_vs_c128_grad_rel": grad_rel}


def run_largest(args, ctx):
    """N=18 (9,9), one LUCJ repetition from Hartree-Fock: complex64 forward +
    VJP (2.36e9 amplitudes, 18.9 GB per state), complex128 forward beside."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    w = inputs.largest_state()
    N, ne = w["norb"], w["nelec"]
    K, Ja, Jb = w["K"], w["J_aa"], w["J_ab"]
    v = inputs.device_state(N, ne, 1, torch.complex64)
    v.zero_()
    cot = inputs.device_state(N, ne, w["cot_seed"], torch.complex64)
    cot0 = cot.clone()
    fsgpu.lucj_forward_(v, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)  # warm-up
    norm_err = abs(float(torch.linalg.vector_norm(v).item()) - 1.0)
    fsgpu.lucj_vjp_(v, cot, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)

    def step():
        fsgpu.lucj_forward_(v, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)
        fsgpu.lucj_vjp_(v, cot, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)

    ms = _timed(step, lambda: cot.copy_(cot0), args.largest)
    rec = float(v[0, 0].real.item()) - 1.0
    rec_err = max(abs(rec), float(v.abs().flatten()[1:].max().item()))
    # <A^dag g, psi_in> = <g, A psi_in>: the VJP of a linear map at HF is
    # the HF amplitude of A^dag g
    fsgpu.lucj_forward_(v, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)
    lhs = sum(complex(torch.vdot(cot0[i:i + 4096].flatten(), v[i:i + 4096].flatten()).item())
              for i in range(0, v.shape[0], 4096))
    c2 = cot0.clone()
    fsgpu.lucj_vjp_(v, c2, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)
    rhs = complex(c2[0, 0].item()).conjugate()
    out64 = v
    fsgpu.lucj_forward_(out64, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)
    del cot, cot0, c2
    torch.cuda.empty_cache()
    v2 = torch.zeros(out64.shape, dtype=torch.complex128, device="cuda")
    fsgpu.lucj_forward_(v2, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx)
    ms128 = _timed(lambda: fsgpu.lucj_forward_(v2, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx))
    ms64f = _timed(lambda: fsgpu.lucj_forward_(out64, K, Ja, Jb, N, ne, from_hf=True, ctx=ctx))
    err = float((out64.to(torch.complex128) - v2).abs().max().item())
    del v2, out64, v
    torch.cuda.empty_cache()
    return {"workload": "lucj_norb18_nelec9_9_1rep_from_hf", "amplitudes": math.comb(18, 9) ** 2,
            "state": "complex64", "fwd_vjp_ms": ms, "layers_per_s": 1e3 / ms,
            "fwd_ms_c64": ms64f, "fwd_ms_c128": ms128, "c64_fwd_speedup": ms128 / ms64f,
            "forward_norm_err": norm_err, "recovered_input_max_abs_err": rec_err,
            "vjp_inner_product_identity_abs_err": abs(lhs - rhs),
            "c64_vs_c128_fwd_max_abs": err}


def run_dc_phase(args, ctx):
    """Standalone diagonal-Coulomb evolution at N=16 (8,8): one streaming
    pass over the state (algorithmic bytes 2S) after the per-string tables.
    complex64 takes the TMA / tcgen05 pass (cross term on the tensor cores),
    complex128 the CUDA-core subset-sum tables."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    peak, kind = peaks()
    g = inputs.rng(2100)
    Ja, Jb = inputs.random_symmetric(16, 0.5, g), inputs.random_symmetric(16, 0.5, g)
    out = {"workload": "diag_coulomb_norb16_nelec8_8_t0.3", "peak_gbs": peak,
           "peak_source": kind}
    for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        v = inputs.device_state(16, (8, 8), 7, dt)
        S = v.numel() * v.element_size()
        f = lambda: fsgpu.apply_diag_coulomb_evolution_(v, Ja, Jb, 0.3, 16, (8, 8), ctx=ctx)
        for _ in range(3):
            f()
        ctx.profile_start()
        ms = _timed(lambda: [f() for _ in range(5)]) / 5
        prof = ctx.profile_stop()
        gbs = 2 * S / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": 2 * S, "achieved_gbs": gbs,
                     "frac": gbs / peak,
                     "kernels_ms": {k: v_[1] / max(1, v_[0]) for k, v_ in prof.items()}}
        # the streaming pass alone (complex64: the TMA / tcgen05 kernel)
        if "phase_tc_f32" in prof:
            kms = prof["phase_tc_f32"][1] / max(1, prof["phase_tc_f32"][0])
            out[name]["stream_kernel_ms"] = kms
            out[name]["stream_kernel_frac"] = 2 * S / (kms / 1e3) / 1e9 / peak
        del v
    torch.cuda.empty_cache()
    return out


def run_trotter(args, ctx):
    """Trotter simulation of a double-factorized Hamiltonian at N=16 (8,8):
    three order-0 steps of a Hamiltonian with a one-body term and three
    two-body terms (the paper's Trotter benchmark shape), from a random
    state; complex64 and complex128."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    g = inputs.rng(2300)
    A = g.normal(0, 0.5, (16, 16)) + 1j * g.normal(0, 0.5, (16, 16))
    h = (A + A.conj().T) / 2
    Js = np.array([inputs.random_symmetric(16, 0.5, g) for _ in range(3)])
    Us = np.array([inputs.haar_unitary(16, g) for _ in range(3)])
    v0 = inputs.device_state(16, (8, 8), 9, torch.complex128)
    out = {"workload": "trotter_double_factorized_norb16_nelec8_8_3terms_3steps_order0",
           "unit": "ms per evolution (3 Trotter steps)"}
    for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        x = v0.to(dt)
        f = lambda: fsgpu.simulate_trotter_double_factorized_(x, h, Js, Us, 1.0, 16, (8, 8),
                                                              n_steps=3, order=0, ctx=ctx)
        f()
        ctx.profile_start()
        ms = _timed(f)
        prof = ctx.profile_stop()
        out[name] = {"ms": ms, "trotter_steps_per_s": 3 / (ms / 1e3),
                     "kernels": {k: {"records": v[0], "ms": round(v[1], 3)}
                                 for k, v in prof.items()}}
        del x
    out["c64_speedup"] = out["c128"]["ms"] / out["c64"]["ms"]
    del v0
    torch.cuda.empty_cache()
    return out


def run_operator_action(args, ctx):
    """H psi for a molecular Hamiltonian with random real symmetric tensors
    (8-fold symmetric h_pqrs) at N=12 (6,6) and N=16 (4,4): milliseconds per
    application and the GEMM rate (2 * N^2 * 3N^2 * 2 * dim flops)."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    res = {"unit": "ms per application"}
    for N, ne in ((12, (6, 6)), (16, (4, 4))):
        g = inputs.rng(2400 + N)
        A = g.normal(0, 1, (N, N))
        B = g.normal(0, 0.5, (N, N, N, N))
        h1 = (A + A.T) / 2
        h2 = (B + B.transpose(1, 0, 3, 2) + B.transpose(2, 3, 0, 1) + B.transpose(3, 2, 1, 0)) / 4
        v0 = inputs.device_state(N, ne, 10, torch.complex128)
        dim = v0.numel()
        row = {"amplitudes": dim}
        for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
            v = v0.to(dt)
            o = torch.empty_like(v)
            f = lambda: fsgpu.apply_molecular_hamiltonian(v, h1, h2, N, ne, out=o, ctx=ctx)
            f()
            ms = _timed(f, steps=2)
            flops = 2 * N * N * 3 * N * N * 2 * dim
            row[name] = {"ms": ms, "gemm_tflops": flops / (ms / 1e3) / 1e12}
            del v, o
        res["norb%d_nelec%d_%d" % (N, ne[0], ne[1])] = row
        del v0
        torch.cuda.empty_cache()
    return res


def run_host_copies(args, ctx):
    """Diagnostics of the end-to-end leg (not part of the default run): the
    time of one 1.33 GB pinned host-to-device copy of the N=16 state when
    copies run back to back, right after an N=16 forward pass, after idle
    pauses of 0.01-2 s, and concurrently with a forward pass (which is timed
    too); and one device-to-host copy."""
    import torch
    from paper_2605_03123_gb300 import fsgpu
    w = workload(None)
    K, Jaa, Jab = w["K"], w["J_aa"], w["J_ab"]
    hv = torch.empty(w["vec"].shape, dtype=torch.complex64, pin_memory=True)
    hv.copy_(torch.from_numpy(w["vec"].astype(np.complex64)))
    dv = torch.empty(hv.shape, dtype=torch.complex64, device="cuda")
    dw = dv.clone()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()

    def copy_ms(dst, src, stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
        return e0, e1

    def fwd():
        fsgpu.lucj_forward_(dw, K, Jaa, Jab, NORB, NELEC, ctx=ctx)

    def el(e):
        return e[0].elapsed_time(e[1])

    fwd()
    torch.cuda.synchronize()
    out = {"bytes": hv.numel() * 8, "unit": "ms"}
    r = []
    for _ in range(4):
        e = copy_ms(dv, hv, main)
        torch.cuda.synchronize()
        r.append(el(e))
    out["h2d_back_to_back"] = r
    e = copy_ms(hv, dv, main)
    torch.cuda.synchronize()
    out["d2h_after_copies"] = el(e)
    for pause in (0.0, 0.01, 0.1, 0.5, 2.0):
        fwd()
        torch.cuda.synchronize()
        time.sleep(pause)
        e = copy_ms(dv, hv, main)
        torch.cuda.synchronize()
        out["h2d_after_forward_and_%gs_idle" % pause] = el(e)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(main)
    fwd()
    f1.record(main)
    torch.cuda.synchronize()
    out["forward_alone"] = f0.elapsed_time(f1)
    time.sleep(0.5)
    f0.record(main)
    fwd()
    f1.record(main)
    e = copy_ms(dv, hv, side)
    torch.cuda.synchronize()
    out["h2d_during_forward_after_0.5s_idle"] = el(e)
    out["forward_during_that_copy"] = f0.elapsed_time(f1)
    return out


SECTIONS = {}


def run_sampling_only(args):
    """Profiling only: the sampling section alone, at the sector given by
    --norb/--nalpha/--nbeta (default the N=16 (8,8) workload)."""
    from paper_2605_03123_gb300 import fsgpu
    global NORB, NELEC
    if args.norb:
        NORB, NELEC = args.norb, (args.nalpha, args.nbeta)
    fsgpu.load_library()
    print(json.dumps(run_sampling(args, fsgpu.context(0), slater=not args.norb)))


def run_sampling(args, ctx, slater=True):
    """Sampling configurations.  From the N=16 (8,8) state (1.66e8
    amplitudes), 1e6 shots per call in complex64 and complex128: time per
    call, samples/s, and the HBM fraction of the prefix pass, whose
    algorithmic traffic is one read of the state.  From spinless Slater
    determinants at 1/4 filling (the paper's Slater-sampling benchmark
    shape), 1000 shots: time per call and the FP64 rate of the chain rule
    (2 N n^2 FP64 FMA per shot)."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    hbm, src = peaks()
    shots = args.shots
    res = {"state": {"workload": "norb%d_nelec%d_%d" % (NORB, NELEC[0], NELEC[1]),
                     "shots": shots, "peak": src,
                     "unit": "ms per call"}}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    u = torch.rand(shots, dtype=torch.float64, device="cuda", generator=gen)
    for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        v = inputs.device_state(NORB, NELEC, 12, dt)
        S = v.numel() * v.element_size()
        f = lambda: fsgpu.sample_state(v, NORB, NELEC, uniforms=u, ctx=ctx)
        for _ in range(3):
            f()
        ctx.profile_start()
        ms = _timed(f, steps=3)
        prof = ctx.profile_stop()
        cdf_ms = prof["sample_cdf"][1] / max(1, prof["sample_cdf"][0])
        search_ms = prof["sample_search"][1] / max(1, prof["sample_search"][0])
        gbs = S / (cdf_ms / 1e3) / 1e9
        res["state"][name] = {"ms": ms, "samples_per_s": shots / (ms / 1e3),
                              "cdf_ms": cdf_ms, "search_ms": search_ms,
                              "cdf_gbs": gbs, "cdf_hbm_frac": gbs / hbm}
        del v
    del u
    torch.cuda.empty_cache()
    if not slater:
        return res
    sl = {"unit": "ms per 1000 shots", "fp64_peak_tflops_nominal": 1.25}
    for N in (64, 256, 1024):
        n = N // 4
        g = inputs.rng(2500 + N)
        U = inputs.haar_unitary(N, g)
        occ = list(range(n))
        f = lambda: fsgpu.sample_slater(N, occ, U, shots=1000, seed=3, ctx=ctx)
        f()
        ctx.profile_start()
        ms = _timed(f, steps=2)
        prof = ctx.profile_stop()
        kms = prof["slater_sample"][1] / max(1, prof["slater_sample"][0])
        fma = 2.0 * N * n * n * 1000
        sl["norb%d_nocc%d" % (N, n)] = {"ms": ms, "kernel_ms": kms,
                                        "fp64_tflops": 2 * fma / (kms / 1e3) / 1e12}
    res["slater"] = sl
    return res


def run_small_rotation(args, ctx):
    """Orbital rotation of small sectors by Givens sweeps and by dense
    minor-matrix GEMMs, and the method the autotuner keeps."""
    import torch
    from paper_2605_03123_gb300 import fsgpu, inputs
    res = {}
    for N in (8, 10, 12):
        ne = (N // 2, N // 2)
        g = inputs.rng(2200 + N)
        U = inputs.haar_unitary(N, g)
        row = {}
        for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
            v = inputs.device_state(N, ne, 8, dt)
            t = {}
            for path, pn in ((fsgpu.FS_ROT_GIVENS, "givens"), (fsgpu.FS_ROT_MINORS, "minors")):
                ctx.set_rotation_path(path)
                f = lambda: fsgpu.apply_orbital_rotation_(v, U, N, ne, ctx=ctx)
                for _ in range(3):
                    f()
                t[pn] = _timed(lambda: [f() for _ in range(10)]) / 10
            ctx.set_rotation_path(fsgpu.FS_ROT_AUTO)
            fsgpu.apply_orbital_rotation_(v, U, N, ne, ctx=ctx)
            t["auto"] = _timed(lambda: [fsgpu.apply_orbital_rotation_(v, U, N, ne, ctx=ctx)
                                        for _ in range(10)]) / 10
            row[name] = {k: round(x, 4) for k, x in t.items()}
        res["norb%d" % N] = row
    return {"unit": "ms per rotation", **res}


# ------------------------------------------------------------------ oracle
# The oracle's LUCJ reverse mode per layer applies 4 orbital rotations
# (U^dag and U forward, both again on the cotangent), each N(N-1)/2 = 120
# Givens rotations per spin from its own decomposition; 2 transition one-body
# reductions (one per rotation gate); 2 diagonal-Coulomb phase evaluations.
GIVENS_PER_LAYER_PER_SPIN = 4 * 120
T_PER_LAYER = 2
DC_PER_LAYER = 2


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_slice_times(norb, nelec, width, seed):
    """One worker's share of the oracle sample: on its own slice of `width`
    columns (alpha operations) and `width` rows (beta operations) of the
    N-orbital state (random values; the cost does not depend on them), time
    one alpha and one beta Givens rotation and the transition one-body
    reduction of both spins, as the oracle runs them.  Runs in a spawned
    process (one host core)."""
    from oracle import gates, lucj
    from paper_2605_03123_gb300 import inputs
    d = math.comb(norb, nelec[0])
    g = inputs.rng(seed)
    mk = lambda shape: g.standard_normal(shape) + 1j * g.standard_normal(shape)
    vc, cc = mk((d, width)), mk((d, width))
    vr, cr = mk((width, d)), mk((width, d))
    gates.givens_pairs(norb, nelec[0], 0, 5)    # the oracle caches its pair lists
    gates.givens_pairs(norb, nelec[1], 3, 11)
    t = time.perf_counter()
    gates.apply_givens(vc, 0.6, 0.8j, 0, 5, 0, norb, nelec)
    t_ga = time.perf_counter() - t
    t = time.perf_counter()
    gates.apply_givens(vr, 0.6, 0.8j, 3, 11, 1, norb, nelec)
    t_gb = time.perf_counter() - t
    t = time.perf_counter()
    lucj.transition_one_body(cc, vc, norb, nelec, spins=(0,))
    lucj.transition_one_body(cr, vr, norb, nelec, spins=(1,))
    t_T = time.perf_counter() - t
    return t_ga, t_gb, t_T


SLICE_WIDTHS = (32, 64)


def oracle_slice_work(norb, nelec, seed):
    """One host process's share of the oracle sample: oracle_slice_times at
    the two SLICE_WIDTHS (the transition reduction has a fixed cost for its
    pair lists plus a part linear in the width; the Givens rotations are
    linear in the width)."""
    return [oracle_slice_times(norb, nelec, wd, seed + wd) for wd in SLICE_WIDTHS]


def _project(times, width):
    """Phase times of a (width)-wide slice from the two measured widths."""
    (a, b) = SLICE_WIDTHS
    ta, tb = times
    slope = (tb[2] - ta[2]) / (b - a)
    return (tb[0] * width / b, tb[1] * width / b, max(tb[2] + slope * (width - b), tb[2]))


def oracle_layer_sample(w, workers):
    """One bounded sample of the oracle on `workers` host processes plus the
    parent.  Every worker, concurrently, times one alpha and one beta Givens
    rotation and the transition reduction of both spins on its own 32- and
    64-vector column and row slices of the N=16 state; the parent meanwhile
    applies one diagonal-Coulomb evolution to the whole state.  With the
    state split evenly over the workers (d / workers vectors each), a
    worker's phase times follow from its two widths (linear in the width,
    plus the reduction's fixed cost, which every worker pays); each phase
    takes the slowest worker's time.  A layer is GIVENS_PER_LAYER_PER_SPIN
    of each Givens phase, T_PER_LAYER reductions and DC_PER_LAYER
    evolutions.  Returns (layer seconds, measured sample seconds, phases)."""
    import concurrent.futures
    import multiprocessing
    import oracle
    norb, nelec = NORB, NELEC
    d = math.comb(norb, nelec[0])
    share = d / workers
    t0 = time.perf_counter()
    if workers == 1:
        res = [oracle_slice_work(norb, nelec, 77)]
        t = time.perf_counter()
        oracle.apply_diag_coulomb_evolution(w["vec"], w["J_aa"][0], w["J_ab"][0], None, 1.0,
                                            norb, nelec)
        t_dc = time.perf_counter() - t
    else:
        ctx = multiprocessing.get_context("spawn")
        with concurrent.futures.ProcessPoolExecutor(workers, mp_context=ctx) as ex:
            futs = [ex.submit(oracle_slice_work, norb, nelec, 77 + 1000 * k)
                    for k in range(workers)]
            t = time.perf_counter()
            oracle.apply_diag_coulomb_evolution(w["vec"], w["J_aa"][0], w["J_ab"][0], None,
                                                1.0, norb, nelec)
            t_dc = time.perf_counter() - t
            res = [f.result() for f in futs]
    wall = time.perf_counter() - t0
    proj = [_project(r, share) for r in res]
    t_ga = max(p[0] for p in proj)
    t_gb = max(p[1] for p in proj)
    t_T = max(p[2] for p in proj)
    layer = (GIVENS_PER_LAYER_PER_SPIN * (t_ga + t_gb) + T_PER_LAYER * t_T
             + DC_PER_LAYER * t_dc)
    return layer, wall, {"givens_alpha_s": t_ga, "givens_beta_s": t_gb,
                         "transition_s": t_T, "diag_coulomb_s": t_dc}


def default_workers():
    """Host processes for the all-core sample: one per core beside the
    parent."""
    return max(1, (os.cpu_count() or 2) - 1)


SAMPLE_TEXT = ("%d host process(es), concurrently, each time one alpha and one beta Givens "
               "rotation and the transition reduction of both spins on 32- and 64-vector "
               "slices of the N=16 (8,8) complex128 state, projected to a 1/%d share of the "
               "state, while the parent times one diagonal-Coulomb evolution of the whole "
               "state; a layer is 480 Givens rotations per spin, 2 reductions and 2 "
               "evolutions (the oracle's gate count)")


def cpu_baseline(w):
    """The oracle, as it stands, on bounded samples of the workload: on all
    host cores (spawned workers) and on one core, each scaled to layers/s
    by the oracle's own gate count per layer."""
    one, wall1, parts1 = oracle_layer_sample(w, 1)
    nw = default_workers()
    allc, wall, parts = oracle_layer_sample(w, nw)
    return {"value": 1.0 / allc, "unit": "layers/s", "cores": nw + 1, "kind": "oracle",
            "cpu_model": cpu_model(), "logical_cpus": os.cpu_count(), "projected": True,
            "sample": SAMPLE_TEXT % (nw, nw),
            "sample_seconds": wall, "phases_s": parts,
            "single_core": {"value": 1.0 / one, "unit": "layers/s", "cores": 1,
                            "sample": SAMPLE_TEXT % (1, 1),
                            "sample_seconds": wall1, "phases_s": parts1}}


def run_reference(args):
    """The oracle arm: each step is one all-core bounded sample; `value` is
    the layer rate it implies, `ms_per_step` the time the sample itself
    took."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    w = workload()
    nw = default_workers()
    rates, walls, parts = [], [], None
    for i in range(args.warmup + args.steps):
        layer, wall, parts_i = oracle_layer_sample(w, nw)
        if i >= args.warmup:
            rates.append(1.0 / layer)
            walls.append(wall)
            parts = parts_i
    v = statistics.median(rates)
    ms_step = 1e3 * sum(walls) / len(walls)
    sample = "per step: " + SAMPLE_TEXT % (nw, nw)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "layers/s",
           "n_gpus": env_int("WORLD_SIZE", 1), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_step, "projected": True,
           "projected_ms_per_layer": 1e3 / v,
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "norb": NORB, "nelec": list(NELEC),
                      "layers": NLAYERS},
           "cpu_baseline": {"value": v, "unit": "layers/s", "cores": nw + 1, "kind": "oracle",
                            "cpu_model": cpu_model(), "sample": sample,
                            "phases_s": parts},
           "e2e": {"value": v, "unit": "layers/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fsgpu", choices=["fsgpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--c128-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=2,
                    help="timed calls of the 512-circuit batch (0 skips it)")
    ap.add_argument("--batch-stride", type=int, default=4,
                    help="plain-path sample of the batch: every k-th circuit")
    ap.add_argument("--largest", type=int, default=1,
                    help="timed steps of the N=18 (9,9) state (0 skips it)")
    ap.add_argument("--extras", type=int, default=1,
                    help="standalone diagonal-Coulomb pass and small-sector rotation "
                         "methods (0 skips them)")
    ap.add_argument("--norb", type=int, default=0,
                    help="profiling only: another sector size instead of the N=16 workload")
    ap.add_argument("--nalpha", type=int, default=0)
    ap.add_argument("--nbeta", type=int, default=0)
    ap.add_argument("--layers", type=int, default=NLAYERS)
    ap.add_argument("--shots", type=int, default=1000000,
                    help="shots per call of the state-sampling section")
    ap.add_argument("--sampling-only", action="store_true",
                    help="profiling only: the sampling section alone")
    ap.add_argument("--section", choices=sorted(SECTIONS),
                    help="profiling only: one of the extra sections alone")
    args = ap.parse_args()
    if args.sampling_only:
        run_sampling_only(args)
    elif args.section:
        from paper_2605_03123_gb300 import fsgpu
        fsgpu.load_library()
        print(json.dumps({args.section: SECTIONS[args.section](args, fsgpu.context(0))}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


SECTIONS.update({"dc_phase": lambda a, c: run_dc_phase(a, c),
                 "small_rotation": lambda a, c: run_small_rotation(a, c),
                 "trotter": lambda a, c: run_trotter(a, c),
                 "operator_action": lambda a, c: run_operator_action(a, c),
                 "sampling": lambda a, c: run_sampling(a, c),
                 "host_copies": lambda a, c: run_host_copies(a, c),
                 "largest": lambda a, c: run_largest(a, c)})

if __name__ == "__main__":
    main()
