#!/usr/bin/env python
"""Benchmark of the rBKI-TK hot path on GB300 (one JSON line on rank 0).

Workload (default): the single large rBKI-TK problem - a 512x512x512 FP32 tensor, 20^3
superdiagonal core with power-law mode spectra (sigma_k ~ k^-1/2) x Haar factors + noise
at SNR 10 dB; ranks (20,20,20), p = 10, q = 3; products in BF16 on the tensor path with
FP32 accumulation, orthonormalisation and eigensolve in FP64.

A step is one whole rBKI-TK decomposition (staging + Algorithms 1-2 for every mode + the
core TTM chain).  Metric: X-pass HBM GB/s = algorithmic bytes of the X passes of one step
(sketch, q+1 Krylov steps per Krylov mode, one pass per Gram mode, the first TTM), each
counted as one read of X at the streamed BF16 precision (2 B/element), divided by the
step time.  The oracle arm (--impl reference) reports the same quantity for the FP64 CPU
oracle on a bounded sample (one mode's Algorithm 1 + Rayleigh-Ritz per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ELEM_BYTES = 2  # X counted at the streamed BF16 precision


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["tucker512", "tucker64", "video", "htr", "serve", "waves"],
                    default="tucker512")
    ap.add_argument("--inflight", type=int, default=8,
                    help="decompositions in flight on separate streams (throughput mode); 1 = one at a time")
    ap.add_argument("--requests", type=int, default=4096, help="served stream length (--workload serve)")
    ap.add_argument("--slots", type=int, default=16, help="server slots (--workload serve)")
    ap.add_argument("--wave-threads", type=int, default=4,
                    help="server workers of the batched path (0: every request on a slot)")
    ap.add_argument("--wave-max", type=int, default=32, help="requests per wave of the batched path")
    ap.add_argument("--tune-cache", default=None,
                    help="work-granularity table of the batched path: loaded if the file exists, else "
                         "measured (rbki_wave_autotune) and written there; default: measured, not kept")
    ap.add_argument("--fp64-requests", type=int, default=256,
                    help="prefix of the served stream also run on the FP64 GPU path (--workload serve)")
    ap.add_argument("--prec", choices=["bf16", "fp64"], default="bf16")
    ap.add_argument("--size", type=int, default=0,
                    help="cube edge for tucker512 (0 = 512); smaller cases for profiler captures")
    ap.add_argument("--sequential", action="store_true",
                    help="sequentially truncated reading (each mode sketched on the contracted tensor)")
    ap.add_argument("--no-sequential-compare", action="store_true")
    ap.add_argument("--parts", type=int, default=0,
                    help="divide-and-conquer: split the last mode into this many parts, decompose them as a batch")
    ap.add_argument("--power", action="store_true", help="power-iteration baseline instead of block Krylov")
    ap.add_argument("--refine", action="store_true", help="FP32 Rayleigh-Ritz refinement of the mixed factors")
    ap.add_argument("--q-tol", type=float, default=None,
                    help="adaptive Krylov depth: stop a mode when its fit changes by at most this (q is the bound)")
    ap.add_argument("--omega", type=float, default=0.0,
                    help="column sampling rate of the Krylov construction (0 < omega < 1)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve-compare", action="store_true",
                    help="skip the bounded served-stream measurement of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    return ap.parse_args()


def make_workload(name, mc, size=0):
    import synth
    if name == "tucker512":
        return synth.config_large(mc=mc, size=size or 512)
    if name == "tucker64":
        return synth.config_small_fp64(mc=mc)
    if name == "video":
        return synth.config_video(mc=mc)
    if name == "htr":
        return synth.config_htr(mc=mc)
    raise ValueError(name)


# DRAM bytes (read + write) of one tensor-core Krylov-step launch on the 512^3 workload
# (k_krylov_tc, mode 0), from the single-pass ncu capture summarised in
# profiles/k_krylov_tc_448cube_bf16.md: 268.5 MB read + 2.7 MB written.  Set to None when
# k_krylov_tc changes until a new capture is taken.
KRYLOV_TC_DRAM_BYTES_512 = 268510720 + 2740224


def plan_passes(dims, ranks, p, q):
    """X passes of one step: per Krylov mode 1 sketch + (q+1) Krylov steps; per Gram mode 1;
    plus the first TTM of the core chain."""
    passes, krylov_steps = 1, 0
    for i_n, r_n in zip(dims, ranks):
        s = min(r_n + p, i_n)
        if s * (q + 1) >= i_n:
            passes += 1
        else:
            passes += q + 2
            krylov_steps += q + 1
    return passes, krylov_steps


def sampled_columns(dims, n, omega):
    """Columns of the sampled unfolding Y of mode n (128-column units, ragged ones padded)."""
    a = 1
    for v in dims[:n]:
        a *= v
    c = 1
    for v in dims[n + 1:]:
        c *= v
    nu = a * -(-c // 128) if c > 1 else -(-a // 128)
    return 128 * int(min(max(math.ceil(omega * nu), 1), nu))


def plan_sampled(dims, ranks, p, q, omega, elem):
    """Bytes of one decomposition with partial column sampling: per Krylov mode the gather
    (read the kept columns, write Y) and 1 sketch + (q+1) Krylov passes over Y; per Gram
    mode one pass of X; the first core product reads X.  Returns (bytes, Krylov bytes,
    Krylov steps)."""
    numel = 1
    for v in dims:
        numel *= v
    total, kbytes, ksteps = numel * elem, 0, 0
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        s = min(r_n + p, i_n)
        if s * (q + 1) >= i_n:
            total += numel * elem
            continue
        y = sampled_columns(dims, n, omega) * i_n * elem
        total += 2 * y + (q + 2) * y
        kbytes += (q + 1) * y
        ksteps += q + 1
    return total, kbytes, ksteps


def plan_sequential(dims, ranks, p, q, elem0, elem_rest):
    """Sequential reading: per step n the passes over Y_n (dims R_1..R_{n-1}, I_n..I_N) of
    Algorithm 1 (1 sketch + q+1 Krylov steps, or 1 Gram pass) plus the product
    Y_n x_n U^(n)T.  Returns (bytes per decomposition, Krylov-step bytes, Krylov steps)."""
    cur = list(dims)
    total = kbytes = ksteps = 0
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        e = 1
        for v in cur:
            e *= v
        eb = elem0 if n == 0 else elem_rest
        s = min(r_n + p, i_n)
        if s * (q + 1) >= i_n:
            m = 1
        else:
            m = q + 2
            kbytes += (q + 1) * e * eb
            ksteps += q + 1
        total += (m + 1) * e * eb
        cur[n] = r_n
    return total, kbytes, ksteps


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join("/tmp", f"rbki_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd[1:1] = ["-i", self.uuid]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 11:
                continue
            rows.append(f)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        util = [float(r[5]) for r in rows if r[5].replace(".", "").isdigit()]
        load = [s for s, u in zip(sm, util) if u > 0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[7:11]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": float(rows[0][3]) if rows[0][3].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, world):
    """Max of a per-rank float over all ranks (NCCL on the GPU, gloo on the CPU)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(step_bytes, ms_max, world):
    """Whole-job GB/s of `world` independent replicas: every rank streams `step_bytes` per
    step, and the job's step time is the slowest rank's."""
    return world * step_bytes / (ms_max * 1e-3) / 1e9


def oracle_cpu_baseline(wl, max_seconds=30.0):
    """The FP64 NumPy oracle as it stands, on this host's cores: full rBKI-TK of the same
    tensor (bounded: stops after the modes that fit in ~max_seconds)."""
    import numpy as np
    from oracle import philox, rbki
    from oracle.tensor import unfold
    x = np.asarray(wl.x, dtype=np.float64)
    t0 = time.perf_counter()
    done_bytes = 0
    modes = 0
    for n in range(x.ndim):
        s = min(wl.ranks[n] + wl.p, x.shape[n])
        xn = unfold(x, n)
        if s * (wl.q + 1) >= x.shape[n]:
            np.linalg.eigh(xn @ xn.T)
            done_bytes += x.size * ELEM_BYTES
        else:
            om = philox.omega_mode(wl.seed, n, x.shape, s)
            qb = np.concatenate(rbki.rbki(xn, om, wl.q), axis=1)
            rbki.rayleigh_ritz(xn, qb, wl.ranks[n])
            done_bytes += (wl.q + 2) * x.size * ELEM_BYTES
        modes += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": done_bytes / dt / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle, Algorithm 1 + Rayleigh-Ritz for {modes} of {x.ndim} modes of the "
                      f"same {'x'.join(map(str, x.shape))} tensor ({dt:.1f} s), X passes counted at "
                      f"{ELEM_BYTES} B/element"}


def run_ours(args):
    import numpy as np
    import torch
    import paper_2211_14828_gb300 as rb
    from paper_2211_14828_gb300 import _binding as B

    world, rank, local = dist_setup(args)
    wl = make_workload(args.workload, rank, args.size)
    dims = list(wl.x.shape)
    numel = int(np.prod(dims))
    prec = args.prec
    flags = rb.FLAG_SEQUENTIAL if args.sequential else 0
    if args.power:
        flags |= rb.FLAG_POWER
    if args.refine:
        flags |= rb.FLAG_REFINE_FP32
    if args.q_tol is not None:
        flags |= rb.FLAG_ADAPTIVE_Q
    qtol = args.q_tol or 0.0
    if args.omega > 0 and args.sequential:
        raise SystemExit("--omega and --sequential: byte accounting of the combination is not implemented")
    if args.omega > 0:
        passes = None
        step_bytes, krylov_bytes, krylov_steps = plan_sampled(dims, wl.ranks, wl.p, wl.q, args.omega,
                                                              ELEM_BYTES if prec != "fp64" else wl.x.itemsize)
    elif args.sequential:
        passes = None
        e0 = ELEM_BYTES if prec != "fp64" else wl.x.itemsize
        step_bytes, krylov_bytes, krylov_steps = plan_sequential(dims, wl.ranks, wl.p, wl.q, e0,
                                                                 ELEM_BYTES if prec != "fp64" else 8)
    else:
        passes, krylov_steps = plan_passes(dims, wl.ranks, wl.p, wl.q)
        step_bytes = passes * numel * ELEM_BYTES
        krylov_bytes = krylov_steps * numel * (ELEM_BYTES if prec != "fp64" else wl.x.itemsize)
    x = torch.from_numpy(wl.x).cuda()
    stream = torch.cuda.current_stream()
    # K decompositions in flight: stream j runs steps j, j+K, ...; each has its own workspace
    # and outputs (the steps are independent decompositions of the input)
    K = max(1, args.inflight)
    streams = [torch.cuda.Stream() for _ in range(K)]
    outs = []
    for j in range(K):
        with torch.cuda.stream(streams[j]):
            outs.append(rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=flags,
                                       omega=args.omega, q_tol=qtol,
                                       stream=streams[j]))
    torch.cuda.synchronize()
    out = outs[0]
    if args.q_tol is not None:
        # the adaptive depths decide the passes: 1 sketch + (q_used + 1) Krylov steps per mode
        qu = out["q_used"].cpu().numpy().tolist()
        step_bytes, krylov_bytes, krylov_steps = numel * ELEM_BYTES, 0, 0
        for n, (i_n, r_n) in enumerate(zip(dims, wl.ranks)):
            s_n = min(r_n + wl.p, i_n)
            if s_n * (wl.q + 1) >= i_n:
                step_bytes += numel * ELEM_BYTES
            else:
                step_bytes += (qu[n] + 2) * numel * ELEM_BYTES
                krylov_bytes += (qu[n] + 1) * numel * (ELEM_BYTES if prec != "fp64" else wl.x.itemsize)
                krylov_steps += qu[n] + 1
        passes = step_bytes // (numel * ELEM_BYTES)

    def run_steps(nsteps):
        ev = torch.cuda.Event()
        ev.record(stream)
        for j in range(K):
            streams[j].wait_event(ev)
        for t in range(nsteps):
            j = t % K
            o = outs[j]
            rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=flags, omega=args.omega, q_tol=qtol,
                           workspace=o["workspace"], out=o, stream=streams[j])
        for j in range(K):
            e = torch.cuda.Event()
            e.record(streams[j])
            stream.wait_event(e)

    run_steps(max(0, args.warmup - 1) * K + K)
    torch.cuda.synchronize()
    # one decomposition alone (latency)
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=flags, omega=args.omega, q_tol=qtol,
                   workspace=out["workspace"], out=out, stream=stream)
    e_b.record(stream)
    torch.cuda.synchronize()
    single_ms = e_a.elapsed_time(e_b)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    rb.rbki_profile_reset()
    rb.rbki_profile_enable(True)
    launches0 = rb.rbki_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    th0 = time.perf_counter()
    run_steps(args.steps)
    host_ms = (time.perf_counter() - th0) * 1e3 / args.steps      # host time to enqueue a step
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    rb.rbki_profile_enable(False)
    launches = rb.rbki_kernel_launches() - launches0
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = allreduce_max(ms_local, world)
    value = replica_throughput(step_bytes, ms, world)

    kcount, kms = rb.rbki_profile_read(rb.PROF_KRYLOV)
    scount, sms = rb.rbki_profile_read(rb.PROF_SKETCH)
    peak, peak_kind = measured_peaks()
    roof = None
    if kcount:
        # algorithmic bytes of all timed Krylov-step launches / their summed duration
        avg = kms / kcount
        ach = krylov_bytes * args.steps / (kms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4),
                "traffic": (KRYLOV_TC_DRAM_BYTES_512 if prec == "bf16" and KRYLOV_TC_DRAM_BYTES_512
                            and numel == 512 ** 3 and not args.sequential
                            and args.omega <= 0 and args.q_tol is None else None),
                "traffic_unit": "bytes per launch (ncu, one 512^3 launch)",
                "kernel": "krylov_step",
                "avg_launch_ms": round(avg, 4), "launches": kcount, "peak_kind": peak_kind}
    breakdown = {}
    for name, cls in (("krylov", rb.PROF_KRYLOV), ("sketch", rb.PROF_SKETCH), ("gram", rb.PROF_GRAM),
                      ("ttm1", rb.PROF_TTM), ("stage", rb.PROF_STAGE),
                      ("sample", rb.PROF_SAMPLE)):
        c, t = rb.rbki_profile_read(cls)
        if c:
            breakdown[name] = {"ms_per_step": round(t / args.steps, 4), "launches_per_step": c / args.steps}
    rb.rbki_profile_reset()

    norms = out["norms"].cpu().numpy()
    rel_err = float(np.sqrt(max(norms[0] - norms[1], 0.0) / norms[0]))

    # the same Krylov-step kernel timed by itself (nothing else on the GPU): one mode's step
    # P = X_(0) (X_(0)^T Q) through the public rbki_krylov_product on the BF16 tensor
    roof_alone = None
    if roof is not None and prec == "bf16" and not args.sequential and args.omega <= 0:
        xb = x.to(torch.bfloat16)
        s_w = min(wl.ranks[0] + wl.p, dims[0])
        # an orthonormal Q (host QR: keeps torch's device linear-algebra library out of the run)
        qh = np.linalg.qr(np.random.default_rng(11).standard_normal((dims[0], s_w)))[0]
        qm = torch.from_numpy(np.ascontiguousarray(qh)).cuda()
        for _ in range(3):
            rb.rbki_krylov_product(xb, 0, qm, prec="bf16")
        torch.cuda.synchronize()
        rb.rbki_profile_reset()
        rb.rbki_profile_enable(True)
        for _ in range(10):
            rb.rbki_krylov_product(xb, 0, qm, prec="bf16")
        torch.cuda.synchronize()
        rb.rbki_profile_enable(False)
        ac, ams = rb.rbki_profile_read(rb.PROF_KRYLOV)
        rb.rbki_profile_reset()
        if ac:
            a_ms = ams / ac
            a_gbs = numel * ELEM_BYTES / (a_ms * 1e-3) / 1e9
            roof_alone = {"bound": "hbm", "achieved": round(a_gbs, 1), "peak": peak, "unit": "GB/s",
                          "frac": round(a_gbs / peak, 4), "kernel": "krylov_step", "avg_launch_ms": round(a_ms, 4),
                          "launches": ac, "peak_kind": peak_kind,
                          "note": "the same kernel timed alone after the timed region (mode 0 of the same tensor)"}
        del xb

    e2e = None
    if not args.no_e2e:
        # through the public call with host buffers (RBKI_FLAG_HOST_IO): every step copies X
        # from pinned host memory and reads the results back; K calls in flight on their own
        # streams and workspaces (RBKI_FLAG_ASYNC), so one step's copies overlap another's
        # computation, as in the device-resident throughput mode
        xh = torch.from_numpy(wl.x).pin_memory()
        hflags = flags | rb.FLAG_HOST_IO | rb.FLAG_ASYNC
        ohs = [B.alloc_outputs(dims, wl.ranks, None, host=True) for _ in range(K)]
        wss = [torch.empty(rb.rbki_tucker_workspace(xh, wl.ranks, wl.p, wl.q, wl.seed, prec, hflags, args.omega,
                                                    qtol), dtype=torch.uint8, device="cuda") for _ in range(K)]

        def e2e_steps(n):
            for t in range(n):
                j = t % K
                rb.rbki_tucker(xh, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=hflags, omega=args.omega,
                               q_tol=qtol, workspace=wss[j], out=ohs[j], stream=streams[j])
            torch.cuda.synchronize()

        e2e_steps(2 * K)
        ke = max(3 * K, min(args.steps, 12))
        barrier(world)
        t0 = time.perf_counter()
        e2e_steps(ke)
        te = (time.perf_counter() - t0) / ke
        te = allreduce_max(te, world)
        oh = ohs[0]
        d2h = sum(int(np.prod(v.shape)) * v.element_size() for k, v in oh.items()
                  if k in ("core", "norms", "info", "q_used"))
        d2h += sum(f.numel() * 8 for f in oh["factors"]) + sum(e.numel() * 8 for e in oh["eigvals"])
        e2e = {"value": round(world * step_bytes / te / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(te * 1e3, 3), "inflight": K}
        del wss

    fp64_cmp = None
    if not args.no_fp64_compare and prec != "fp64":
        o64 = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=flags, omega=args.omega)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=flags, omega=args.omega, q_tol=qtol,
                       workspace=o64["workspace"], out=o64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        n64 = o64["norms"].cpu().numpy()
        rel64 = float(np.sqrt(max(n64[0] - n64[1], 0.0) / n64[0]))
        fp64_cmp = {"ms_per_step": round(t64 * 1e3, 2), "rel_err": rel64,
                    "mixed_rel_err": rel_err, "mixed_vs_fp64": (rel_err - rel64) / rel64}
        if not (flags & rb.FLAG_REFINE_FP32) and args.q_tol is None:
            # the FP32 Rayleigh-Ritz refinement of the mixed factors: the Ritz values against the
            # FP64 path's (largest deviation relative to lambda_1, over every Krylov-path mode)
            # with and without it, its reconstruction error and one refined decomposition alone
            orf = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=flags | rb.FLAG_REFINE_FP32,
                                 omega=args.omega)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=flags | rb.FLAG_REFINE_FP32,
                           omega=args.omega, workspace=orf["workspace"], out=orf)
            torch.cuda.synchronize()
            trf = time.perf_counter() - t0
            nrf = orf["norms"].cpu().numpy()
            dev_plain, dev_ref = 0.0, 0.0
            for n in range(len(dims)):
                l64 = o64["eigvals"][n].cpu().numpy()
                dev_plain = max(dev_plain, float(np.max(np.abs(out["eigvals"][n].cpu().numpy() - l64)) / l64[0]))
                dev_ref = max(dev_ref, float(np.max(np.abs(orf["eigvals"][n].cpu().numpy() - l64)) / l64[0]))
            fp64_cmp["refine_fp32"] = {"single_decomposition_ms": round(trf * 1e3, 4),
                                       "rel_err": float(np.sqrt(max(nrf[0] - nrf[1], 0.0) / nrf[0])),
                                       "ritz_dev_vs_fp64_unrefined": dev_plain,
                                       "ritz_dev_vs_fp64_refined": dev_ref}
            del orf
        del o64

    seq_cmp = None
    if (not args.sequential and not args.no_sequential_compare and args.omega <= 0 and not args.power
            and args.q_tol is None):
        # the sequentially truncated reading on the same input: one decomposition alone
        osq = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=rb.FLAG_SEQUENTIAL)
        times = []
        for _ in range(4):
            e_a.record(stream)
            rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=rb.FLAG_SEQUENTIAL,
                           workspace=osq["workspace"], out=osq, stream=stream)
            e_b.record(stream)
            torch.cuda.synchronize()
            times.append(e_a.elapsed_time(e_b))
        nsq = osq["norms"].cpu().numpy()
        e_sq = 2 if prec != "fp64" else wl.x.itemsize
        sq_bytes = plan_sequential(dims, wl.ranks, wl.p, wl.q, e_sq, 2 if prec != "fp64" else 8)[0]
        seq_cmp = {"single_decomposition_ms": round(min(times[1:]), 4),
                   "rel_err": float(np.sqrt(max(nsq[0] - nsq[1], 0.0) / nsq[0])),
                   "bytes_per_decomposition": sq_bytes}
        del osq

    serve_cmp = None
    if rank == 0 and world == 1 and not args.no_serve_compare and args.workload == "tucker512" and not args.size:
        # the served-stream half of the metric, bounded: 1024 requests of the stream
        res, _ = serve_measure(1024, args.slots, 128, (0.8,), 1, args.wave_threads, args.wave_max, args.tune_cache)
        serve_cmp = {k: res[k] for k in ("requests", "slots", "wave_threads", "wave_max", "tuning", "solves_per_s",
                                          "graph_replay",
                                          "launches_per_request",
                                          "x_pass_gbs", "latency", "fp64_compare", "rel_err_mixed")}
        serve_cmp["unit"] = "solves/s"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_cpu_baseline(wl)

    if rank == 0:
        line = {
            "metric": "rBKI-TK Krylov-pass HBM GB/s (X-pass bytes of one full decomposition / step time)",
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec == "bf16" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {'x'.join(map(str, dims))} {wl.x.dtype}, ranks {wl.ranks}, "
                                   f"p={wl.p}, q={wl.q}, {prec} products"
                                   + (", sequential truncation" if args.sequential else "")
                                   + (f", column sampling omega={args.omega}" if args.omega > 0 else "")
                                   + (", power iteration" if args.power else "")
                                   + (f", adaptive q (q_tol={args.q_tol}, depths "
                                      f"{out['q_used'].cpu().numpy().tolist()})" if args.q_tol is not None else ""),
                       "inflight": K, "single_decomposition_ms": round(single_ms, 4),
                       "host_enqueue_ms_per_step": round(host_ms, 4),
                       "passes_per_step": passes, "krylov_steps_per_step": krylov_steps,
                       "bytes_per_step": step_bytes, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "roofline_alone": roof_alone, "breakdown": breakdown, "rel_err": rel_err,
            "fp64_compare": fp64_cmp,
            "sequential_compare": seq_cmp, "serve_compare": serve_cmp,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 NumPy oracle on the host cores, same metric/unit/config; each step = one
    mode's Algorithm 1 + Rayleigh-Ritz over the full tensor (a bounded sample)."""
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import philox, rbki
    from oracle.tensor import unfold
    if args.workload == "serve":
        import synth
        reqs = synth.serve_stream(n_requests=args.requests, seed=5000)
        for r in reqs[:args.warmup]:
            wl = synth.serve_request_tensor(r, dtype=np.float64)
            rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
        t0 = time.perf_counter()
        for r in reqs[args.warmup:args.warmup + args.steps]:
            wl = synth.serve_request_tensor(r, dtype=np.float64)
            rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
        dt = time.perf_counter() - t0
        value = args.steps / dt
        print(json.dumps({
            "metric": "served rBKI-TK solves/s (closed loop; p50/p99 latency under Poisson arrivals)",
            "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "serve: requests of the served stream, one per step, solved one after another"},
            "cpu_baseline": {"value": round(value, 3), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle, {args.steps} requests of the stream"},
            "e2e": {"value": round(value, 3), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    wl = make_workload(args.workload, 0, args.size)
    x = np.asarray(wl.x, dtype=np.float64)
    dims = list(x.shape)
    numel = x.size

    def step(k):
        if args.sequential:
            rbki.rbki_st_tucker(x, wl.ranks, wl.p, wl.q, wl.seed)
            return plan_sequential(dims, wl.ranks, wl.p, wl.q, ELEM_BYTES, ELEM_BYTES)[0]
        n = k % x.ndim
        s = min(wl.ranks[n] + wl.p, x.shape[n])
        xn = unfold(x, n)
        if s * (wl.q + 1) >= x.shape[n]:
            np.linalg.eigh(xn @ xn.T)
            return numel * ELEM_BYTES
        if args.omega > 0:
            rbki.krylov_mode(xn, x, n, s, wl.ranks[n], wl.q, wl.seed, args.omega)
            return (wl.q + 4) * sampled_columns(dims, n, args.omega) * x.shape[n] * ELEM_BYTES
        om = philox.omega_mode(wl.seed, n, x.shape, s)
        qb = np.concatenate(rbki.rbki(xn, om, wl.q), axis=1)
        rbki.rayleigh_ritz(xn, qb, wl.ranks[n])
        return (wl.q + 2) * numel * ELEM_BYTES

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    tot = 0
    for k in range(args.steps):
        tot += step(k)
    dt = time.perf_counter() - t0
    value = tot / dt / 1e9
    line = {
        "metric": "rBKI-TK Krylov-pass HBM GB/s (X-pass bytes of one full decomposition / step time)",
        "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": f"{args.workload}: {'x'.join(map(str, dims))}, ranks {wl.ranks}, p={wl.p}, q={wl.q}"
                               + (", sequential truncation" if args.sequential else "")
                               + (f", column sampling omega={args.omega}" if args.omega > 0 else ""),
                   "sample": ("one full sequentially truncated decomposition per step" if args.sequential
                              else "one mode's Algorithm 1 + Rayleigh-Ritz per step")},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "FP64 NumPy oracle, one mode's Algorithm 1 + Rayleigh-Ritz per step, X passes "
                                   f"counted at {ELEM_BYTES} B/element"},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def serve_passes(dims, ranks, p, q):
    """X passes of one served request (same rule as `plan_passes`)."""
    return plan_passes(dims, ranks, p, q)[0]


def _serve_closed_loop(rb, srv, items, outs, prec):
    """Submit every request at once and wait for all: (seconds, latencies, statuses)."""
    t0 = time.perf_counter()
    tickets = [srv.submit(x, rk, p, q, sd, prec=prec, out=o)[0] for (x, rk, p, q, sd), o in zip(items, outs)]
    pending = set(tickets)
    lat, status = {}, {}
    while pending:
        for t in list(pending):
            ok, st, l = srv.poll(t)
            if ok:
                pending.discard(t)
                lat[t], status[t] = l, st
        if pending:
            time.sleep(2e-4)
    return time.perf_counter() - t0, [lat[t] for t in tickets], [status[t] for t in tickets]


def _serve_poisson(rb, srv, items, outs, prec, rate, seed):
    """Open loop: request i is submitted at its Poisson arrival time; latency = completion
    - arrival (any lateness of the submitter counts against the server)."""
    import numpy as np
    g = np.random.default_rng(seed)
    arrivals = np.cumsum(g.exponential(1.0 / rate, len(items)))
    t0 = time.perf_counter()
    pending, lat, i = {}, [], 0
    while i < len(items) or pending:
        now = time.perf_counter() - t0
        while i < len(items) and arrivals[i] <= now:
            x, rk, p, q, sd = items[i]
            t, _ = srv.submit(x, rk, p, q, sd, prec=prec, out=outs[i])
            pending[t] = (arrivals[i], now)
            i += 1
        for t in list(pending):
            ok, st, l = srv.poll(t)
            if ok:
                arr, sub = pending.pop(t)
                lat.append((sub - arr) + l)
        time.sleep(1e-4)
    return time.perf_counter() - t0, lat


def run_divide(args):
    """Divide-and-conquer step (Sec. 4.1.2): split X along its last mode into K consecutive
    parts and decompose the parts as one batch (part k: seed + k, the frame rank scaled by
    the part's share of frames).  Bytes: the split (read + write X) plus every part's X
    passes (same rule as the one-pass plan)."""
    import numpy as np
    import torch
    import paper_2211_14828_gb300 as rb

    world, rank, local = dist_setup(args)
    wl = make_workload(args.workload, rank, args.size)
    dims = list(wl.x.shape)
    mode, K = len(dims) - 1, args.parts
    prec = args.prec
    x = torch.from_numpy(wl.x).cuda()
    stream = torch.cuda.current_stream()
    sizes = [(k + 1) * dims[mode] // K - k * dims[mode] // K for k in range(K)]
    ranks = []
    for f in sizes:
        r = list(wl.ranks)
        r[mode] = max(1, min(f, round(wl.ranks[mode] * f / dims[mode])))
        ranks.append(r)
    numel = int(np.prod(dims))
    step_bytes = 2 * numel * wl.x.itemsize
    for k, f in enumerate(sizes):
        pd = list(dims)
        pd[mode] = f
        passes, _ = plan_passes(pd, ranks[k], wl.p, wl.q)
        step_bytes += passes * int(np.prod(pd)) * ELEM_BYTES
    parts = rb.rbki_split_mode(x, mode, K)
    outs = rb.rbki_tucker_batch(parts, ranks, wl.p, wl.q, [wl.seed + k for k in range(K)], prec=prec)
    ws = outs[0]["workspace"]

    import ctypes
    from paper_2211_14828_gb300 import _binding as B
    part_ptrs = (ctypes.c_void_p * K)(*[t.data_ptr() for t in parts])
    xt = B.make_tensor(x)

    def step():
        # split into the same part buffers, then the batch into the same outputs
        B.check(B.lib().rbki_split_mode(ctypes.byref(xt), mode, K, part_ptrs, B.stream_ptr(stream)),
                "rbki_split_mode")
        rb.rbki_tucker_batch(parts, ranks, wl.p, wl.q, [wl.seed + k for k in range(K)], prec=prec, workspace=ws,
                             outs=outs, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(None)
    rb.rbki_profile_reset()
    rb.rbki_profile_enable(True)
    launches0 = rb.rbki_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    rb.rbki_profile_enable(False)
    launches = rb.rbki_kernel_launches() - launches0
    ms = allreduce_max(ev0.elapsed_time(ev1) / args.steps, world)
    kcount, kms = rb.rbki_profile_read(rb.PROF_KRYLOV)
    peak, peak_kind = measured_peaks()
    roof = None
    if kcount:
        kb = 0
        for k, f in enumerate(sizes):
            pd = list(dims)
            pd[mode] = f
            kb += plan_passes(pd, ranks[k], wl.p, wl.q)[1] * int(np.prod(pd)) * ELEM_BYTES
        ach = kb * args.steps / (kms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": None, "kernel": "krylov_step", "avg_launch_ms": round(kms / kcount, 4),
                "launches": kcount, "peak_kind": peak_kind}
    rb.rbki_profile_reset()
    err2 = sum(max(float(o["norms"][0]) - float(o["norms"][1]), 0.0) for o in outs)
    x2 = sum(float(o["norms"][0]) for o in outs)
    if rank == 0:
        print(json.dumps({
            "metric": "rBKI-TK Krylov-pass HBM GB/s (X-pass bytes of one full decomposition / step time)",
            "value": round(world * step_bytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec == "bf16" else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {'x'.join(map(str, dims))} {wl.x.dtype}, divide-and-conquer "
                                   f"into {K} parts along mode {mode}, part ranks {ranks[0]}, p={wl.p}, q={wl.q}, "
                                   f"{prec} products, parts decomposed as one batch",
                       "bytes_per_step": step_bytes, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "rel_err": float(np.sqrt(err2 / x2)), "e2e": None, "gpu_launches": int(launches),
            "clocks": clk, "cpu_baseline": None,
        }))


def wave_tuning(rb, cache):
    """Autotuned work granularity of the batched path (from `cache` when it exists)."""
    if cache and os.path.exists(cache):
        rb.rbki_wave_tune_load(cache)
        return {"source": "file", "table": rb.rbki_wave_tune_table()}
    t0 = time.perf_counter()
    rb.rbki_wave_autotune()
    secs = time.perf_counter() - t0
    if cache:
        rb.rbki_wave_tune_save(cache)
    return {"source": "measured", "seconds": round(secs, 3), "table": rb.rbki_wave_tune_table()}


def serve_measure(n_requests, slots, fp64_prefix, rhos, warmup=1, wave_threads=4, wave_max=32, tune_cache=None):
    """The served stream (Sec. 4 workloads as a request stream): n_requests rBKI-TK requests
    (3rd order, dims in [32, 256], ranks in [4, 32], q in {1, 2, 3}, p = 5, SNR in [5, 25] dB,
    BF16 products) through the server.  Closed-loop solves/s (every request submitted at
    once); p50/p99 latency under Poisson arrivals at rho x that rate; the FP64 GPU path on a
    prefix of the same stream, with the largest relative deviation of the mixed path's
    reconstruction error from the FP64 path's (matched error: <= 1%)."""
    import numpy as np
    import torch
    import synth
    import paper_2211_14828_gb300 as rb
    from paper_2211_14828_gb300 import _binding as B
    reqs = synth.serve_stream(n_requests=n_requests, seed=5000)
    items, outs, x32 = [], [], []
    numel_passes = 0
    for i, r in enumerate(reqs):
        x, rk, p, q, sd = synth.serve_request_device(r)
        items.append((x, rk, p, q, sd))
        outs.append(B.alloc_outputs(x.shape, rk, x.device))
        numel_passes += serve_passes(x.shape, rk, p, q) * x.numel()
        if i < fp64_prefix:
            x32.append(x.float())
    torch.cuda.synchronize()
    budget = 8 << 30
    res = {"tuning": wave_tuning(rb, tune_cache) if wave_threads else None}
    with rb.RbkiServer(0, mem_budget=budget, max_slots=slots, wave_threads=wave_threads, wave_max=wave_max) as srv:
        nw = min(len(items), max(warmup, 1) * max(slots, wave_max if wave_threads else 0))
        _serve_closed_loop(rb, srv, items[:nw], outs[:nw], "bf16")
        clocks = ClockSampler()
        clocks.start()
        torch.cuda.synchronize()
        launches0 = rb.rbki_kernel_launches()
        secs, lat, status = _serve_closed_loop(rb, srv, items, outs, "bf16")
        torch.cuda.synchronize()
        launches = rb.rbki_kernel_launches() - launches0
        res["clocks"] = clocks.stop()
        assert all(s == 0 for s in status), "served request failed"
        sat = len(items) / secs
        errs_mixed = []
        for o in outs:
            n = o["norms"].cpu().numpy()
            errs_mixed.append(float(np.sqrt(max(n[0] - n[1], 0.0) / n[0])))
        latency = {"closed_loop": {"p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
                                   "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3)}}
        for rho in rhos:
            t, l = _serve_poisson(rb, srv, items, outs, "bf16", rho * sat, seed=int(rho * 1000))
            latency[f"poisson_rho_{rho}"] = {"offered_per_s": round(rho * sat, 1),
                                             "achieved_per_s": round(len(items) / t, 1),
                                             "p50_ms": round(1e3 * float(np.percentile(l, 50)), 3),
                                             "p99_ms": round(1e3 * float(np.percentile(l, 99)), 3)}
        # the graph pattern: a fixed batch (the stream's first wave_max requests, in their own
        # buffers) captured once and replayed per batch
        replay = None
        if wave_threads:
            nb = min(len(items), wave_max)
            plan = rb.BatchedPlan([it[0] for it in items[:nb]], [it[1] for it in items[:nb]], items[0][2],
                                  [it[3] for it in items[:nb]], [it[4] for it in items[:nb]])
            for _ in range(3):
                plan.launch()
            torch.cuda.synchronize()
            reps = 20
            l0 = rb.rbki_kernel_launches()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.launch()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            replay = {"requests_per_batch": nb, "batches": reps, "ms_per_batch": round(ms, 3),
                      "solves_per_s": round(nb / (ms * 1e-3), 1),
                      "kernels_per_batch": int((rb.rbki_kernel_launches() - l0) / reps), "graph_launches_per_batch": 1}
            plan.close()
        res["graph_replay"] = replay
        f64 = None
        if x32:
            its = [(x32[i],) + items[i][1:] for i in range(len(x32))]
            o64 = [B.alloc_outputs(x.shape, it[1], x.device) for x, it in zip(x32, its)]
            secs64, lat64, st64 = _serve_closed_loop(rb, srv, its, o64, "fp64")
            assert all(s == 0 for s in st64), "served FP64 request failed"
            e64 = []
            for o in o64:
                n = o["norms"].cpu().numpy()
                e64.append(float(np.sqrt(max(n[0] - n[1], 0.0) / n[0])))
            dev = [abs(a - b) / b for a, b in zip(errs_mixed[:len(e64)], e64)]
            secs_m, lat_m, _ = _serve_closed_loop(rb, srv, items[:len(its)], outs[:len(its)], "bf16")
            f64 = {"requests": len(its), "fp64_solves_per_s": round(len(its) / secs64, 1),
                   "fp64_p50_ms": round(1e3 * float(np.percentile(lat64, 50)), 3),
                   "fp64_p99_ms": round(1e3 * float(np.percentile(lat64, 99)), 3),
                   "mixed_solves_per_s": round(len(its) / secs_m, 1),
                   "mixed_p50_ms": round(1e3 * float(np.percentile(lat_m, 50)), 3),
                   "mixed_p99_ms": round(1e3 * float(np.percentile(lat_m, 99)), 3),
                   "max_rel_err_dev_mixed_vs_fp64": max(dev), "all_within_1pct": bool(max(dev) <= 0.01)}
    res.update({
        "requests": len(items), "slots": slots, "wave_threads": wave_threads, "wave_max": wave_max,
        "budget_bytes": budget,
        "solves_per_s": round(sat, 2), "closed_loop_s": round(secs, 4),
        "x_pass_bytes": int(2 * numel_passes), "x_pass_gbs": round(2 * numel_passes / secs / 1e9, 2),
        "launches_per_request": round(launches / len(items), 1), "gpu_launches": int(launches),
        "latency": latency, "fp64_compare": f64,
        "rel_err_mixed": {"median": float(np.median(errs_mixed)), "max": float(np.max(errs_mixed))},
    })
    return res, reqs


def run_serve(args):
    """Served stream: --requests requests through the server (see serve_measure).  value =
    closed-loop solves/s; p50/p99 latency under Poisson arrivals at 0.5/0.8/0.95 of that rate;
    the FP64 GPU path on a prefix of the same stream for the matched-error check."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        raise SystemExit("--workload serve runs on one GPU")
    torch.cuda.set_device(0)
    res, reqs = serve_measure(args.requests, args.slots, args.fp64_requests, (0.5, 0.8, 0.95), args.warmup,
                              args.wave_threads, args.wave_max, args.tune_cache)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = serve_cpu_baseline(reqs)
    line = {
        "metric": "served rBKI-TK solves/s (closed loop; p50/p99 latency under Poisson arrivals)",
        "value": res["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": round(res["closed_loop_s"] * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"serve: {res['requests']} requests, dims U[32,256]^3, ranks U[4,32], p=5, "
                               f"q in {{1,2,3}}, SNR U[5,25] dB, BF16 products", "slots": args.slots,
                   "wave_threads": args.wave_threads, "wave_max": args.wave_max,
                   "budget_bytes": res["budget_bytes"], "x_pass_bytes": res["x_pass_bytes"],
                   "x_pass_gbs": res["x_pass_gbs"],
                   "l2": "requests are mostly smaller than L2; throughput is latency-bound"},
        "latency": res["latency"], "fp64_compare": res["fp64_compare"], "rel_err_mixed": res["rel_err_mixed"],
        "launches_per_request": res["launches_per_request"], "tuning": res["tuning"],
        "graph_replay": res["graph_replay"],
        "e2e": None, "gpu_launches": res["gpu_launches"], "clocks": res["clocks"], "cpu_baseline": cpu,
    }
    print(json.dumps(line))


def serve_cpu_baseline(reqs, max_seconds=20.0):
    """The FP64 oracle on the host cores over a bounded prefix of the served stream."""
    import numpy as np
    import synth
    from oracle import rbki
    t0 = time.perf_counter()
    n = 0
    for r in reqs:
        wl = synth.serve_request_tensor(r, dtype=np.float64)
        rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
        n += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(n / dt, 3), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle, the first {n} requests of the stream ({dt:.1f} s, NumPy-generated "
                      f"tensors of the same recipe)"}


def run_waves(args):
    """Batched path alone: the served stream's first --requests requests as waves of
    --wave-max through rbki_tucker_batched, one after another on one stream (no server, no
    arrivals).  A step is one pass over all the requests; value = requests / step time."""
    import numpy as np
    import torch
    import synth
    import paper_2211_14828_gb300 as rb
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload waves runs on one GPU")
    torch.cuda.set_device(0)
    reqs = synth.serve_stream(n_requests=args.requests, seed=5000)
    items = [synth.serve_request_device(r) for r in reqs]
    W = max(1, args.wave_max)
    waves = [items[i:i + W] for i in range(0, len(items), W)]
    outs = [None] * len(waves)

    def step():
        for k, wv in enumerate(waves):
            o = rb.rbki_tucker_batched([t[0] for t in wv], [t[1] for t in wv], wv[0][2], [t[3] for t in wv],
                                       [t[4] for t in wv], workspace=outs[k][0]["workspace"] if outs[k] else None,
                                       outs=outs[k])
            outs[k] = o

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    l0 = rb.rbki_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    launches = rb.rbki_kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    errs = []
    for wv, o in zip(waves, outs):
        for out in o:
            n = out["norms"].cpu().numpy()
            errs.append(float(np.sqrt(max(n[0] - n[1], 0.0) / n[0])))
    print(json.dumps({
        "metric": "batched rBKI-TK solves/s (waves through rbki_tucker_batched, one stream)",
        "value": round(len(items) / (ms * 1e-3), 2), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"waves: the first {len(items)} requests of the served stream in waves of {W}",
                   "l2": "requests are mostly smaller than L2; latency-bound small stages"},
        "rel_err_mixed": {"median": float(np.median(errs)), "max": float(np.max(errs))},
        "launches_per_request": round(launches / args.steps / len(items), 2),
        "e2e": None, "gpu_launches": int(launches), "clocks": clocks.stop(), "cpu_baseline": None,
    }))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "waves":
        run_waves(args)
    elif args.parts > 1:
        run_divide(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
