"""Benchmark: macro-elements condensed per second (one Newton step of the
entropy-variable macro-element HDG method, arXiv 2507.22195).

Workload (one "step"): inviscid Taylor-Green vortex, Mach 0.1, periodic
[0, 2 pi]^3, 8^3 macro-elements of 3^3 micro-elements, p = 3 (N_v = 5000
unknowns per element), KEPES flux, stage term with dt = 1: residual, dense
Jacobian S^K, batched LU, FP64-refined S^-1 R_V and b-hat, for all 512
elements (mehdg_condense).  Inputs are resident in HBM; the dense S^K of the
512 elements (53.7 GB FP32) is far larger than L2, so nothing is cached
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32|bf16|fp64]
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores

Under torchrun every rank condenses its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "macro-elements condensed/sec at p=3 (mixed vs FP64 GPU), err vs FP64 oracle"
UNIT = "macro-elements/s"
WORKLOAD = "inviscid Taylor-Green vortex, 8^3 macro-elements x 3^3 micro-elements, p=3, KEPES, one Newton-step condensation"
PREC = {"tf32": 1, "bf16": 2, "fp64": 0, "tf32x3": 3, "bf16x3": 4}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region"""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU)
def _oracle_one(args):
    K, nk = args
    import oracle
    from paper_2507_22195_gb300 import inputs as I
    mesh = I.periodic_mesh(nk, 3, 3)
    st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
    prm = oracle.params(flux=oracle.KEPES, Mach=0.1)
    t = time.time()
    R, B = oracle.element_system(prm, mesh, st, K)
    oracle.condense_K(0, R, B, False)
    return time.time() - t


def oracle_rate(n_elem: int, cores: int):
    """FP64 CPU oracle, as it stands: n_elem elements of the workload, one per
    process (spawned), on `cores` host cores.  Returns (elements/s, seconds)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    t = time.time()
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_one, [(K * 37 % 512, 8) for K in range(n_elem)])
    dt = time.time() - t
    return n_elem / dt, dt


def reference_main(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = min(os.cpu_count() or 1, 16)
    per_step = cores                     # one element per core per step
    for _ in range(a.warmup):
        oracle_rate(per_step, cores)
    times = []
    for _ in range(a.steps):
        _, dt = oracle_rate(per_step, cores)
        times.append(dt)
    tot = sum(times)
    val = per_step * a.steps / tot
    sample = f"{per_step} of the 512 elements per step (element ids 37k mod 512), one per process"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 512, "seq_len": None, "parallelism": "none"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ---------------------------------------------------------------- GPU arm
def once_main(a):
    """Workload setup, `warmup` condenses and one more, nothing timed: the
    command the ncu summaries under profiles/ are taken with."""
    import numpy as np
    import torch
    from paper_2507_22195_gb300 import inputs as I
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh(a.nk, 3, 3)
    st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
    dev = torch.device("cuda:0")
    v, vh, vs = (torch.tensor(x, device=dev) for x in (st.v, st.vhat, st.vstar))
    ctx = M.Context(mesh, flux=M.MEHDG_FLUX_KEPES, prec=PREC[a.prec], Mach=0.1)
    ctx.set_state(v, vh, None, vs)
    for _ in range(a.warmup + 1):
        ctx.condense()
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    print(json.dumps({"once": True, "nK": mesh.nK, "prec": a.prec, "status_ok": bool((stat == 0).all()),
                      "refine_iters": sorted(set(int(x) for x in iters)), "launches": M.mehdg_launch_count()}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=list(PREC))
    ap.add_argument("--nk", type=int, default=8)
    ap.add_argument("--fp64-sample", type=int, default=2, help="nk of the FP64 comparison mesh (nk^3 elements)")
    ap.add_argument("--cpu-sample", type=int, default=-1, help="elements for the CPU oracle baseline (-1: one per core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--once", action="store_true", help="one condense after --warmup ones, no timing (for profilers)")
    a = ap.parse_args()
    if a.impl == "reference":
        return reference_main(a)
    if a.once:
        return once_main(a)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline first (spawned pool, before any CUDA call), rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cores = min(os.cpu_count() or 1, 16)
        n = cores if a.cpu_sample < 0 else a.cpu_sample
        val, dt = oracle_rate(n, cores)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} of the 512 elements (residual, complex-step Jacobian, dense GEPP, b-hat), "
                         f"one per process, {dt:.1f} s wall"}

    import numpy as np
    import torch
    from paper_2507_22195_gb300 import inputs as I
    from paper_2507_22195_gb300 import mehdg as M

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    mesh = I.periodic_mesh(a.nk, 3, 3)
    st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
    v, vh, vs = (torch.tensor(x, device=dev) for x in (st.v, st.vhat, st.vstar))
    ctx = M.Context(mesh, flux=M.MEHDG_FLUX_KEPES, prec=PREC[a.prec], Mach=0.1)
    ctx.set_state(v, vh, None, vs)
    bh = torch.empty((mesh.n_global_faces, 5, mesh.n2), dtype=torch.float64, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(a.warmup):
        ctx.condense(bh)
    stat, iters = ctx.status()

    # timed region: K steps, events on the library's stream (torch current stream)
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    M.mehdg_profile_enable(ctx.ctx, True)
    n0 = M.mehdg_launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(a.steps):
        ctx.condense(bh)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = M.mehdg_launch_count() - n0
    prof = M.mehdg_profile_read(ctx.ctx)
    M.mehdg_profile_enable(ctx.ctx, False)
    clocks = clk.stop()
    stat, iters = ctx.status()
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * mesh.nK * a.steps / (ms / 1e3)

    # end to end through the public API: pinned host inputs -> device,
    # condense, b-hat -> host, every step
    hv, hvh, hvs = (torch.tensor(x).pin_memory() for x in (st.v, st.vhat, st.vstar))
    hb = torch.empty(bh.shape, dtype=torch.float64).pin_memory()
    v2, vh2, vs2 = torch.empty_like(v), torch.empty_like(vh), torch.empty_like(vs)
    ctx.set_state(v2, vh2, None, vs2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        v2.copy_(hv, non_blocking=True); vh2.copy_(hvh, non_blocking=True); vs2.copy_(hvs, non_blocking=True)
        ctx.condense(bh)
        hb.copy_(bh, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = hv.numel() * 8 + hvh.numel() * 8 + hvs.numel() * 8
    d2h = hb.numel() * 8
    ctx.set_state(v, vh, None, vs)

    # roofline of the dominant kernel: the outer trailing update of the LU
    pk = peaks()
    gem = prof["lu_trailing_update"]
    ld = (5 * mesh.Nn + 255) // 256 * 256
    # algorithmic bytes of all trailing updates of one step: C read+write (FP32)
    # and the two operand panels (rest x 256, FP32), per element
    byt = 0
    for c0 in range(0, ld, 256):
        rest = ld - c0 - 256
        if rest > 0:
            byt += (8 * rest * rest + 2 * 4 * rest * 256)
    byt *= mesh.nK * a.steps
    if a.prec == "fp64":
        fl = gem["flops"]
        roof = {"bound": "alu", "achieved": fl / (gem["ms"] / 1e3) / 1e12, "peak": 1.2,
                "unit": "TFLOP/s", "frac": None, "traffic": None,
                "note": "FP64 SIMT trailing update; peak = 152 SMs x 64 FP64 FMA/clk x 2 x ~1.9 GHz boost (fallback estimate)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        ach = byt / (gem["ms"] / 1e3) / 1e9
        hbm = pk.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": "measured" if "hbm_gbs" in pk else "fallback",
                "kernel": "lu_trailing_update (depth 256)", "launches": gem["launches"],
                "ms": gem["ms"], "tflops": gem["flops"] / (gem["ms"] / 1e3) / 1e12}

    # FP64 GPU path and error on a small mesh of the same elements
    fp = None
    if a.prec != "fp64" and a.fp64_sample > 0:
        m2 = I.periodic_mesh(a.fp64_sample, 3, 3)
        s2 = I.make_state(m2, "tgv", 1e-3, 22197, 22198, M0=0.1)
        w, wh, ws = (torch.tensor(x, device=dev) for x in (s2.v, s2.vhat, s2.vstar))
        outs = {}
        for pr in ("fp64", a.prec):
            c2 = M.Context(m2, flux=M.MEHDG_FLUX_KEPES, prec=PREC[pr], Mach=0.1)
            c2.set_state(w, wh, None, ws)
            b2 = c2.condense()
            barrier()
            t1 = time.perf_counter()
            c2.condense(b2)
            barrier()
            outs[pr] = (b2.clone(), time.perf_counter() - t1)
            c2.close()
        err = float(torch.linalg.norm(outs[a.prec][0] - outs["fp64"][0]) / torch.linalg.norm(outs["fp64"][0]))
        fp = {"value": m2.nK / outs["fp64"][1], "unit": UNIT, "sample": f"{m2.nK} elements ({a.fp64_sample}^3 periodic mesh)",
              "mixed_same_sample": m2.nK / outs[a.prec][1],
              "err_bhat_mixed_vs_fp64": err}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"tf32": "tf32 (f32 accumulate) + f64", "bf16": "bf16 (f32 accumulate) + f64",
                      "tf32x3": "split tf32 x3 (f32 accumulate) + f64", "bf16x3": "split bf16 x3 (f32 accumulate) + f64",
                      "fp64": "f64"}[a.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": mesh.nK, "seq_len": None,
                       "parallelism": f"dp{world}" if world > 1 else "none", "nK": mesh.nK, "p": 3, "m": 3,
                       "N_v": 5 * mesh.Nn, "prec": a.prec,
                       "l2": "inputs larger than L2 (dense S^K of all elements: %.1f GB)" % (
                           mesh.nK * ld * ld * (8 if a.prec == "fp64" else 4) / 1e9)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * mesh.nK * a.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "refine_iters": sorted(set(int(x) for x in iters)),
            "status_ok": bool((stat == 0).all()),
            "phases_ms_per_step": {k: round(vv["ms"] / a.steps, 3) for k, vv in prof.items()},
            "fp64_gpu": fp,
        }
        print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
