"""Benchmark: macro-elements condensed per second (one Newton step of the
entropy-variable macro-element HDG method, arXiv 2507.22195).

Default workload (one "step"): inviscid Taylor-Green vortex, Mach 0.1,
periodic [0, 2 pi]^3, 8^3 macro-elements of 3^3 micro-elements, p = 3 (N_v =
5000 unknowns per element), KEPES flux, stage term with dt = 1: residual,
dense Jacobian S^K, batched LU, FP64-refined S^-1 R_V and b-hat, for all
512 elements (mehdg_condense).  Inputs are resident in HBM; the dense S^K of
the 512 elements (53.7 GB FP32) is far larger than L2, so nothing is cached
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3|tf32x3|tf32|bf16|fp64]
  python bench.py --workload tgv_viscous [--block B]   # B^3 block of the 16^3 x 4^3 viscous TGV
  python bench.py --workload vortex                    # 2^3 x 2^3 isentropic vortex, p = 2
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores
  python bench.py --once               # one condense, untimed (for profilers)

Under torchrun every rank condenses its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
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
WORKLOADS = {
    "tgv_inviscid": "inviscid Taylor-Green vortex, 8^3 macro-elements x 3^3 micro-elements, p=3, KEPES, "
                    "one Newton-step condensation",
    "tgv_viscous": "viscous Taylor-Green vortex Re=1600, block of the 16^3 x 4^3 mesh, p=3, ES, "
                   "one Newton-step condensation (Q-elimination)",
    "vortex": "isentropic vortex, 2^3 macro-elements x 2^3 micro-elements, p=2, ES, one Newton-step condensation",
}
PREC = {"tf32": 1, "bf16": 2, "fp64": 0, "tf32x3": 3, "bf16x3": 4}
DTYPE = {"tf32": "tf32 (f32 accumulate) + f64", "bf16": "bf16 (f32 accumulate) + f64",
         "tf32x3": "split tf32 x3 (f32 accumulate) + f64", "bf16x3": "split bf16 x3 (f32 accumulate) + f64",
         "fp64": "f64"}


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


# ---------------------------------------------------------------- workloads
def workload(name, nk=8, block=4):
    """(mesh, state, library params) of a named workload"""
    from paper_2507_22195_gb300 import inputs as I
    if name == "tgv_inviscid":
        mesh = I.periodic_mesh(nk, 3, 3)
        st = I.make_state(mesh, "tgv", 1e-3, 22197, 22198, M0=0.1)
        return mesh, st, dict(flux=2, Mach=0.1, Re=1600.0, Pr=0.71, viscous=0)
    if name == "tgv_viscous":
        full = I.periodic_mesh(16, 3, 4)
        mesh = I.sub_mesh(full, I.block_elements(16, block))
        st = I.make_state(mesh, "tgv", 1e-3, 22201, 22202, viscous=True, M0=0.1)
        return mesh, st, dict(flux=1, Mach=0.1, Re=1600.0, Pr=0.71, viscous=1)
    if name == "vortex":
        mesh = I.periodic_mesh(2, 2, 2, 0.0, 10.0)
        st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
        return mesh, st, dict(flux=1, Mach=0.1, viscous=0)
    raise ValueError(name)


# ---------------------------------------------------------------- oracle (CPU)
def oracle_sample(mesh, st, prm_kw, Ks, dvh, procs):
    """The FP64 CPU oracle, as it stands, on the elements Ks of a workload
    (residual, complex-step Jacobian, dense GEPP, b-hat and dV for the trace
    increment dvh), one element per spawned process on `procs` host cores.
    Returns (elements/s over the wall time, [seconds per element],
    {K: dV^K})."""
    import oracle
    oracle.build()
    prm = oracle.params(**prm_kw)
    t = time.time()
    res = oracle.condense_elements(prm, mesh, st, Ks, dvh, procs=procs)
    dt = time.time() - t
    return len(Ks) / dt, [r[3] for r in res], {K: (r[1], r[0]) for K, r in zip(Ks, res)}


def _oracle_prm(kw):
    return dict(flux=kw["flux"], Mach=kw["Mach"], Re=kw.get("Re", 1600.0), Pr=kw.get("Pr", 0.71),
                viscous=kw["viscous"])


def reference_main(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2507_22195_gb300 import inputs as I
    cores = min(os.cpu_count() or 1, 16)
    per_step = cores                     # one element per core per step
    mesh, st, kw = workload("tgv_inviscid")
    dvh = I.random_direction(st.vhat.shape, 77, 1e-3)
    Ks = [K * 37 % mesh.nK for K in range(per_step)]
    for _ in range(a.warmup):
        oracle_sample(mesh, st, _oracle_prm(kw), Ks, dvh, cores)
    times = []
    for _ in range(a.steps):
        t = time.time()
        oracle_sample(mesh, st, _oracle_prm(kw), Ks, dvh, cores)
        times.append(time.time() - t)
    tot = sum(times)
    val = per_step * a.steps / tot
    sample = f"{per_step} of the 512 elements per step (element ids 37k mod 512), one per process"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["tgv_inviscid"], "global_batch": 512, "seq_len": None,
                   "parallelism": "none"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ---------------------------------------------------------------- ranks
def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over all ranks (x itself without a process group): each
    rank times its own replica, and the job's time is the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, n_elem: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank condenses its own n_elem elements per
    step (weak scaling), in `seconds` of the slowest rank."""
    return world * n_elem * steps / seconds


# ---------------------------------------------------------------- GPU arm
def _to_dev(st, dev):
    import torch
    q = None if st.q is None else torch.tensor(st.q, device=dev)
    return torch.tensor(st.v, device=dev), torch.tensor(st.vhat, device=dev), q, torch.tensor(st.vstar, device=dev)


def once_main(a):
    """Workload setup, `warmup` condenses and one more, nothing timed: the
    command the ncu summaries under profiles/ are taken with.  The LU is
    launched kernel by kernel (no CUDA graph), which is what a kernel
    profiler replays."""
    os.environ["MEHDG_NO_GRAPH"] = "1"
    import torch
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw = workload(a.workload, a.nk, a.block)
    dev = torch.device("cuda:0")
    ctx = M.Context(mesh, prec=PREC[a.prec], **kw)
    ctx.set_state(*_to_dev(st, dev))
    for _ in range(a.warmup + 1):
        ctx.condense()
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    print(json.dumps({"once": True, "workload": a.workload, "nK": mesh.nK, "prec": a.prec,
                      "status_ok": bool((stat == 0).all()), "refine_iters": sorted(set(int(x) for x in iters)),
                      "launches": M.mehdg_launch_count()}))
    ctx.close()
    return 0


# DRAM bytes / algorithmic bytes of the outer trailing updates (split BF16),
# measured with ncu on one launch of each kind on a 27-element case of the
# same kernels (3^3 elements of the p = 3, m = 3 TGV, 2.8 GB of S): C is
# streamed once per launch, so the ratios carry over to the full workload.
# "one": the depth-256 update of the one-panel form; with merged pairs,
# "merged": the depth-512 update, "cols": the depth-256 update of the second
# panel's 256 columns, "rows": the depth-256 correction of its 256 block rows.
# A kind not captured since its kernel last changed has no entry, and the
# traffic is then reported as null.
TRAFFIC_RATIO = {"bf16x3": {"merged": 0.988, "cols": 0.867, "rows": 0.870}}
# tensor rate of a precision mode relative to BF16 (nominal dense GB300 rates:
# TF32 1.1, BF16 2.25 PFLOP/s) and the tensor products per method flop
TENSOR_RATE = {"bf16": 1.0, "bf16x3": 1.0, "tf32": 1.1 / 2.25, "tf32x3": 1.1 / 2.25}
PRODUCTS = {"bf16": 1, "bf16x3": 3, "tf32": 1, "tf32x3": 3}


def lu_pairs(prec):
    """whether the library merges the outer updates of two panels (split BF16,
    unless MEHDG_LU_PAIRS=0)"""
    return prec == "bf16x3" and os.environ.get("MEHDG_LU_PAIRS", "1") != "0"


def outer_updates(ld, pairs):
    """(kind, M, N, Kd) of every outer trailing update of one factorisation"""
    ups = []
    if not pairs:
        for c0 in range(0, ld, 256):
            r = ld - c0 - 256
            if r > 0:
                ups.append(("one", r, r, 256))
        return ups
    for ca in range(0, ld, 512):
        cb, jr = ca + 256, ca + 512
        if cb >= ld:
            break
        ups.append(("cols", ld - cb, 256, 256))
        nr = ld - jr
        if nr <= 0:
            break
        ups += [("rows", 256, nr, 256), ("merged", nr, nr, 512)]
    return ups


def update_bytes(M, N, Kd, kind=""):
    """algorithmic bytes of one update: C read and written (FP32; the block-row
    correction writes its result to the TRSM's FP32 operand panel instead of
    S, also 4 bytes) and the two operand panels (M x Kd and Kd x N, counted in
    FP32)"""
    return 8 * M * N + 4 * (M + N) * Kd


def trailing_bytes(ld, nK, pairs=False):
    """algorithmic bytes of all outer trailing updates of one condensation"""
    return sum(update_bytes(M, N, Kd, k) for k, M, N, Kd in outer_updates(ld, pairs)) * nK


def rel_per_element(a, b):
    """max over the leading index of ||a_i - b_i|| / ||b_i|| (numpy arrays)"""
    import numpy as np
    a2, b2 = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    return float((np.linalg.norm(a2 - b2, axis=1) / np.linalg.norm(b2, axis=1)).max())


def timed_condense(ctx, bh, steps, barrier):
    """device time of `steps` condensations (CUDA events on the current stream)"""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        ctx.condense(bh)
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1)


def fp64_full(mesh, st, kw, dev, bh_mixed, dV_mixed, dvh, barrier, M):
    """The FP64 GPU path on the whole workload: one timed condensation (its
    kernels were loaded by the subset comparison before), b-hat and the
    recovered dV against the mixed path's"""
    import torch
    ld = (5 * mesh.Nn + 255) // 256 * 256
    c = M.Context(mesh, prec=PREC["fp64"], **kw)
    c.set_state(*_to_dev(st, dev))
    bh = torch.empty_like(bh_mixed)
    ms = timed_condense(c, bh, 1, barrier)
    st64, it64 = c.status()
    dV = c.recover(dvh)
    torch.cuda.synchronize()
    out = {"value": mesh.nK / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": 1,
           "sample": f"all {mesh.nK} elements (FP64 S: {mesh.nK * 8 * ld * ld / 1e9:.1f} GB)",
           "err_bhat_mixed_vs_fp64": rel_per_element(bh_mixed.cpu().numpy(), bh.cpu().numpy()),
           "err_dV_mixed_vs_fp64": rel_per_element(dV_mixed, dV.cpu().numpy()),
           "refine_iters": sorted(set(int(x) for x in it64)), "status_ok": bool((st64 == 0).all())}
    c.close()
    return out


def subset_compare(mesh, st, kw, dev, n_s, prec, barrier, M):
    """FP64 and mixed GPU paths on the first n_s elements of a workload: rates
    (one untimed and one timed condensation each) and the b-hat error"""
    import numpy as np
    import torch
    from paper_2507_22195_gb300 import inputs as I
    m2 = I.sub_mesh(mesh, list(range(n_s)))
    s2 = I.State(v=st.v[:n_s].copy(), vhat=st.vhat[np.unique(mesh.face_gid[:n_s])].copy(),
                 q=None if st.q is None else st.q[:n_s].copy(), vstar=st.vstar[:n_s].copy())
    w = _to_dev(s2, dev)
    outs = {}
    for pr in ("fp64", prec):
        c2 = M.Context(m2, prec=PREC[pr], **kw)
        c2.set_state(*w)
        b2 = c2.condense()
        ms = timed_condense(c2, b2, 1, barrier)
        st2, _ = c2.status()
        outs[pr] = (b2.cpu().numpy(), ms, bool((st2 == 0).all()))
        c2.close()
    return {"value": n_s / (outs["fp64"][1] / 1e3), "unit": UNIT, "sample": f"the first {n_s} elements",
            "mixed_same_sample": n_s / (outs[prec][1] / 1e3),
            "err_bhat_mixed_vs_fp64": rel_per_element(outs[prec][0], outs["fp64"][0]),
            "status_ok": outs["fp64"][2] and outs[prec][2]}


def viscous_wave(block, dev, barrier, M, steps=2):
    """one wave of the viscous TGV workload (Re 1600, 16^3 macro-elements of
    4^3, p = 3): a block^3 block of it (block 7 holds 166 GB of FP32 S, under
    60 % of HBM) in split BF16 and split TF32, and the FP64 GPU path on its
    first 8 elements"""
    mesh, st, kw = workload("tgv_viscous", block=block)
    out = {"workload": f"viscous TGV Re=1600, {block}^3 block of the 16^3 x 4^3 mesh, p=3, ES",
           "nK": mesh.nK, "N_v": 5 * mesh.Nn, "steps": steps, "warmup": 1}
    w = _to_dev(st, dev)
    import torch
    for pr in ("bf16x3", "tf32x3"):
        c = M.Context(mesh, prec=PREC[pr], **kw)
        c.set_state(*w)
        bh = c.condense()
        ms = timed_condense(c, bh, steps, barrier)
        stt, it = c.status()
        out[pr] = {"value": mesh.nK * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                   "refine_iters": sorted(set(int(x) for x in it)), "status_ok": bool((stt == 0).all())}
        c.close()
        del bh
    del w
    torch.cuda.empty_cache()
    out["fp64_gpu"] = subset_compare(mesh, st, kw, dev, 8, "bf16x3", barrier, M)
    return out


def uneven_batch(nK, dev, barrier, M, sample_per_group=2):
    """the uneven batch workload: nK macro-elements with p in {1..4} and m in {2, 3, 4}
    drawn with seed 22199, each a TGV-like field with its own Mach number
    M0 ~ U(0.1, 0.3) plus U(-1e-2, 1e-2), viscous (Re 1600, Pr 0.71), ES flux,
    split BF16 with FP64 refinement: autotuned, then one timed condensation of
    the whole batch (groups streamed in waves when they exceed the memory
    budget); beside it the FP64 GPU path and the same mixed path on a seeded
    sample of every group the FP64 viscous Jacobian supports (p <= 3)"""
    import numpy as np
    import torch
    from paper_2507_22195_gb300 import inputs as I
    mesh = I.uneven_batch(nK, 22199)
    st = I.make_uneven_state(mesh, 1e-2, 22200, 22201, 22202, M0_range=(0.1, 0.3), viscous=True)
    kw = dict(flux=1, Mach=0.1, Re=1600.0, Pr=0.71, viscous=1)
    d = torch.device(dev)
    w = [torch.tensor(x, device=d) for x in (st.v, st.vhat, st.q, st.vstar)]
    ctx = M.BatchContext(mesh, prec=PREC["bf16x3"], **kw)
    ctx.set_state(*w)
    t0 = time.perf_counter()
    ctx.autotune(trial_max=8)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    bh = torch.empty(int(mesh.toff[-1]), dtype=torch.float64, device=d)
    ms = timed_condense(ctx, bh, 1, barrier)
    stat, it = ctx.status()
    rep = ctx.report()
    ctx.close()
    del w
    torch.cuda.empty_cache()
    # FP64 and mixed on a seeded sample of each group with p <= 3
    r = np.random.Generator(np.random.PCG64(22203))
    Ks = []
    for key in sorted(set(zip(mesh.p.tolist(), mesh.m.tolist()))):
        if key[0] > 3:
            continue
        ids = np.flatnonzero((mesh.p == key[0]) & (mesh.m == key[1]))
        Ks += sorted(r.choice(ids, size=min(sample_per_group, len(ids)), replace=False).tolist())
    sub = I.UnevenMesh(mesh.p[Ks], mesh.m[Ks], mesh.boxes[Ks], np.arange(6 * len(Ks), dtype=np.int64).reshape(-1, 6),
                       6 * len(Ks))
    voff, toff = mesh.voff, mesh.toff
    pick = lambda a, off, sc: np.concatenate([a[sc * off[K]:sc * off[K + 1]] for K in Ks])
    pickt = lambda a: np.concatenate([a[toff[g]:toff[g + 1]] for K in Ks for g in mesh.face_gid[K]])
    ss = I.State(v=pick(st.v, voff, 1), vhat=pickt(st.vhat), q=pick(st.q, voff, 3), vstar=pick(st.vstar, voff, 1))
    ws = [torch.tensor(x, device=d) for x in (ss.v, ss.vhat, ss.q, ss.vstar)]
    outs = {}
    for pr in ("fp64", "bf16x3"):
        c = M.BatchContext(sub, prec=PREC[pr], **kw)
        c.set_state(*ws)
        b = c.condense()
        msp = timed_condense(c, b, 1, barrier)
        s2, _ = c.status()
        outs[pr] = (b.cpu().numpy(), msp, bool((s2 == 0).all()))
        c.close()
    tf = sub.toff
    errs = [np.linalg.norm(outs["bf16x3"][0][tf[6 * i]:tf[6 * i + 6]] - outs["fp64"][0][tf[6 * i]:tf[6 * i + 6]]) /
            np.linalg.norm(outs["fp64"][0][tf[6 * i]:tf[6 * i + 6]]) for i in range(len(Ks))]
    groups = {f"p{g['p']}m{g['m']}": {"elements": g["elements"], "wave": g["wave"], "leaf_ctas": g["leaf_ctas"],
                                      "solve_ctas": g["solve_ctas"],
                                      "trials_ms": [round(t["ms"], 3) for t in g.get("trials", [])]}
              for g in rep["groups"]}
    return {"workload": f"{nK} independent macro-elements, p in {{1..4}} x m in {{2,3,4}} (seed 22199), TGV-like "
                        f"fields M0 ~ U(0.1,0.3) + U(-1e-2,1e-2), viscous Re=1600 Pr=0.71, ES, split bf16 x3 + f64 "
                        f"refinement, autotuned",
            "value": nK / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": 1,
            "status_ok": bool((stat == 0).all()), "refine_iters": sorted(set(int(x) for x in it)),
            "resident": rep["resident"], "budget_gb": rep["budget_bytes"] / 1e9, "autotune_s": tune_s,
            "groups": groups,
            "fp64_gpu": {"value": len(Ks) / (outs["fp64"][1] / 1e3), "unit": UNIT,
                         "mixed_same_sample": len(Ks) / (outs["bf16x3"][1] / 1e3),
                         "sample": f"{len(Ks)} elements: {sample_per_group} per (p, m) group with p <= 3 (seed 22203)",
                         "err_bhat_mixed_vs_fp64_max_per_element": float(max(errs)),
                         "status_ok": outs["fp64"][2] and outs["bf16x3"][2]}}


def graph_condense(dev, barrier, M, steps=20):
    """direct calls against the condensation replayed from one CUDA graph, on
    two launch-bound cases: the 2^3 x 2^3, p = 2 isentropic vortex (8
    elements) and a resident batch of 2048 elements with p in {1, 2, 3} and
    m in {2, 3} (seed 22204; inviscid TGV-like fields, ES, split BF16)"""
    import torch
    from paper_2507_22195_gb300 import inputs as I
    out = {}
    cases = []
    mesh, st, kw = workload("vortex")
    cases.append(("vortex_8", lambda: M.Context(mesh, prec=PREC["bf16x3"], **kw), mesh.nK,
                  (st.v, st.vhat, None, st.vstar), (mesh.n_global_faces, 5, mesh.n2)))
    um = I.uneven_batch(2048, 22204, p_choices=(1, 2, 3), m_choices=(2, 3))
    us = I.make_uneven_state(um, 1e-2, 22205, 22206, 22207)
    cases.append(("uneven_2048", lambda: M.BatchContext(um, prec=PREC["bf16x3"], flux=1, Mach=0.1), um.nK,
                  (us.v, us.vhat, None, us.vstar), (int(um.toff[-1]),)))
    for name, make, nK, state, bshape in cases:
        c = make()
        w = [None if a is None else torch.tensor(a, device=dev) for a in state]
        c.set_state(*w)
        bh = torch.empty(bshape, dtype=torch.float64, device=dev)
        for _ in range(3):
            c.condense(bh)
        ms_d = timed_condense(c, bh, steps, barrier)
        M.mehdg_condense_graph(c.ctx, bh)
        for _ in range(2):
            M.mehdg_condense_graph(c.ctx, bh)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(steps):
            M.mehdg_condense_graph(c.ctx, bh)
        e1.record(stream)
        barrier()
        ms_g = e0.elapsed_time(e1)
        stt, _ = c.status()
        out[name] = {"elements": nK, "direct": nK * steps / (ms_d / 1e3), "graph": nK * steps / (ms_g / 1e3),
                     "unit": UNIT, "steps": steps, "status_ok": bool((stt == 0).all())}
        c.close()
        del w
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=list(PREC))
    ap.add_argument("--workload", default="tgv_inviscid", choices=list(WORKLOADS))
    ap.add_argument("--nk", type=int, default=8, help="tgv_inviscid: nk^3 elements")
    ap.add_argument("--block", type=int, default=4, help="tgv_viscous: block^3 elements of the 16^3 mesh")
    ap.add_argument("--fp64-sample", type=int, default=8, help="elements of the FP64 subset comparison (0: skip)")
    ap.add_argument("--no-fp64-full", action="store_true", help="skip the FP64 GPU path on the whole workload")
    ap.add_argument("--viscous-block", type=int, default=7,
                    help="block^3 elements of the viscous TGV timed beside the headline (0: skip)")
    ap.add_argument("--uneven", type=int, default=4096,
                    help="elements of the uneven (p, m) batch timed beside the headline (0: skip)")
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
    from paper_2507_22195_gb300 import inputs as I
    mesh, st, kw = workload(a.workload, a.nk, a.block)
    vis = bool(kw["viscous"])
    dvh_np = I.random_direction(st.vhat.shape, 77, 1e-3)

    # CPU baseline and oracle reference values first (spawned pool, before any
    # CUDA call), rank 0 only: the oracle condenses a sample of the same
    # elements and recovers dV for the same seeded trace increment
    cpu, ref_dV = None, {}
    if rank == 0 and world == 1 and not a.no_cpu and a.workload == "tgv_inviscid":
        cores = min(os.cpu_count() or 1, 16)
        n = cores if a.cpu_sample < 0 else a.cpu_sample
        Ks = [K * 37 % mesh.nK for K in range(n)]
        t0 = time.time()
        val, per, ref_dV = oracle_sample(mesh, st, _oracle_prm(kw), Ks, dvh_np, cores)
        dt = time.time() - t0
        vmesh, vst, vkw = workload("vortex")
        vval, vper, _ = oracle_sample(vmesh, vst, _oracle_prm(vkw), list(range(vmesh.nK)), None,
                                      min(cores, vmesh.nK))
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} of the 512 elements (ids 37k mod 512: residual, complex-step Jacobian, dense GEPP, "
                         f"b-hat, dV), one per spawned process, {dt:.1f} s wall",
               "single_core": {"value": 1.0 / statistics.mean(per), "unit": UNIT,
                               "what": "1 / mean seconds per element of one process while all cores are busy"},
               "vortex_2x2x2_p2": {"value": vval, "single_core": 1.0 / statistics.mean(vper), "unit": UNIT,
                                   "sample": f"all {vmesh.nK} elements of the 2^3 x 2^3, p = 2 vortex (ES)"},
               "viscous_tgv_p3m4": "not timed: the oracle's dense A_qq of a p = 3, m = 4 element is 8.7 GB and "
                                   "its GEPP alone is 2.4e13 flop (hours on one core)"}

    import numpy as np
    import torch
    from paper_2507_22195_gb300 import mehdg as M

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    v, vh, q, vs = _to_dev(st, dev)
    ctx = M.Context(mesh, prec=PREC[a.prec], **kw)
    ctx.set_state(v, vh, q, vs)
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
    ms = timed_condense(ctx, bh, a.steps, barrier)
    launches = M.mehdg_launch_count() - n0
    prof = M.mehdg_profile_read(ctx.ctx)
    M.mehdg_profile_enable(ctx.ctx, False)
    clocks = clk.stop()
    stat, iters = ctx.status()
    ms = max_over_ranks(ms, dist, dev)
    value = job_rate(world, mesh.nK, a.steps, ms / 1e3)

    # end to end through the public API: pinned host inputs -> device,
    # condense, b-hat -> host, every step
    host = [torch.tensor(x).pin_memory() for x in (st.v, st.vhat, st.vstar) + ((st.q,) if vis else ())]
    hb = torch.empty(bh.shape, dtype=torch.float64).pin_memory()
    devb = [torch.empty(h.shape, dtype=torch.float64, device=dev) for h in host]
    ctx.set_state(devb[0], devb[1], devb[3] if vis else None, devb[2])
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        for d_, h_ in zip(devb, host):
            d_.copy_(h_, non_blocking=True)
        ctx.condense(bh)
        hb.copy_(bh, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    h2d = sum(h.numel() * 8 for h in host)
    d2h = hb.numel() * 8
    # recovery (eq. R2, R6) timed on its own, after the condensation above, for a
    # seeded trace increment
    ctx.set_state(v, vh, q, vs)
    del devb
    ctx.condense(bh)
    dvh = torch.tensor(dvh_np, device=dev)
    dV = ctx.recover(dvh)
    stream = torch.cuda.current_stream()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    r0.record(stream)
    for _ in range(a.steps):
        ctx.recover(dvh, out=dV)
    r1.record(stream)
    barrier()
    rec_ms = max_over_ranks(r0.elapsed_time(r1), dist, dev)
    rec = {"value": job_rate(world, mesh.nK, a.steps, rec_ms / 1e3), "unit": "macro-elements/s",
           "ms_per_step": rec_ms / a.steps,
           "what": "recover: dV = S^-1(-R_V - A_v,vhat dVhat) with FP64 refinement (and dQ when viscous), "
                   "seeded dVhat"}
    dV_np = dV.cpu().numpy()
    bh_mixed = bh.clone()
    err_or = None
    if ref_dV:
        e = {K: float(np.linalg.norm(dV_np[K] - d[0]) / np.linalg.norm(d[0])) for K, d in ref_dV.items()}
        # b-hat^K of the sample elements: the same elements in a context of their own with unshared
        # faces (each face one element side), the same state and precision
        Ks = sorted(ref_dV)
        sub = I.unshared(mesh, Ks)
        gsel = mesh.face_gid[Ks].ravel()
        s_sub = I.State(v=st.v[Ks].copy(), vhat=st.vhat[gsel].copy(), q=None, vstar=st.vstar[Ks].copy())
        csub = M.Context(sub, prec=PREC[a.prec], **kw)
        csub.set_state(*_to_dev(s_sub, dev))
        bsub = csub.condense().cpu().numpy()
        csub.close()
        eb = {K: float(np.linalg.norm(bsub[6 * i:6 * i + 6] - ref_dV[K][1]) / np.linalg.norm(ref_dV[K][1]))
              for i, K in enumerate(Ks)}
        err_or = {"value": max(max(e.values()), max(eb.values())),
                  "what": "max over the oracle's sample elements of the relative errors of b-hat^K and of dV^K "
                          "(recovered for the seeded dVhat after this condensation)",
                  "bhat_max": max(eb.values()), "bhat_median": float(statistics.median(eb.values())),
                  "dV_max": max(e.values()), "dV_median": float(statistics.median(e.values())),
                  "dV_per_element": {str(K): float("%.3g" % x) for K, x in sorted(e.items())},
                  "note": "KEPES: at a face point with P close to P-hat the hybrid's theta = sqrt(|P - P-hat| / "
                          "(P + P-hat)) has an unbounded derivative, and dV^K of such an element moves by up to "
                          "1e-8 under a one-ulp change of the inputs in the oracle itself"}

    # roofline of the dominant kernel: the outer trailing updates of the LU
    pk = peaks()
    gem = prof["lu_trailing_update"]
    ld = (5 * mesh.Nn + 255) // 256 * 256
    roof_t = None
    if a.prec == "fp64":
        fl = gem["flops"]
        ach = fl / (gem["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s", "frac": ach / 1.25,
                "traffic": None, "peak_source": "nominal FP64 rate of GB300 (no measured FP64 peak)",
                "kernel": "lu_trailing_update (FP64 SIMT, depth 256)", "launches": gem["launches"], "ms": gem["ms"]}
    else:
        pairs = lu_pairs(a.prec)
        ups = outer_updates(ld, pairs)
        byt = trailing_bytes(ld, mesh.nK, pairs) * a.steps
        sec = gem["ms"] / 1e3
        hbm = pk.get("hbm_gbs", 6800.0)
        ratios = TRAFFIC_RATIO.get(a.prec) if a.workload == "tgv_inviscid" else None
        tr = (sum(ratios[k] * update_bytes(M, N, Kd, k) for k, M, N, Kd in ups) * mesh.nK / len(ups)
              if ratios and ups and all(k in ratios for k, _, _, _ in ups) else None)
        kernel = ("lu_trailing_update (tcgen05, 128 x 256 tiles; per pair of outer panels one depth-512 update "
                  "and two depth-256 updates of 256 rows or columns)" if pairs
                  else "lu_trailing_update (tcgen05, depth 256)")
        roof_h = {"bound": "hbm", "achieved": byt / sec / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": byt / sec / 1e9 / hbm, "traffic": tr,
                  "traffic_unit": "bytes per launch (27-element ncu captures, scaled)" if tr else None,
                  "algorithmic_per_launch": byt / max(gem["launches"], 1),
                  "peak_source": "measured" if "hbm_gbs" in pk else "fallback",
                  "kernel": kernel, "launches": gem["launches"],
                  "launches_expected": len(ups) * a.steps, "ms": gem["ms"]}
        # the same launches on the tensor pipe: 2 M N Kd method flops per
        # update, and the split modes issue three products per method flop;
        # the peak is the measured sustained BF16 rate (TF32: x 1.1/2.25)
        sus = pk.get("bf16_tflops_sustained", 1700.0) * TENSOR_RATE[a.prec]
        mfl = gem["flops"] / sec / 1e12
        tfl = PRODUCTS[a.prec] * mfl
        roof_t = {"bound": "tensor", "achieved": tfl, "peak": sus, "unit": "TFLOP/s", "frac": tfl / sus,
                  "traffic": tr,
                  "achieved_counts": "tensor-core products: %d per method flop" % PRODUCTS[a.prec],
                  "method_flops_achieved": mfl, "method_frac": mfl / sus,
                  "peak_source": ("measured sustained bf16" if "bf16_tflops_sustained" in pk else "fallback")
                  + ("" if TENSOR_RATE[a.prec] == 1.0 else " x nominal tf32/bf16 ratio"),
                  "kernel": kernel, "launches": gem["launches"], "ms": gem["ms"],
                  "flops_per_step": gem["flops"] / a.steps,
                  "lu_method_flops_per_step": 2.0 / 3.0 * (5 * mesh.Nn) ** 3 * mesh.nK,
                  "traffic_vs_compulsory": byt / a.steps / (2 * 4 * ld * ld * mesh.nK)}
        # the binding roofline: the larger of the two floors (time at peak)
        floor_h, floor_t = byt / (hbm * 1e9), PRODUCTS[a.prec] * gem["flops"] / (sus * 1e12)
        roof_h["floor_ms"], roof_t["floor_ms"] = floor_h * 1e3, floor_t * 1e3
        roof, roof_t = (roof_t, roof_h) if floor_t > floor_h else (roof_h, roof_t)
    fp = None
    if a.prec != "fp64" and a.fp64_sample > 0:
        ctx.close()
        del bh
        torch.cuda.empty_cache()
        fp = {"subset": subset_compare(mesh, st, kw, dev, min(a.fp64_sample, mesh.nK), a.prec, barrier, M)}
        if not a.no_fp64_full:
            fp["full"] = fp64_full(mesh, st, kw, dev, bh_mixed, dV_np, dvh, barrier, M)
            fp.update(value=fp["full"]["value"], unit=UNIT)
    else:
        ctx.close()
    del v, vh, q, vs
    torch.cuda.empty_cache()
    def side(fn, *args):
        """a measurement beside the headline: its failure is reported in its key"""
        try:
            return fn(*args)
        except Exception as ex:                       # noqa: BLE001
            torch.cuda.synchronize()
            return {"error": f"{type(ex).__name__}: {ex}"[:400]}
        finally:
            torch.cuda.empty_cache()

    visc = None
    if a.workload == "tgv_inviscid" and a.viscous_block > 0 and world == 1:
        visc = side(viscous_wave, a.viscous_block, dev, barrier, M)
    unev = None
    if a.workload == "tgv_inviscid" and a.uneven > 0 and world == 1:
        unev = side(uneven_batch, a.uneven, dev, barrier, M)
    graph = side(graph_condense, dev, barrier, M) if a.workload == "tgv_inviscid" and world == 1 else None

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[a.prec], "data": "synthetic",
            "config": {"workload": WORKLOADS[a.workload], "global_batch": mesh.nK, "seq_len": None,
                       "parallelism": f"dp{world}" if world > 1 else "none", "nK": mesh.nK, "p": mesh.p,
                       "m": mesh.m, "N_v": 5 * mesh.Nn, "prec": a.prec,
                       "l2": "inputs larger than L2 (dense S^K of all elements: %.1f GB)" % (
                           mesh.nK * ld * ld * (8 if a.prec == "fp64" else 4) / 1e9)},
            "roofline": roof,
            "roofline_other": roof_t,
            "cpu_baseline": cpu,
            "err_vs_oracle": err_or,
            "e2e": {"value": job_rate(world, mesh.nK, a.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "refine_iters": sorted(set(int(x) for x in iters)),
            "status_ok": bool((stat == 0).all()),
            "phases_ms_per_step": {k: round(vv["ms"] / a.steps, 3) for k, vv in prof.items()},
            "fp64_gpu": fp,
            "viscous_tgv": visc,
            "uneven_batch": unev,
            "graph_condense": graph,
            "recover": rec,
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
