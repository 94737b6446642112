#!/usr/bin/env python
"""Benchmark: path solves/s to 1e-5 m stationarity, forward + implicit backward.

Workload (one step): the urban canyon -- 32 vertical facades (5-30 m) on a
200 x 200 m grid plus their 128 edges, a 32-object alphabet (16 facades, 16
edges), TX at (100, 100, 10) m and a 32 x 32 RX grid at 1.5 m; every order-3
sequence for every RX: 32^3 * 1024 = 33,554,432 paths.  A step enumerates,
solves (plain init, FP32 BFGS with Eq. 6 step sizes, a Newton polish whose
gradient is formed in double-float arithmetic, validity), and back-propagates the sum of the valid solved paths'
lengths to TX, RX and every vertex by implicit differentiation -- one
fpt_solve_grad call.  A path counts as solved when its stationarity residual
is <= 1e-5 m.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload canyon|city]

--workload city times the ragged large batch instead: 100,000,000 seeded
sequences of order 1-5 on a 256-object city with the learned start (and the
plain start alongside), one fpt_solve_grad call per step.

Under torchrun (N > 1) every rank solves its own copy of the workload (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "path solves/s to 1e-5 m stationarity, fwd+implicit bwd; learned vs plain init"
UNIT = "solves/s"
WORKLOAD = ("urban canyon: 32 facades + 128 edges, 32-object alphabet (16 R + 16 D), order 3, "
            "1 TX x 32x32 RX = 33,554,432 paths; plain init; FP32 BFGS + Eq.6 fixed point, Newton polish with an "
            "extended-precision gradient, validity, implicit backward of the sum of valid path lengths "
            "(one fpt_solve_grad call)")
L2_FLUSH_BYTES = 512 << 20


# ---------------------------------------------------------------------------
# algorithmic work (FP32 flops, FMA = 2) of the BFGS kernel, per path
# ---------------------------------------------------------------------------
def bfgs_flops_per_iter(n: int, fp: int, nq: int | None = None) -> int:
    """Static op count of one BFGS step of order n with nq planar reflectors (2 parameters each) and n - nq
    edges (1 parameter each), fp rounds of Eq. 6 (bfgs.cuh).  nq = n is the unified d = 2 kernel."""
    nq = n if nq is None else nq
    ne = n - nq
    m, s = n + nq, n + 1
    hp = m * (m + 1) // 2
    direction = 2 * m * m + m              # p = -H g
    world = 15 * nq + 9 * ne               # A_i p_i and |A_i p_i|^2
    segs = 3 * (n - 1) + 10 * s            # q_j, q_j.z_j, q_j.q_j
    fixed = fp * (9 * s + 1)               # Eq. 6 rounds
    step = 2 * m                           # s = alpha p, t += s
    grad = 28 * nq + 17 * ne + 9 * s       # z_j, |z_j|, u_j, g
    curv = 7 * m + 4                       # y, s.y, s.s, y.y, guard
    update = 1 + 2 * m * m + 2 * m + 3 + 4 * m + 4 * hp  # inverse-Hessian update
    conv = 2 + n
    return direction + world + segs + fixed + step + grad + curv + update + conv


def bfgs_flops_init(n: int, nq: int | None = None) -> int:
    nq = n if nq is None else nq
    return 28 * nq + 17 * (n - nq) + 9 * (n + 1)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_identifier(torch, dev) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("bfgs.cuh", "k_bfgs.cu", "k_bfgs_pat.cu", "fpt_device.cuh", "fpt_kernels.h"):
        with open(os.path.join(ROOT, "paper_2510_16172_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


# FP32 operations (FFMA counted as 2) the polish executes per path of the urban-canyon batch, both passes:
# ncu SASS counters on the 8.4M-path canyon (profiles/polish_op_count_urban_canyon_8M.md).  Most are the
# error-free transformations of its double-float gradient.
POLISH_FP32_OPS_PER_PATH = 1674

# DRAM traffic per launch from an ncu capture (profiles/), valid for the kernel sources with this hash.
NCU_TRAFFIC = {
    # DRAM read + write of one step's bfgs_refill_kernel<3, Q> launches, ncu capture of these sources
    # (profiles/launch_list_urban_canyon_33M.md)
    ("39df173948b3", "bfgs"): 570.1e6,
    ("f6467978743f", "bfgs"): 568.6e6,
    ("886638d3c5ec", "bfgs"): 568.8e6,
    ("e1979203e5c7", "bfgs"): 567.1e6,
}


# ---------------------------------------------------------------------------
# the oracle (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(sc, n_paths, seed, target_s=None, max_paths=None, decode=None, threads=None):
    """Oracle fwd+bwd on a seeded uniform sample of the workload: (solved/s, sample size, seconds, threads).

    decode(g) -> (ids, order, tx_idx, rx_idx) of global path indices g (default: the canyon's order-3
    exhaustive enumeration).  threads: host threads (default all cores)."""
    import numpy as np

    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    threads = threads or os.cpu_count() or 1
    decode = decode or (lambda g: oracle.exhaustive_paths(sc, 3, 3, g))

    def run(m):
        g = np.sort(rng.choice(n_paths, m, replace=False))
        ids, order, ti, ri = decode(g)
        t0 = time.perf_counter()
        out = oracle.solve(sc, ids, order, ti, ri, dL=np.ones(m), n_threads=threads)
        dt = time.perf_counter() - t0
        return int(((out["status"] & oracle.SOLVED) > 0).sum()), dt

    m = 20000
    solved, dt = run(m)
    if target_s:
        m = int(min(max_paths or 4_000_000, max(m, m * target_s / max(dt, 1e-3))))
        solved, dt = run(m)
    return solved / dt, m, dt, threads


def sample_outputs(ctx, scene, batch, out, torch, fpt, dev, n_paths, m=100_000, seed=7):
    """The timed step's outputs on a seeded uniform sample of paths, and the implicit backward of the sum
    of the sample's valid solved lengths (fpt_backward with dL = 1 on those paths, 0 elsewhere).  The
    comparison with the oracle is made on the host by oracle_agreement()."""
    import numpy as np

    g = np.sort(np.random.default_rng(seed).choice(n_paths, m, replace=False))
    gi = torch.as_tensor(g, device=dev)
    st = out["status"][gi]
    both = fpt.ST_VALID | fpt.ST_SOLVED
    w = (st & both) == both
    dL = torch.zeros(n_paths, dtype=torch.float32, device=dev)
    dL[gi] = w.float()
    grads = fpt.backward(ctx, scene, batch, out["T"], out["status"], None, dL)
    ctx.sync()
    res = {"g": g, "T": out["T"][gi].double().cpu().numpy(), "L": out["L"][gi].double().cpu().numpy(),
           "status": st.cpu().numpy().astype(np.int64), "w": w.cpu().numpy(),
           "grads": [x.double().cpu().numpy() for x in grads]}
    del dL
    return res


def residual_distribution(ctx, scene, batch, params, out, torch, fpt):
    """The stationarity residual rho (the world-space size of the Newton step at the returned point) of one
    more, untimed solve with the bench's settings: quantiles over the solved paths, and over the paths that
    BFGS reported converged but the polish did not certify.  Overwrites the solve outputs in `out`."""
    rho = torch.empty(batch.n_paths, dtype=torch.float32, device=out["T"].device)
    o = dict(out)
    o["rho"] = rho
    fpt.solve(ctx, scene, batch, params, out=o)
    ctx.sync()
    st = o["status"]
    groups = {"solved": (st & fpt.ST_SOLVED) != 0,
              "converged_not_solved": ((st & fpt.ST_CONVERGED) != 0) & ((st & fpt.ST_SOLVED) == 0)}
    res = {}
    for name, m in groups.items():
        r = rho[m]
        r = torch.sort(r[torch.isfinite(r)]).values
        n = r.numel()
        res[name] = {"paths": int(n)}
        if n:
            res[name].update({"p50_m": float(r[(n - 1) // 2]), "p99_m": float(r[int(0.99 * (n - 1))]),
                              "max_m": float(r[-1])})
    del rho, o
    return res


def oracle_agreement(sc, S, decode):
    """Error of the timed step's results against the oracle on the sample of sample_outputs():
    solved-set agreement, max |dX| and |dL|/L over the paths both solve, validity-mask mismatches, and
    the relative error of the sample's TX/RX/vertex gradients against the oracle's FP64 implicit VJP
    (Eq. 12-13) evaluated at the GPU's parameters."""
    import numpy as np

    import oracle

    oracle.build()
    ids, order, ti, ri = decode(S["g"])
    t0 = time.perf_counter()
    ref = oracle.solve(sc, ids, order, ti, ri)
    w = S["w"].astype(np.float64)
    at = oracle.solve(sc, ids, order, ti, ri, solver=oracle.BFGS, max_iters=0, T_start=S["T"], dL=w)
    dt = time.perf_counter() - t0
    gs = (S["status"] & oracle.SOLVED) > 0
    rs = (ref["status"] & oracle.SOLVED) > 0
    both = gs & rs
    slot = np.arange(ids.shape[1])[None, :] < np.asarray(order)[:, None]
    dx = np.where(slot, np.linalg.norm(at["X"] - ref["X"], axis=2), 0.0).max(axis=1)
    dl = np.abs(S["L"] - ref["L"]) / np.maximum(ref["L"], 1e-30)
    vmis = ((S["status"] & oracle.VALID) > 0) != ((ref["status"] & oracle.VALID) > 0)
    far = np.abs(ref["bdist"]) > 1e-5
    want = oracle.reduce_gradients(sc, ids, order, ti, ri, at["dtheta"] * w[:, None])
    rel = {}
    for name, got, exp in zip(("tx", "rx", "vertices"), S["grads"], want):
        rel[name] = float(np.abs(got - exp).max() / max(np.abs(exp).max(), 1e-30))
    return {"sample_paths": int(len(S["g"])), "solved_both": int(both.sum()), "solved_gpu_only": int((gs & ~rs).sum()),
            "solved_oracle_only": int((rs & ~gs).sum()),
            "max_dX_m": float(dx[both].max()) if both.any() else None,
            "max_rel_dL": float(dl[both].max()) if both.any() else None,
            "mask_mismatches": int((vmis & both).sum()),
            "mask_mismatches_beyond_1e-5_m_of_a_boundary": int((vmis & both & far).sum()),
            "gradient_paths": int(w.sum()), "gradient_rel_err": rel,
            "note": "oracle = FP64 damped Newton on the same paths; dX of the GPU's parameters mapped to points in "
                    "FP64; gradients: fpt_backward with dL = 1 on the sample's valid solved paths vs the oracle's VJP "
                    "at the GPU's parameters", "oracle_s": round(dt, 2)}


def oracle_decode_canyon(sc, g):
    import oracle

    return oracle.exhaustive_paths(sc, 3, 3, g)


def combine_ranks(total_ms, solved, dist, device):
    """Whole-job figures of a replicated run: the slowest rank's timed total and the sum of the ranks' solved
    paths (every rank solves its own copy of the workload; nothing else is exchanged)."""
    if dist is None:
        return float(total_ms), float(solved)
    import torch

    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(solved)], device=device, dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the machine's host cores, rank 0 only."""
    if rank != 0:
        return
    from paper_2510_16172_gb300 import scenes

    sc = scenes.urban_canyon(0)
    n_paths = 32 ** 3 * len(sc.rx)
    rate0, m0, dt0, threads = oracle_rate(sc, n_paths, 1)
    per_step = int(min(2_000_000, max(20000, rate0 * 4.0)))  # about 4 s of CPU work per step
    import numpy as np

    import oracle

    rng = np.random.default_rng(2)
    times, solved = [], 0
    for k in range(args.warmup + args.steps):
        g = np.sort(rng.choice(n_paths, per_step, replace=False))
        ids, order, ti, ri = oracle.exhaustive_paths(sc, 3, 3, g)
        t0 = time.perf_counter()
        out = oracle.solve(sc, ids, order, ti, ri, dL=np.ones(per_step), n_threads=threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            solved += int(((out["status"] & oracle.SOLVED) > 0).sum())
    total = sum(times)
    value = solved / total
    sample = f"{per_step} uniformly sampled paths of the workload per step (seeded), FP64 damped Newton + VJP"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_paths_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def library_defaults_leg(ctx, scene, batch, out, grads, mask, flush, stream, torch, fpt, dev, steps=5, warmup=2):
    """The same canyon step (solve, polish, validity, implicit backward of the valid solved lengths) with the
    library's default solver settings instead of the benchmark's step cap and kink stop; timed the same way
    (CUDA events, L2 flushed between steps), outside the headline's timed region."""
    p = fpt.default_params()

    def step():
        fpt.solve_grad(ctx, scene, batch, p, dL_status_mask=mask, out=out, grads=grads)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    solved = fpt.count_status(ctx, out["status"], fpt.ST_SOLVED)
    # kink_stop 0 selects the library's default, one tenth of the degeneracy tolerance
    kink = float(p.kink_stop) if p.kink_stop > 0 else 0.1 * float(p.deg_tol)
    return {"value": solved / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "solved_per_step": solved, "steps": steps,
            "max_bfgs_iters": int(p.max_iters), "kink_stop_m": kink}

def run_ours(args, world, rank, local_rank):
    import numpy as np
    import torch

    from paper_2510_16172_gb300 import build, fpt, scenes

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

    sc = scenes.urban_canyon(0, rx_grid=args.rx_grid)
    ctx = fpt.Context(local_rank)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    N = batch.n_paths
    params = fpt.default_params(max_iters=args.max_iters, kink_stop=args.kink_stop)
    out = fpt.alloc_outputs(ctx, batch, with_X=False, with_rho=False, with_iters=True)
    grads = (torch.empty((scene.n_tx, 3), device=dev), torch.empty((scene.n_rx, 3), device=dev),
             torch.empty((scene.n_obj, 3, 3), device=dev))
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fpt.solve_grad(ctx, scene, batch, params, dL_status_mask=mask, out=out, grads=grads)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    torch.cuda.synchronize(dev)

    fpt.profile_enable(ctx, True)
    fpt.profile_read(ctx, reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(gpu_identifier(torch, dev)) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.zero_()  # write 512 MB between steps: evict L2 (129 MB)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kms, klaunch = fpt.profile_read(ctx, reset=True)
    fpt.profile_enable(ctx, False)
    total_ms = sum(step_ms)
    solved = fpt.count_status(ctx, out["status"], fpt.ST_SOLVED)
    iters = out["iters"].to(torch.int64)
    total_iters = int(iters.sum().item())
    run_paths = N - fpt.count_status(ctx, out["status"], fpt.ST_REPEAT)
    total_ms, solved_all = combine_ranks(total_ms, solved, dist, dev)
    value = solved_all * args.steps / (total_ms / 1e3)
    # the step's run statistics: converged and FP64-polished fractions, BFGS steps (mean above, p99 here)
    stats = {"converged_fraction": fpt.count_status(ctx, out["status"], fpt.ST_CONVERGED) / N,
             "fp64_fraction": fpt.count_status(ctx, out["status"], fpt.ST_FP64) / N}
    hist = torch.bincount(iters[(out["status"] & fpt.ST_REPEAT) == 0], minlength=256).double()
    cdf = torch.cumsum(hist, 0) / hist.sum().clamp(min=1.0)
    stats["bfgs_iters_p99"] = int((cdf < 0.99).sum().item())
    del hist, cdf
    sample = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample = sample_outputs(ctx, scene, batch, out, torch, fpt, dev, N)

    # roofline of the dominant kernel (device time per launch from the library's event timing)
    peaks = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    # algorithmic flops of the pattern kernels: per path, its pattern's count per step x its steps
    ids = fpt.enumerate(ctx, batch)[0]
    is_quad = torch.tensor(np.asarray(sc.types) == scenes.QUAD, device=dev)
    qbits = is_quad[ids.long()].to(torch.int64)
    pattern = qbits[:, 0] | (qbits[:, 1] << 1) | (qbits[:, 2] << 2)  # bit i: slot i is a reflector
    nq = qbits.sum(dim=1)
    del ids, qbits
    run = (out["status"] & fpt.ST_REPEAT) == 0
    f_step = torch.tensor([bfgs_flops_per_iter(3, params.fp_iters, q) for q in range(4)], dtype=torch.float64,
                          device=dev)
    f_init = torch.tensor([bfgs_flops_init(3, q) for q in range(4)], dtype=torch.float64, device=dev)
    per_path = (f_init[nq] + f_step[nq] * iters.double()) * run.double()
    bfgs_flops = float(per_path.sum().item())
    # the static count per pattern kernel (one launch each per step), for comparison with executed FP32 ops
    flops_by_pattern = {int(q): float(per_path[pattern == q].sum().item()) for q in range(8)}
    del nq, run, per_path, pattern
    # obstruction of the step's valid solved paths (post-processing, not part of the timed step)
    blocked = fpt.occlusion(ctx, scene, batch, out["T"], out["status"], mask)
    torch.cuda.synchronize(dev)
    oa, ob = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    oa.record(stream)
    for _ in range(5):
        fpt.occlusion(ctx, scene, batch, out["T"], out["status"], mask, out=blocked)
    ob.record(stream)
    ob.synchronize()
    occ = {"ms_per_call": oa.elapsed_time(ob) / 5, "paths_tested": int(fpt.count_status(ctx, out["status"], mask)),
           "blocked": int((blocked != 0).sum().item()),
           "kernel": "occlusion_kernel: every segment of each valid solved path against the 32 facades"}
    del blocked
    names = {fpt.K_BFGS: "bfgs_refill_kernel<3, Q> (8 reflector/edge patterns)",
             fpt.K_POLISH: "polish_ff_kernel<3> + polish64_kernel<3> (rescue)",
             fpt.K_BACKWARD: "backward_kernel<3> + backward_rescue_kernel<3>", fpt.K_OTHER: "backward_finalize_kernel",
             fpt.K_MLP: "mlp_infer_kernel (learned start)"}
    dom = max(range(fpt.K_COUNT), key=lambda k: kms[k])
    clocks = clk.summary()
    roof_bfgs = {"kernel": names[fpt.K_BFGS], "bound": "alu",
                 "achieved": bfgs_flops / (kms[fpt.K_BFGS] / args.steps * 1e-3) / 1e12,
                 "peak": fp32_peak, "unit": "TFLOP/s",
                 "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock of measured peaks)",
                 "traffic": NCU_TRAFFIC.get((kernel_source_hash(), "bfgs"))}
    roof_bfgs["frac"] = roof_bfgs["achieved"] / roof_bfgs["peak"]
    if clocks.get("sm_mhz"):
        roof_bfgs["frac_at_measured_clock"] = roof_bfgs["achieved"] / (fp32_peak * clocks["sm_mhz"] / sm_max)
    roof_polish = {"kernel": names[fpt.K_POLISH], "bound": "alu",
                   "achieved": POLISH_FP32_OPS_PER_PATH * N / (kms[fpt.K_POLISH] / args.steps * 1e-3) / 1e12,
                   "peak": fp32_peak, "unit": "TFLOP/s",
                   "basis": f"executed FP32 operations, {POLISH_FP32_OPS_PER_PATH} per path of the batch (ncu SASS "
                            "counters, both passes; mostly the double-float gradient's error-free sums)",
                   "traffic": None}
    roof_polish["frac"] = roof_polish["achieved"] / roof_polish["peak"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.rx_grid == 32 else WORKLOAD + f" (RX grid {args.rx_grid}^2)",
                       "n_paths": N, "init": "plain", "max_bfgs_iters": args.max_iters, "fp_iters": 1,
                       "kink_stop_m": args.kink_stop,
                       "polish": "1 Newton step, double-float gradient (FP64 for ill-conditioned Hessians)",
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
            "solved_per_step": solved, "solved_fraction": solved / N, "mean_bfgs_iters": total_iters / max(1, run_paths),
            **stats,
            "kernel_ms_per_step": {names[k]: kms[k] / args.steps for k in range(fpt.K_COUNT) if klaunch[k]},
            "dominant_kernel": names[dom],
            "roofline": roof_bfgs,
            "polish_roofline": roof_polish,
            "bfgs_flops_by_pattern": flops_by_pattern,
            "gpu_launches": int(sum(klaunch)),
            "clocks": clocks,
            "occlusion": occ}
    if dom != fpt.K_BFGS:
        line["roofline_note"] = f"dominant kernel is {names[dom]}; roofline reported for the FP32 solver kernel"
    line["residual_m"] = residual_distribution(ctx, scene, batch, params, out, torch, fpt)
    if world == 1:
        line["at_library_defaults"] = library_defaults_leg(ctx, scene, batch, out, grads, mask, flush, stream, torch,
                                                           fpt, dev)

    # end to end through the public API with host buffers
    if not args.no_e2e:
        line["e2e"] = e2e(args, sc, ctx, dev, torch, fpt)
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, m, dt, threads = oracle_rate(sc, N, 1, target_s=args.cpu_seconds)
        rate1, m1, dt1, _ = oracle_rate(sc, N, 2, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{m} seeded uniformly sampled paths of the workload, FP64 damped Newton "
                                          f"+ implicit VJP, {dt:.1f} s on {threads} threads",
                                "value_1_core": rate1, "sample_1_core": f"{m1} paths, {dt1:.1f} s on 1 thread"}
        line["oracle_agreement"] = oracle_agreement(sc, sample, lambda g: oracle_decode_canyon(sc, g))
    if rank == 0 and world == 1 and not args.no_learned:
        line["learned_vs_plain"], net = learned_vs_plain(ctx, fpt, args.epochs)
        if not args.no_city:
            # config 5, the ragged city batch, from the network just trained (learned) and from t = 1/2
            net.attach()
            m = measure_city(ctx, dev, args, args.city_steps, 2, True)
            L, P = m["res"][1], m["res"][0]
            line["ragged_city"] = {
                "workload": CITY_WORKLOAD, "n_paths": m["n_paths"], "steps": args.city_steps, "warmup": 2,
                "learned": {k: L[k] for k in ("value", "ms_per_step", "solved_per_step", "mean_bfgs_iters",
                                              "kernel_ms_per_step", "launches")},
                "plain": {k: P[k] for k in ("value", "ms_per_step", "solved_per_step", "mean_bfgs_iters",
                                            "kernel_ms_per_step", "launches")},
                "unit": UNIT, "roofline": m["roofline"], "clocks": L["clocks"],
                "launch_structure": "one launch per (order, reflector/edge pattern) bucket, on four streams"}
        net.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def learned_vs_plain(ctx, fpt, epochs):
    """The learned start against the plain one (same solver, same unseen scenes).

    The network (64-256-256-256-8, GELU, BF16 weights, FP32 accumulation) is
    trained here by the library's tensor-core kernels on the solver's own
    solutions of seeded order-1..4 sequences on 50 random 10 m scenes (8 quads
    and 4 edges each), then both starts solve seeded order-1..4 sequences on 10
    unseen scenes; each side is timed with CUDA events over solve + implicit
    backward.
    """
    from paper_2510_16172_gb300 import warmstart

    t0 = time.perf_counter()
    # 285,000 sequences per scene give about 10 M solved paths as training samples
    net, ev = warmstart.run(ctx, per_pair_train=285_000, per_pair_eval=200_000, epochs=epochs)
    res = {"workload": "train: 50 seeded 10 m scenes (8 quads + 4 edges) x 285,000 seeded order-1..4 sequences, "
                       f"solved paths as targets, {epochs} epochs of Adam; eval: 10 unseen scenes x 200,000 "
                       "sequences",
           "train_samples": ev["train_samples"], "train_loss_per_epoch": ev["train_loss_per_epoch"],
           "train_s": ev["train_s"],
           "train_tflops": MLP_TRAIN_FLOP * (ev["train_samples"] // 8192) * 8192 * epochs / ev["train_s"] / 1e12,
           "plain": ev["plain"], "learned": ev["learned"],
           "learned_over_plain_solves_per_s": ev["learned"]["solves_per_s"] / ev["plain"]["solves_per_s"],
           "learned_over_plain_iterations": ev["learned"]["mean_bfgs_iters"] / ev["plain"]["mean_bfgs_iters"],
           "wall_s": time.perf_counter() - t0}
    return res, net


CITY_WORKLOAD = ("ragged city: 256 objects (154 facades 5-30 m, 102 of their edges, 500 x 500 x 60 m), 1 TX x 16 RX, "
                 "100,000,000 seeded sequences of order 1-5; learned start (the network trained here on the solver's "
                 "solutions of 50 random 10 m scenes), FP32 BFGS + Eq.6 fixed point, double-float Newton polish, "
                 "validity, implicit backward of the sum of valid path lengths (one fpt_solve_grad call)")
CITY_WORKLOAD_PLAIN = ("ragged city: 256 objects (154 facades 5-30 m, 102 of their edges, 500 x 500 x 60 m), 1 TX x 16 "
                       "RX, seeded sequences of order 1-5; plain start, FP32 BFGS + Eq.6 fixed point, double-float "
                       "Newton polish, validity, implicit backward of the sum of valid path lengths (one fpt_solve_grad "
                       "call)")


def measure_city(ctx, dev, args, steps, warmup, learned, dist=None):
    """The ragged large batch (config 5): 100,000,000 seeded sequences of order 1-5 on the 256-object city, one
    fpt_solve_grad per step (solve and implicit backward of the sum of the valid solved lengths), timed with
    CUDA events (L2 flushed between steps) from the learned start (when `learned`: the network attached to ctx)
    and from the plain start.  Returns per start the whole-job solves/s, ms per step, solved paths, mean BFGS
    steps, kernel ms per class and launches, and the BFGS roofline of the main start."""
    import numpy as np
    import torch

    from paper_2510_16172_gb300 import fpt, scenes

    sc = scenes.city(0, n_rx=16)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    per_pair = args.city_paths // (len(sc.tx) * len(sc.rx))
    batch = fpt.Batch.seeded(ctx, scene, 5, per_pair, 1, 5)
    N = batch.n_paths
    out = fpt.alloc_outputs(ctx, batch, with_X=False, with_rho=False, with_iters=True)
    grads = (torch.empty((scene.n_tx, 3), device=dev), torch.empty((scene.n_rx, 3), device=dev),
             torch.empty((scene.n_obj, 3, 3), device=dev))
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    main = 1 if learned else 0
    res = {}
    for init in ((1, 0) if learned else (0,)):
        params = fpt.default_params(max_iters=args.max_iters, init_mode=init)
        for _ in range(warmup):
            fpt.solve_grad(ctx, scene, batch, params, dL_status_mask=mask, out=out, grads=grads)
        ctx.sync()
        fpt.profile_enable(ctx, True)
        fpt.profile_read(ctx, reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with ClockSampler(gpu_identifier(torch, dev)) as clk:
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                fpt.solve_grad(ctx, scene, batch, params, dL_status_mask=mask, out=out, grads=grads)
                ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
        ctx.sync()
        total_ms = sum(a.elapsed_time(b) for a, b in ev)
        kms, klaunch = fpt.profile_read(ctx, reset=True)
        fpt.profile_enable(ctx, False)
        solved = fpt.count_status(ctx, out["status"], fpt.ST_SOLVED)
        run = (out["status"] & fpt.ST_REPEAT) == 0
        iters = out["iters"].to(torch.int64)
        if dist:
            dist.barrier()
        total_ms, solved_all = combine_ranks(total_ms, solved, dist, dev)
        res[init] = {"value": solved_all * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
                     "solved_per_step": solved, "mean_bfgs_iters": float(iters[run].double().mean()),
                     "kernel_ms": kms, "launches": int(sum(klaunch)), "clocks": clk.summary()}
        if init == main:
            # algorithmic BFGS flops of this step: per path, its (order, reflector count)'s count per step
            ids, order, _, _ = fpt.enumerate(ctx, batch)
            is_quad = torch.tensor(np.asarray(sc.types) == scenes.QUAD, device=dev)
            flops = 0.0
            for n in range(1, 6):
                sel = order == n
                nq = (is_quad[ids[sel][:, :n].long()]).sum(dim=1)
                f_step = torch.tensor([bfgs_flops_per_iter(n, params.fp_iters, q) for q in range(n + 1)],
                                      dtype=torch.float64, device=dev)
                f_init = torch.tensor([bfgs_flops_init(n, q) for q in range(n + 1)], dtype=torch.float64,
                                      device=dev)
                r = run[sel].double()
                flops += float(((f_init[nq] + f_step[nq] * iters[sel].double()) * r).sum().item())
            del ids, order
            res[init]["bfgs_flops"] = flops
    del out, batch, scene
    peaks = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    L = res[main]
    bfgs_ms = L["kernel_ms"][fpt.K_BFGS] / steps
    roof = {"kernel": "bfgs_refill_kernel<n, Q> (orders 1-5, reflector/edge patterns)", "bound": "alu",
            "achieved": L["bfgs_flops"] / (bfgs_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
            "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz", "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    names = {fpt.K_BFGS: "bfgs", fpt.K_POLISH: "polish", fpt.K_BACKWARD: "backward", fpt.K_OTHER: "finalize",
             fpt.K_MLP: "mlp_infer_kernel (learned start)"}
    for r in res.values():
        r["kernel_ms_per_step"] = {names[k]: r["kernel_ms"][k] / steps for k in range(fpt.K_COUNT)}
        del r["kernel_ms"]
    return {"n_paths": N, "res": res, "roofline": roof, "main": main}


def run_city(args, world, rank, local_rank):
    """The ragged large batch: seeded orders 1-5 on a city, learned start; the plain start alongside
    (with --no-learned: the plain start alone, no network trained)."""
    import torch

    from paper_2510_16172_gb300 import build, fpt, warmstart

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ctx = fpt.Context(local_rank)
    learned = not args.no_learned
    dist = None
    if world > 1:
        import torch.distributed as dist
    train_s, hist = None, None
    if learned:
        t0 = time.perf_counter()
        X, T, G = warmstart.make_dataset(ctx)
        net, hist = warmstart.train(ctx, X, T, G, epochs=args.epochs)
        del X, T, G
        train_s = time.perf_counter() - t0
        net.attach()
    m = measure_city(ctx, dev, args, args.steps, args.warmup, learned, dist)
    L = m["res"][m["main"]]
    line = {"metric": METRIC, "value": L["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": L["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CITY_WORKLOAD if learned else CITY_WORKLOAD_PLAIN, "n_paths": m["n_paths"],
                       "init": "learned" if learned else "plain", "max_bfgs_iters": args.max_iters,
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
            "solved_per_step": L["solved_per_step"], "mean_bfgs_iters": L["mean_bfgs_iters"],
            "kernel_ms_per_step": L["kernel_ms_per_step"],
            "roofline": m["roofline"], "gpu_launches": L["launches"], "clocks": L["clocks"]}
    if learned:
        P = m["res"][0]
        line["plain_start"] = {"value": P["value"], "ms_per_step": P["ms_per_step"],
                               "solved_per_step": P["solved_per_step"], "mean_bfgs_iters": P["mean_bfgs_iters"],
                               "kernel_ms_per_step": P["kernel_ms_per_step"]}
        line["network"] = {"train_s": train_s, "train_loss_per_epoch": hist}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        from paper_2510_16172_gb300 import scenes

        sc = scenes.city(0, n_rx=16)
        per_pair = args.city_paths // (len(sc.tx) * len(sc.rx))
        rate, mm, dt, threads = oracle_rate(sc, m["n_paths"], 1, target_s=args.cpu_seconds,
                                            decode=lambda g: oracle.seeded_paths(sc, 5, per_pair, 1, 5, g))
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{mm} uniformly sampled paths of the batch, FP64 damped Newton + implicit "
                                          f"VJP, {dt:.1f} s on {threads} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fig2(args, world, rank, local_rank):
    """Sec. IV-A, Fig. 2 (our solver's side): mean point error against solver time.

    For diffraction-only (d = 1), reflection-only (d = 2) and mixed sequences of order n = 1..5 on
    random 10 m scenes (12 objects of one kind, or 8 planes + 4 edges), 1000 seeded paths per case are
    solved with exactly k BFGS steps (no polish) for k = 1..100, with one ('ours') or 64 ('ours-64')
    Eq. 6 rounds per step; diffractions also in the unified d = 2 form.  The error is the mean distance
    of the interaction points from the polished solution (stationarity residual <= 1e-5 m) over the
    paths that reach it; the time is the BFGS kernels' device time (CUDA events), for the 1000 paths
    and per path at 1,000,000 paths.
    """
    import numpy as np
    import torch

    from paper_2510_16172_gb300 import build, fpt, scenes

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ctx = fpt.Context(local_rank)
    kinds = {"d1": dict(n_quads=0, n_edges=12), "d2": dict(n_quads=12, n_edges=0),
             "mixed": dict(n_quads=8, n_edges=4)}
    ks = [1, 2, 3, 5, 8, 12, 20, 32, 50, 100]
    curves = []
    for kind, kw in kinds.items():
        sc = scenes.tiny_scene(3, **kw)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        for n in range(1, 6):
            small = fpt.Batch.seeded(ctx, scene, 100 + n, 1000, n, n)
            big = fpt.Batch.seeded(ctx, scene, 200 + n, 1_000_000, n, n)
            ref = fpt.solve(ctx, scene, small, fpt.default_params(max_iters=100, polish=2))
            ok = (ref["status"] & fpt.ST_SOLVED) > 0
            Xr = ref["X"][ok].double()
            variants = [("ours", 1, 2), ("ours-64", 64, 2)]
            if kind == "d1":
                variants += [("ours d=2", 1, 0), ("ours-64 d=2", 64, 0)]
            for name, fp, spec in variants:
                pts = []
                for k in ks:
                    p = fpt.default_params(max_iters=k, fixed_iters=1, fp_iters=fp, polish=0, specialize=spec)
                    row = {"k": k}
                    for label, batch in (("small", small), ("big", big)):
                        out = fpt.alloc_outputs(ctx, batch, with_X=label == "small")
                        fpt.solve(ctx, scene, batch, p, out)  # warm-up
                        ctx.sync()
                        fpt.profile_enable(ctx, True)
                        fpt.profile_read(ctx, reset=True)
                        reps = 5 if label == "small" else 2
                        for _ in range(reps):
                            fpt.solve(ctx, scene, batch, p, out)
                        kms, _ = fpt.profile_read(ctx, reset=True)
                        fpt.profile_enable(ctx, False)
                        if label == "small":
                            row["ms_1000_paths"] = kms[fpt.K_BFGS] / reps
                            err = (out["X"][ok].double() - Xr).norm(dim=2)[:, :n].mean(dim=1)
                            fin = torch.isfinite(err)
                            row["mean_err_m"] = float(err[fin].mean())
                            row["nonfinite_paths"] = int((~fin).sum())
                        else:
                            row["ns_per_path_at_1M"] = kms[fpt.K_BFGS] / reps * 1e6 / batch.n_paths
                        del out
                    pts.append(row)
                curves.append({"kind": kind, "n": n, "solver": name, "paths_with_reference": int(ok.sum()),
                               "points": pts})
    line = {"metric": "mean interaction-point error vs BFGS time (Fig. 2, our solver)", "unit": "m",
            "config": {"workload": "1000 seeded paths per (kind, n) on a random 10 m scene; k = 1..100 fixed BFGS "
                                   "steps, no polish; reference = polished solution (residual <= 1e-5 m)"},
            "curves": curves}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fig3(args, world, rank, local_rank):
    """Sec. IV-B, Fig. 3: time of the gradient of the path lengths, implicit vs through the iterations.

    On a random 10 m scene (8 planes + 4 edges), seeded sequences of order n = 1..10: the gradient of
    sum L with respect to TX, RX and every vertex after k = 16 or 128 solver steps with 1 or 64 Eq. 6
    rounds per step (d = 2).  'implicit' = fpt_solve_grad (k fixed steps, the Newton polish, the
    implicit backward of Sec. III-D); 'ad' = fpt_backward_unrolled (the same k steps taped, then
    reverse mode through every step).  Device time by CUDA events on the launching stream, for 1000
    paths (the paper's batch) and per path at 1,000,000 paths.
    """
    import torch

    from paper_2510_16172_gb300 import build, fpt, scenes

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ctx = fpt.Context(local_rank)
    sc = scenes.tiny_scene(3, n_quads=8, n_edges=4)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    rows = []
    for n in range(1, 11):
        for label, per_pair in (("1000", 1000), ("1M", 1_000_000)):
            batch = fpt.Batch.seeded(ctx, scene, 300 + n, per_pair, n, n)
            N = batch.n_paths
            ones = torch.ones(N, dtype=torch.float32, device=dev)
            out = fpt.alloc_outputs(ctx, batch)
            for k in (16, 128):
                for fp in (1, 64):
                    p = fpt.default_params(max_iters=k, fixed_iters=1, fp_iters=fp)
                    reps = 10 if label == "1000" else 2
                    t_imp = timed(lambda: fpt.solve_grad(ctx, scene, batch, p, dL=ones, out=out), reps)
                    t_ad = timed(lambda: fpt.backward_unrolled(ctx, scene, batch, k, fp, dL=ones), reps)
                    row = {"n": n, "paths": N, "k": k, "fp_iters": fp, "implicit_ms": t_imp, "ad_ms": t_ad,
                           "ad_over_implicit": t_ad / t_imp}
                    if label == "1000":
                        # how far the gradient through the k FP32 steps is from the implicit one
                        _, (_, _, gi) = fpt.solve_grad(ctx, scene, batch, p, dL=ones, out=out)
                        _, _, ga, _, _ = fpt.backward_unrolled(ctx, scene, batch, k, fp, dL=ones)
                        row["ad_vs_implicit_rel_diff"] = float((ga - gi).norm() / gi.norm())
                    rows.append(row)
                    if rank == 0:
                        print(json.dumps(row), file=sys.stderr, flush=True)
            del out, ones
    line = {"metric": "gradient time of sum L, implicit vs AD through the iterations (Fig. 3)", "unit": "ms",
            "config": {"workload": "seeded order-n sequences on a random 10 m scene (8 planes + 4 edges), "
                                   "1000 paths and 1,000,000 paths per n; k fixed solver steps, fp Eq. 6 rounds"},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


# algorithmic work of one training sample of the 64-256-256-256-16 network: the forward pass (2 flop per
# multiply-add), the back-propagation to the inputs of layers 2-4 and the weight gradients of all four
MLP_MACS = 64 * 256 + 2 * 256 * 256 + 256 * 16
MLP_TRAIN_FLOP = 2 * MLP_MACS + 2 * (MLP_MACS - 64 * 256) + 2 * MLP_MACS


def run_train(args, world, rank, local_rank):
    """Training throughput of the warm-start network (fpt_mlp_train: seeded shuffles, forward, loss,
    backward and Adam on the tensor cores) on the solver's solutions of 10 random 10 m scenes, per batch
    size: one timed epoch after one untimed one, CUDA events on the context's stream."""
    import torch

    from paper_2510_16172_gb300 import build, fpt, warmstart

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ctx = fpt.Context(local_rank)
    X, T, G = warmstart.make_dataset(ctx, seeds=tuple(range(1000, 1010)), per_pair=100_000)
    rows = []
    stream = torch.cuda.current_stream(dev)
    for batch in (int(v) for v in args.train_batches.split(",")):
        net = fpt.Mlp(ctx, 0, warmstart.LENGTH_SCALE)
        net.train(X, T, G, max(1, args.warmup), batch=batch, lr=1e-3, lr_decay=1.0, seed=1)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.train(X, T, G, args.steps, batch=batch, lr=1e-3, lr_decay=1.0, seed=2)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        samples = (X.shape[0] // batch) * batch * args.steps
        rows.append({"batch": batch, "epochs": args.steps, "ms": ms, "samples": samples,
                     "tflops": MLP_TRAIN_FLOP * samples / (ms * 1e-3) / 1e12})
        net.close()
    peaks = measured_peaks()
    line = {"metric": "warm-start network training throughput (fpt_mlp_train)", "unit": "TFLOP/s",
            "config": {"workload": f"{X.shape[0]} samples (solver solutions of 10 random 10 m scenes), "
                                   "64-256-256-256-16 GELU, BF16 operands, FP32 accumulation and Adam",
                       "flop_per_sample": MLP_TRAIN_FLOP},
            "peak_bf16_sustained_tflops": peaks.get("bf16_tflops_sustained"), "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e(args, sc, ctx, dev, torch, fpt):
    """Same metric through the public API: host scene/endpoints in, host parameters/lengths/status/gradients out.

    Every step uploads its scene and endpoints from pinned host memory, builds the batch, runs
    fpt_solve_grad and copies the solved parameters T (the interaction points are x_i = A_i t_i + b_i),
    the lengths, the status and the gradients back to pinned host memory.  The device
    outputs are double-buffered: step k's device-to-host copy runs on a copy stream while step k + 1
    computes (a serving loop's pipeline); the timed region ends when the last step's results are on
    the host.  Scenes and batches are released, and the solved paths counted on the host, after the
    timed steps (a release synchronises the device).
    """
    types = torch.from_numpy(sc.types).pin_memory()
    verts = torch.from_numpy(sc.verts).pin_memory()
    tx = torch.from_numpy(sc.tx).pin_memory()
    rx = torch.from_numpy(sc.rx).pin_memory()
    alphabet = sc.alphabet
    N = 32 ** 3 * len(sc.rx)
    # half the device-timed steps (at most 20): the drain of the last step's copies (about 1 GB over the
    # host link) is part of the timed region, and a longer run shows the pipeline's steady state
    steps = max(3, min(20, args.steps // 2))
    total = args.warmup + steps
    L_h = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(2)]
    T_h = [torch.empty((N, 3, 2), dtype=torch.float32).pin_memory() for _ in range(2)]
    st_h = [torch.empty(N, dtype=torch.uint8).pin_memory() for _ in range(total)]
    g_h = [(torch.empty((len(sc.tx), 3), dtype=torch.float32).pin_memory(),
            torch.empty((len(sc.rx), 3), dtype=torch.float32).pin_memory(),
            torch.empty((len(sc.types), 3, 3), dtype=torch.float32).pin_memory()) for _ in range(2)]
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    params = fpt.default_params(max_iters=args.max_iters, kink_stop=args.kink_stop)
    h2d = types.numel() + verts.numel() * 8 + tx.numel() * 8 + rx.numel() * 8 + alphabet.size * 4
    d2h = T_h[0].numel() * 4 + N * 4 + N + sum(t.numel() * 4 for t in g_h[0])
    copy_stream = torch.cuda.Stream(dev)
    outs = [None, None]
    grads = [None, None]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    keep = []
    t0 = None
    for k in range(total):
        b = k % 2
        if k >= 2:
            copied[b].synchronize()  # step k - 2's results are on the host: its buffers are free
        if k == args.warmup:
            torch.cuda.synchronize(dev)
            copy_stream.synchronize()
            t0 = time.perf_counter()
        scene = fpt.Scene(ctx, types.numpy(), verts.numpy(), tx.numpy(), rx.numpy())
        batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, alphabet)
        keep.append((scene, batch))
        if outs[b] is None:
            outs[b] = fpt.alloc_outputs(ctx, batch, with_X=False, with_rho=False, with_iters=False)
            grads[b] = tuple(torch.empty(t.shape, dtype=torch.float32, device=dev) for t in g_h[b])
        fpt.solve_grad(ctx, scene, batch, params, dL_status_mask=mask, out=outs[b], grads=grads[b])
        done[b].record(ctx.stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(done[b])
            T_h[b].copy_(outs[b]["T"], non_blocking=True)
            L_h[b].copy_(outs[b]["L"], non_blocking=True)
            st_h[k].copy_(outs[b]["status"], non_blocking=True)
            for h, d in zip(g_h[b], grads[b]):
                h.copy_(d, non_blocking=True)
            copied[b].record(copy_stream)
    copy_stream.synchronize()
    dt = time.perf_counter() - t0
    solved = sum(int(((st_h[k].numpy() & fpt.ST_SOLVED) > 0).sum()) for k in range(args.warmup, total))
    for scene, batch in keep:
        batch.close()
        scene.close()
    return {"value": solved / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * dt / steps, "pipelined": "outputs double-buffered; copies overlap the next step",
            "d2h": "T [N,3,2] (the solved parameters), L [N], status [N] and the TX/RX/vertex gradients, every step",
            "l2": "not flushed: every step writes ~1 GB of outputs (T, L, status), far more than L2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--max-iters", type=int, default=32,
                    help="BFGS step cap (32 keeps 99.9 %% of the canyon solves that 40 steps give)")
    ap.add_argument("--kink-stop", type=float, default=0.01,
                    help="urban canyon: stop a path whose segment falls below this many metres before converging "
                         "(1 cm, 1/500 of the smallest facade; loses 96 of 20.5 M solves against 0.1 mm)")
    ap.add_argument("--rx-grid", type=int, default=32, help="RX grid side (32 = the 33.5M-path workload)")
    ap.add_argument("--no-learned", action="store_true",
                    help="canyon: skip the learned-vs-plain start comparison; city: the plain start alone")
    ap.add_argument("--workload", choices=["canyon", "city", "fig2", "fig3", "train"], default="canyon",
                    help="canyon: the 33.5M-path urban canyon (default); city: the 100M-path ragged city batch; "
                         "fig2: point error against solver time by iteration budget; fig3: gradient time, implicit vs AD "
                         "through the iterations; train: warm-start network training throughput (--steps epochs)")
    ap.add_argument("--city-paths", type=int, default=100_000_000)
    ap.add_argument("--city-steps", type=int, default=5, help="timed steps of the city leg of the default run")
    ap.add_argument("--no-city", action="store_true", help="canyon run: skip the ragged city leg")
    ap.add_argument("--epochs", type=int, default=6, help="training epochs of the warm-start network")
    ap.add_argument("--train-batches", default="8192,16384,65536", help="train workload: batch sizes to time")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "city":
        run_city(args, world, rank, local_rank)
    elif args.workload == "fig2":
        run_fig2(args, world, rank, local_rank)
    elif args.workload == "fig3":
        run_fig3(args, world, rank, local_rank)
    elif args.workload == "train":
        run_train(args, world, rank, local_rank)
    else:
        run_ours(args, world, rank, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
