"""Benchmark of the CTA hot path on GB300 (one JSON line on stdout).

Workload (one "step"): one CTA solve (Alg. 1.1, H = A Aᵀ, ping-pong t-cycling
up to t = 5, true residual every 40 steps) from x = 0 toward the 1e-8 relative
residual target on the 2D convection-diffusion 5-point stencil on a 1000 x 1000
grid (n = 1e6, 4,996,000 nonzeros, CSR, FP64, b = A·1), capped at
ITERS_PER_STEP F_t applications. The system needs far more iterations than
the cap to reach 1e-8 (kappa(AAᵀ) ~ 1e11), so every step runs the full cap and
the metric is the F_t iteration rate; the residual reached is reported.

value      : F_t iterations per second over the K timed steps (device events),
             inputs resident in HBM, L2 flushed between steps.
e2e        : same metric through the one-shot C ABI call with host buffers
             (pinned): A and b copied in, plan built (device transpose), solve,
             x and the residual history copied out, all inside the timed region.
roofline   : the fused step kernel (one cooperative launch per F_t step: the 2t products
             with Aᵀ and A on the diagonal form of the stencil, the moments, the
             auxiliary solve and the x, r update), timed with CUDA events around every
             launch inside a profiled solve of the same workload, as HBM bandwidth on the
             survey's algorithmic bytes of an F_t step (CSR products, 559.7 MB at the
             mean order t = 3) against the measured copy peak. Beside it: the whole solve
             step at the measured F_t rate ("step", gated residual launch and launch gaps
             included), the DRAM bytes ncu counted ("dram"), the bytes the diagonal form
             needs ("format") and the FP64 FMA rate against the nominal 1.25 TFLOP/s
             ("fp64").
cpu_baseline: the FP64 numpy oracle on the same workload, a bounded sample of
             CPU_SAMPLE_ITERS iterations, on all host cores (numpy's BLAS pool) and
             on one thread.

--impl reference times the oracle itself (the CPU statement of the method) on
the same config, each step a bounded sample of REF_ITERS_PER_STEP iterations.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = 1000
ITERS_PER_STEP = 1000
TOL = 1e-8
CPU_SAMPLE_ITERS = 40
REF_ITERS_PER_STEP = 4
METRIC = "TA/CTA iterations/sec and time-to-1e-8 rel. residual; achieved HBM GB/s vs peak"
UNIT = "CTA iterations/s"
WORKLOAD = "cta_fp64_convdiff_5pt_1000x1000"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# GB300 FP64 rate (CUDA cores), the nominal figure of the platform's data sheet: 1.25
# TFLOP/s, i.e. 152 SMs x ~2 FP64 FMA per SM-cycle x 2.07 GHz x 2 flops (an FMA microbenchmark
# on the box measured 1.91 FMA/clk/SM, 1.20 TFLOP/s)
FP64_TFLOPS_NOMINAL = 1.25


def kernel_source_hash():
    """sha256 of the dominant kernel's source: the fused step (chain.cu), the row-tile
    stages and copy issue it uses (rowtiles.cuh), the mbarrier helpers, the step decision,
    finishers and solve it calls (aux_step.cuh, finish.cuh, hankel.cuh) and the layout
    constants (internal.h), comment lines dropped."""
    csrc = os.path.join(ROOT, "paper_2304_12168_gb300", "csrc")
    code = ""
    for f in ("chain.cu", "rowtiles.cuh", "mbarrier.cuh", "aux_step.cuh", "finish.cuh", "hankel.cuh",
              "internal.h"):
        src = open(os.path.join(csrc, f)).read()
        code += "\n".join(l for l in src.splitlines() if not l.strip().startswith("//"))
    return hashlib.sha256(code.encode()).hexdigest()


def traffic_record():
    """DRAM bytes per F_t step of the fused step kernel (a captured launch's bytes over its
    steps, at the cycle's mean order t = 3) from the committed ncu capture, if the kernel's
    source is unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if kernel_source_hash() != rec.get("kernel_source_sha256"):
            return None
        return float(rec["dram_bytes_per_step"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def problem():
    import gen
    return gen.convdiff_stencil(GRID)


def aggregate(dist, device, local_ms: float, local_units: int):
    """Whole-job figures over ranks: the slowest rank's time and the sum of the
    units (F_t iterations) all ranks processed. With one process, the local values."""
    if dist is None:
        return local_ms, local_units
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def timed_solve(plan, b, stream, **kw):
    """One plan CTA solve timed with CUDA events on the launching stream (ms, x, info)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    x, _, info = plan.cta(b, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), x, info


def extra_workloads(tacta, dev, stream, plan_stencil, b_stencil, steps):
    """The other configurations, each timed with device events (inputs resident): the
    mixed-precision CTA rate and the TA rate on the benchmark stencil, time to 1e-8 on the
    LP-like rectangular system (FP64 and mixed), the Clement rate, the batched dense
    workload, the dense 256 x 256 systems and the differentiable 2000 x 8000 solve."""
    import gen
    import numpy as np
    import torch
    out = {}
    opts = dict(tol=TOL, tol_normal=0.0, max_iter=ITERS_PER_STEP, precision=tacta.PRECISION_MIXED)
    for _ in range(2):
        plan_stencil.cta(b_stencil, **opts)
    ms, its = 0.0, 0
    for _ in range(steps):
        t, _, info = timed_solve(plan_stencil, b_stencil, stream, **opts)
        ms += t
        its += info["iters"]
    # TA (Alg. 2.2) on the same stencil: iterations per second over a fixed budget
    kw = dict(tol=TOL, tol_normal=0.0, max_iter=ITERS_PER_STEP)
    plan_stencil.ta(b_stencil, **kw)
    ta_ms, ta_its = 0.0, 0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, _, info = plan_stencil.ta(b_stencil, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ta_ms += e0.elapsed_time(e1)
        ta_its += info["iters"]
    # the same FP64 CTA solve with one launch per product (fused_chain = 0), for comparison
    kw0 = dict(tol=TOL, tol_normal=0.0, max_iter=ITERS_PER_STEP, fused_chain=0)
    plan_stencil.cta(b_stencil, **kw0)
    u_ms, u_its = 0.0, 0
    for _ in range(steps):
        t, _, info0 = timed_solve(plan_stencil, b_stencil, stream, **kw0)
        u_ms += t
        u_its += info0["iters"]
    out["cta_fp64_per_product_launches"] = {"value": u_its / (u_ms * 1e-3), "unit": UNIT, "steps": steps,
                                            "iters_per_step": ITERS_PER_STEP, "launches_per_step": info0["launches"]}
    out["ta_fp64_convdiff_1000x1000"] = {"value": ta_its / (ta_ms * 1e-3), "unit": "TA iterations/s",
                                         "steps": steps, "iters_per_step": ITERS_PER_STEP,
                                         "rel_res_after_step": info["rel_res"]}
    out["cta_mixed_convdiff_1000x1000"] = {
        "value": its / (ms * 1e-3), "unit": UNIT, "steps": steps, "iters_per_step": ITERS_PER_STEP,
        "dtype": "f32 chain (values, vectors, products), f64 moments reduction, centering solve, "
                 "stop tests, and residual refinement every 40 steps or once the f32 residual fell by 1e-3"}
    # LP-like rectangular min-norm system, 10,000 x 1,000,000, 31.6M nonzeros: time to 1e-8
    p = gen.lp_rect()
    A = tacta.CSR(torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colidx).to(dev),
                  torch.from_numpy(p.vals).to(dev), (p.m, p.n))
    b = torch.from_numpy(p.b).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = tacta.Plan(A)
    plan_s = time.perf_counter() - t0
    res = {"workload": "lp_rect_10000x1000000 (30 nnz per column, 500 duplicated scaled rows)",
           "nnz": p.nnz, "plan_build_s": plan_s, "tol": TOL}
    xs = {}
    for name, prec in (("fp64", tacta.PRECISION_FP64), ("mixed", tacta.PRECISION_MIXED)):
        kw = dict(tol=TOL, tol_normal=0.0, max_iter=5000, precision=prec)
        plan.cta(b, **kw)                                   # warm (graph capture, FP32 copies)
        best = None
        for _ in range(3):
            t, x, info = timed_solve(plan, b, stream, **kw)
            best = t if best is None else min(best, t)
        xs[name] = x.double()
        res[name] = {"time_to_tol_ms": best, "iters": info["iters"], "rel_res": info["rel_res"],
                     "reason": info["reason_name"]}
    res["mixed_vs_fp64_rel_x_diff"] = float(torch.linalg.norm(xs["mixed"] - xs["fp64"]) /
                                            torch.linalg.norm(xs["fp64"]))
    res["speedup_mixed_over_fp64"] = res["fp64"]["time_to_tol_ms"] / res["mixed"]["time_to_tol_ms"]
    out["time_to_1e-8_lp_rect"] = res
    plan.close()
    # Clement n = 100001 (singular, b in range): F_t rate over a fixed budget
    q = gen.clement(100001)
    Aq = tacta.CSR(torch.from_numpy(q.rowptr).to(dev), torch.from_numpy(q.colidx).to(dev),
                   torch.from_numpy(q.vals).to(dev), (q.m, q.n))
    bq = torch.from_numpy(q.b).to(dev)
    plan = tacta.Plan(Aq)
    kw = dict(tol=TOL, tol_normal=0.0, max_iter=20000)
    plan.cta(bq, **kw)
    t, x, info = timed_solve(plan, bq, stream, **kw)
    out["cta_fp64_clement_100001"] = {"value": info["iters"] / (t * 1e-3), "unit": UNIT,
                                      "iters": info["iters"], "rel_res": info["rel_res"]}
    plan.close()
    out["batched_dense_4096"] = batched_workload(tacta, dev, stream)
    out["dense_256"] = dense_workload(tacta, dev, stream)
    out["autograd_2000x8000"] = autograd_workload(tacta, dev, stream)
    out["dense_2000x8000"] = dense_minnorm_workload(tacta, dev, stream)
    return out


def dense_minnorm_workload(tacta, dev, stream):
    """Dense full-row-rank 2000 x 8000 N(0,1) min-norm system (b = A x0): CTA time to 1e-8
    in FP64 and in mixed precision (FP32 copies of A and Aᵀ), and one profiled solve per
    precision for the dense products' bandwidth: algorithmic bytes per product (the values
    once, x read and y written once) over the product's event-timed duration, against the
    measured HBM peak."""
    import numpy as np
    import torch
    rng = np.random.default_rng(9)
    D = rng.standard_normal((2000, 8000))
    bh = D @ rng.standard_normal(8000)
    A = torch.from_numpy(D).to(dev)
    b = torch.from_numpy(bh).to(dev)
    plan = tacta.Plan(A)
    peak, peak_src = peaks()
    res = {"workload": "dense 2000 x 8000 N(0,1), b = A x0, CTA to 1e-8", "tol": TOL,
           "hbm_peak_gbs": peak, "hbm_peak_source": peak_src}
    xs = {}
    for name, prec in (("fp64", tacta.PRECISION_FP64), ("mixed", tacta.PRECISION_MIXED)):
        kw = dict(tol=TOL, tol_normal=0.0, max_iter=20000, precision=prec)
        plan.cta(b, **kw)
        best = None
        for _ in range(3):
            t, x, info = timed_solve(plan, b, stream, **kw)
            best = t if best is None else min(best, t)
        xs[name] = x.double()
        # profiled to exactly the steps the solve took: no launch runs past the stop, and the
        # products run back to back (launch latency hidden) as in the solve
        kwp = dict(kw, max_iter=info["iters"])
        _, _, prof = plan.cta(b, profile=1, **kwp)
        gbs = prof["spmv_bytes"] / (prof["spmv_ms"] * 1e-3) / 1e9 if prof["spmv_ms"] > 0 else None
        res[name] = {"time_to_tol_ms": best, "iters": info["iters"], "rel_res": info["rel_res"],
                     "reason": info["reason_name"], "products_profiled": prof["spmv_count"],
                     "us_per_product": 1e3 * prof["spmv_ms"] / max(prof["spmv_count"], 1),
                     "product_gbs": gbs, "product_hbm_frac": gbs / peak if gbs else None}
    res["mixed_vs_fp64_rel_x_diff"] = float(torch.linalg.norm(xs["mixed"] - xs["fp64"]) /
                                            torch.linalg.norm(xs["fp64"]))
    res["speedup_mixed_over_fp64"] = res["fp64"]["time_to_tol_ms"] / res["mixed"]["time_to_tol_ms"]
    plan.close()
    return res


def dense_workload(tacta, dev, stream):
    """Dense 256 x 256 N(0,1) (seed 0) and its rank-128 variant U Vᵀ: CTA and TA to a
    relative residual of 1e-10 (at most 20000 steps), inputs resident, device events."""
    import gen
    import torch
    res = {}
    for name, p in (("full_rank", gen.dense_gaussian(256, 256, seed=0)),
                    ("rank_128", gen.dense_low_rank(256, 256, 128, seed=1))):
        A = torch.from_numpy(p.dense).to(dev)
        b = torch.from_numpy(p.b).to(dev)
        plan = tacta.Plan(A)
        for alg, extra in (("cta", {}), ("ta", {}), ("cta_mixed", {"precision": tacta.PRECISION_MIXED})):
            kw = dict(tol=1e-10, tol_normal=0.0, max_iter=20000, **extra)
            fn = getattr(plan, alg.split("_")[0])
            fn(b, **kw)
            t, (x, _, info) = timed(lambda: fn(b, **kw), stream)
            res[f"{name}_{alg}"] = {"time_to_tol_ms": t, "iters": info["iters"],
                                    "it_per_s": info["iters"] / (t * 1e-3), "rel_res": info["rel_res"],
                                    "reason": info["reason_name"]}
        plan.close()
    return res


def autograd_workload(tacta, dev, stream):
    """Differentiable min-norm solve on a dense 2000 x 8000 N(0,1) system, L = ||x - x_t||²:
    forward + backward time and dL/db against the closed form (A Aᵀ)^{-1} A g (numpy)."""
    import numpy as np
    import torch
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    rng = np.random.default_rng(5)
    D = rng.standard_normal((2000, 8000))
    bh = rng.standard_normal(2000)
    xt = torch.from_numpy(rng.standard_normal(8000)).to(dev)
    opts = dict(tol=1e-12, tol_normal=0.0, max_iter=20000)

    def step():
        A = torch.tensor(D, device=dev, requires_grad=True)
        b = torch.tensor(bh, device=dev, requires_grad=True)
        x = cta_solve_autograd(A, b, **opts)
        ((x - xt) ** 2).sum().backward()
        return x, b.grad
    step()
    t, (x, gb) = timed(step, stream)
    G = D @ D.T
    xs = D.T @ np.linalg.solve(G, bh)
    lam = np.linalg.solve(G, D @ (2 * (xs - xt.cpu().numpy())))
    return {"fwd_bwd_ms": t, "tol": 1e-12,
            "rel_err_x": float(np.linalg.norm(x.detach().cpu().numpy() - xs) / np.linalg.norm(xs)),
            "rel_err_dL_db": float(np.linalg.norm(gb.cpu().numpy() - lam) / np.linalg.norm(lam))}


def batched_workload(tacta, dev, stream):
    """4096 uneven dense systems (m in [32, 512], n in [m/2, 2m], 10% rank m/2) to 1e-8,
    per storage precision: the longest systems on thread-block clusters and the rest on
    single blocks of one persistent launch (launch shape and ring stage autotuned after a
    first full solve, whose step counts and measured times set the tuner's makespan
    model, the queue order and the clusters' share; two warm solves refit the planner's
    per-step cluster overhead), against the single-system FP64 path (Plan per system)
    timed on an evenly spaced sample."""
    import gen
    import numpy as np
    import torch
    B0 = gen.dense_batch(4096, seed=7)
    b = torch.from_numpy(B0.packed_b()).to(dev)
    mats = [torch.from_numpy(a).to(dev) for a in B0.mats]
    kw = dict(tol=TOL, tol_normal=0.0, max_iter=20000)
    res = {"workload": "4096 dense systems, m ~ U[32,512], n ~ U[m/2,2m], 10% rank m/2, b = A x*",
           "entries": int(sum(a.size for a in B0.mats)), "tol": TOL, "max_iter_per_system": 20000}
    for name, st in (("fp64", tacta.BATCH_FP64), ("fp32", tacta.BATCH_FP32), ("bf16", tacta.BATCH_BF16)):
        B = tacta.Batch(mats, storage=st)
        B.cta(b, **kw)                     # a first full solve: step counts and queue order
        cfg, _ = B.tune(b, tol=TOL, tol_normal=0.0, max_iter=100)
        for _ in range(2):   # warm: the planner refits its cluster overhead; graph capture
            B.cta(b, **kw)
        plan = B.wide_plan(**kw)                             # the share the timed solve uses
        t, (x, iters, rel, reason) = timed(lambda: B.cta(b, **kw), stream)
        conv = reason == 1
        shape = tacta.Batch.configs()[cfg]
        blocks = min(B0.count, torch.cuda.get_device_properties(dev).multi_processor_count * shape[1])
        res[name] = {"time_ms": t, "converged": int(conv.sum()), "maxiter": int((reason == 3).sum()),
                     "system_iters": int(iters.sum()), "system_iters_per_s": float(iters.sum() / (t * 1e-3)),
                     "max_rel_res_converged": float(rel[conv].max()) if conv.any() else None,
                     "config": shape,
                     "clusters": {"systems": plan[0], "blocks_per_cluster": plan[1], "clusters": plan[2],
                                  "predicted_ms": plan[3]},
                     "completion": completion_profile(*B.timeline(), blocks, clustered=plan[0] > 0)}
        B.close()
    # single-system FP64 path on a sample, extrapolated to the batch
    idx = np.linspace(0, B0.count - 1, 24).astype(int)
    tot, its = 0.0, 0
    for s_ in idx:
        plan = tacta.Plan(mats[s_])
        plan.cta(torch.from_numpy(B0.bs[s_]).to(dev), **kw)
        t, (x, _, info) = timed(lambda: plan.cta(torch.from_numpy(B0.bs[s_]).to(dev), **kw), stream)
        tot += t
        its += info["iters"]
        plan.close()
    res["plan_fp64_per_system_sample"] = {"systems": len(idx), "mean_ms": tot / len(idx),
                                          "extrapolated_batch_ms": tot / len(idx) * B0.count,
                                          "system_iters_per_s": its / (tot * 1e-3)}
    for name in ("fp64", "fp32", "bf16"):
        res[name]["speedup_over_plan_fp64"] = res["plan_fp64_per_system_sample"]["extrapolated_batch_ms"] / \
            res[name]["time_ms"]
    return res


def batch_sample():
    """152 systems of the batched workload's distribution (seed 3), BF16 storage, each
    solved for at most 300 steps (tol 1e-8) with the fused-pass kernel on CUDA cores and
    then on the tensor cores, direct launches (the case profiled in profiles/)."""
    import gen
    import torch
    import paper_2304_12168_gb300 as tacta
    tacta.load_library()
    torch.cuda.set_device(0)
    B0 = gen.dense_batch(152, seed=3)
    b = B0.packed_b()
    for cfg in (5, tacta.Batch.tensor_core_configs()[0]):   # the default 32 KB / 40 KB ring stages
        B = tacta.Batch(B0.mats, storage=tacta.BATCH_BF16)
        B.set_config(cfg)
        x, it, rel, reason = B.cta(b, tol=TOL, tol_normal=0.0, max_iter=300, use_graph=0)
        tb, te = B.timeline()
        print(json.dumps({"config": cfg, "shape": tacta.Batch.configs()[cfg], "system_steps": int(it.sum()),
                          "span_ms": float((te.max() - tb.min()) * 1e-6)}))
        B.close()


def completion_profile(tb, te, blocks, clustered=False):
    """The batch's completion profile from the per-system device clocks of one solve: when
    50/90/99/100 % of the systems were done (ms after the first was taken), the longest
    system's time, and -- when single blocks took every system -- the share of the launch's
    block-time spent on systems and the mean share of blocks still busy after the 90 % mark
    (the tail). (A system on a cluster holds several SMs: those shares are then omitted.)"""
    import numpy as np
    t0 = int(tb.min())
    done = np.sort((te - t0) * 1e-6)
    span = float(done[-1])
    pct = {f"p{q}_ms": float(done[min(len(done) - 1, int(np.ceil(q / 100 * len(done))) - 1)])
           for q in (50, 90, 99, 100)}
    busy = float(np.sum(te - tb)) * 1e-6
    t90 = pct["p90_ms"]
    beg, end = (tb - t0) * 1e-6, (te - t0) * 1e-6
    tail = float(np.sum(np.clip(end, t90, None) - np.clip(beg, t90, None)))
    out = dict(pct, longest_system_ms=float(((te - tb) * 1e-6).max()))
    if not clustered:
        out.update(blocks=int(blocks), busy_frac=busy / (blocks * span) if span > 0 else None,
                   tail_busy_frac=tail / (blocks * (span - t90)) if span > t90 else None)
    return out


def timed(fn, stream):
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    r = fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e), r


def cpu_baseline(p, iters):
    import oracle
    A = oracle.make_operator(p)
    t0 = time.perf_counter()
    r = oracle.cta_solve(A, p.b, tol=TOL, tol_normal=0.0, max_iter=iters)
    dt = time.perf_counter() - t0
    return r.iters / dt, dt, r


def host_cores():
    """Cores this process may run on (the GPU machine's host cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_ORACLE_CHILD = """
import json, sys, time
sys.path.insert(0, {root!r})
import gen, oracle
p = gen.convdiff_stencil({grid})
A = oracle.make_operator(p)
t0 = time.perf_counter()
r = oracle.cta_solve(A, p.b, tol={tol!r}, tol_normal=0.0, max_iter={iters})
dt = time.perf_counter() - t0
print(json.dumps({{"iters": int(r.iters), "seconds": dt}}))
"""


def oracle_rate(threads, iters):
    """The oracle as it stands on the same workload (first `iters` F_t steps of the solve) in
    a fresh process whose BLAS / OpenMP pools have `threads` threads. numpy's vector
    operations (dots, norms, axpys) use that pool; scipy's CSR products run on one thread
    whatever the setting, so the all-core figure shows how far the oracle as written can
    use the host. Returns (F_t per second, seconds) or None if the child failed."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    code = _ORACLE_CHILD.format(root=ROOT, grid=GRID, tol=TOL, iters=iters)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600, check=True).stdout
        d = json.loads(out.strip().splitlines()[-1])
        return d["iters"] / d["seconds"], d["seconds"]
    except Exception:
        return None


def fpt_schedule(k, t_max=5):
    """t of F_t step k under the ping-pong cycle 1, 2, .., t_max, .., 2, 1, 2, .."""
    period = 2 * t_max - 2
    j = k % period
    return j + 1 if j < t_max else 2 * t_max - 1 - j


def survey_bytes_per_product(m, n, nnz):
    """Algorithmic bytes of one CSR product with A (m x n, FP64 values, int32 indices):
    values and column indices 12 nnz, row offsets 4 (m + 1), x read once 8 n, y written
    once 8 m."""
    return 12.0 * nnz + 4.0 * (m + 1) + 8.0 * n + 8.0 * m


def survey_bytes_per_fpt(m, n, nnz, t):
    """Algorithmic bytes of one CTA F_t step of order t, unfused: t products with Aᵀ and t
    with A (CSR), the chain's vectors read and written once per product, and the update
    reading t z's, t u's and x, r and writing x, r: t (B_A + B_Aᵀ) + 8 t (m + 2 n + m) +
    8 (t + 2)(n + m)."""
    ba = 12.0 * nnz + 4.0 * (m + 1)
    bat = 12.0 * nnz + 4.0 * (n + 1)
    return t * (ba + bat) + 8.0 * t * (m + 2 * n + m) + 8.0 * (t + 2) * (n + m)


def run_reference(args):
    """The oracle as it stands, on the host cores, on this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = problem()
    for _ in range(args.warmup):
        cpu_baseline(p, REF_ITERS_PER_STEP)
    times = []
    for _ in range(args.steps):
        _, dt, r = cpu_baseline(p, REF_ITERS_PER_STEP)
        times.append(dt)
    total = sum(times)
    value = args.steps * REF_ITERS_PER_STEP / total
    sample = f"first {REF_ITERS_PER_STEP} F_t steps of the solve per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{GRID}x{GRID}", "n": p.n, "nnz": p.nnz,
                       "iters_per_step": REF_ITERS_PER_STEP, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": sample + " (numpy's BLAS pool at its default, all host cores; "
                                                "scipy's CSR products on one thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tacta", choices=["tacta", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--iters", type=int, default=ITERS_PER_STEP,
                    help="F_t iterations per step (default %(default)s; smaller for profiler runs)")
    ap.add_argument("--batch-sample", action="store_true",
                    help="only run a 152-system sample of the batched workload (BF16 storage, the CUDA-core and "
                         "the tensor-core launch configurations, 300 steps each): the profiler's case")
    ap.add_argument("--no-graph", action="store_true",
                    help="direct launches instead of the solve's graph (profilers cannot replay kernels of "
                         "a graph with a conditional node)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_sample:
        return batch_sample()

    import numpy as np
    import torch
    import paper_2304_12168_gb300 as tacta

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    tacta.load_library()

    p = problem()
    A = tacta.CSR(torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colidx).to(dev),
                  torch.from_numpy(p.vals).to(dev), (p.m, p.n))
    b = torch.from_numpy(p.b).to(dev)
    plan = tacta.Plan(A)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    iters_per_step = args.iters
    opts = dict(tol=TOL, tol_normal=0.0, max_iter=iters_per_step, use_graph=0 if args.no_graph else 1)

    for _ in range(args.warmup):
        plan.cta(b, **opts)
    torch.cuda.synchronize()

    # ---------------- timed region: K steps, device events, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    iters = []
    launches = 0
    infos = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            x, hist, info = plan.cta(b, **opts)
            ev[i][1].record(stream)
            iters.append(info["iters"])
            launches += info["launches"]
            infos.append(info)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms, all_iters = aggregate(dist, dev, sum(step_ms), sum(iters))
    value = all_iters / (total_ms * 1e-3)
    clocks = clk.summary()
    last = infos[-1]

    # ---------------- roofline: the fused step kernel, every launch timed with events
    _, _, prof = plan.cta(b, profile=1, **opts)
    # every launch of the fused step kernel timed with events; the unit is an F_t step
    # (a launch runs up to 64 of them): the launches' summed time over the steps they ran
    step_us = 1e3 * prof["spmv_ms"] / prof["spmv_count"]
    alg_bytes = prof["spmv_bytes"] / prof["spmv_count"]      # the survey's bytes per F_t step
    ts = [fpt_schedule(k) for k in range(prof["spmv_count"])]
    t_mean = statistics.fmean(ts)
    peak, peak_kind = peaks()
    achieved = alg_bytes / (step_us * 1e-6) / 1e9
    traffic = traffic_record()
    fpt_bytes = statistics.fmean(survey_bytes_per_fpt(p.m, p.n, p.nnz, fpt_schedule(k))
                                 for k in range(iters_per_step))
    step_gbs = fpt_bytes * value / 1e9
    rows_t = -(-p.m // 256) * 256
    dia_product = 8.0 * 5 * rows_t + rows_t + 8.0 * p.n + 8.0 * p.m     # the diagonal form, k = 5
    fmt_bytes = statistics.fmean(2 * t * dia_product + 8.0 * (t + 2) * (p.m + p.n) for t in ts)
    fmas = statistics.fmean(2 * t * (p.nnz + p.m) + t * (p.n + p.m) + p.m for t in ts)
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "traffic": traffic, "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)",
        "kernel": "cta_chain<double, DiaFmt, true>: the fused step, a persistent cooperative launch "
                  "of up to 64 F_t steps -- per step the 2t products with A\u1d40 and A on the "
                  "diagonal form (bulk-copy row tiles, warp-specialised, grid-wide waits between "
                  "products), then in every block the moments, the auxiliary solve, the stop tests "
                  "and the block's slice of the x and r update",
        "unit_of_work": "one F_t step: the survey's algorithmic bytes of an unfused F_t step of order t, "
                        "t (B_A + B_At) + 8 t (2 m + 2 n) + 8 (t + 2)(m + n) with B_A = 12 nnz + "
                        "4 (m + 1), over the event-timed launches' duration per step",
        "steps_timed": prof["spmv_count"], "avg_step_us": step_us, "mean_t": t_mean,
        "bytes_per_step": alg_bytes, "traffic_unit": "DRAM bytes per F_t step at the mean order t = 3 (ncu)",
        # the whole solve step (the step kernel plus the gated true-residual launch and the
        # gaps between launches) against the same peak
        "step": {"bytes_per_fpt": fpt_bytes, "achieved": step_gbs, "unit": "GB/s", "frac": step_gbs / peak},
        # what DRAM actually served (ncu's dram__bytes per launch over the event-timed launch)
        "dram": ({"achieved": traffic / (step_us * 1e-6) / 1e9, "unit": "GB/s",
                  "frac": traffic / (step_us * 1e-6) / 1e9 / peak} if traffic else None),
        # the diagonal form moves fewer bytes than CSR: values only, k = 5 per row
        "format": {"bytes_per_step": fmt_bytes, "achieved": fmt_bytes / (step_us * 1e-6) / 1e9,
                   "unit": "GB/s", "frac": fmt_bytes / (step_us * 1e-6) / 1e9 / peak},
        "fp64": {"bound": "alu", "flops_per_step": 2.0 * fmas,
                 "achieved": 2.0 * fmas / (step_us * 1e-6) / 1e12,
                 "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                 "frac": 2.0 * fmas / (step_us * 1e-6) / 1e12 / FP64_TFLOPS_NOMINAL,
                 "peak_kind": "nominal FP64 on CUDA cores: 152 SMs x 2 FMA/clk x 2.07 GHz x 2 flops "
                              "(not measured by the driver)"}}

    # ---------------- e2e: one-shot C ABI call with pinned host buffers
    hA = tacta.CSR(torch.from_numpy(p.rowptr).pin_memory(), torch.from_numpy(p.colidx).pin_memory(),
                   torch.from_numpy(p.vals).pin_memory(), (p.m, p.n))
    hb = torch.from_numpy(p.b).pin_memory()
    e2e_steps = min(args.steps, 5)
    tacta.cta_solve(hA, hb, hist_cap=iters_per_step + 1, **opts)       # warm
    e2e_iters, t0 = 0, time.perf_counter()
    for _ in range(e2e_steps):
        xh, hh, ih = tacta.cta_solve(hA, hb, hist_cap=iters_per_step + 1, **opts)
        e2e_iters += ih["iters"]
    e2e_s = time.perf_counter() - t0
    h2d = 4 * (p.m + 1) + 12 * p.nnz + 8 * p.m
    d2h = 8 * p.n + 8 * (iters_per_step + 1)
    e2e = {"value": world * e2e_iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "includes": "H2D of A and b, plan build (device CSR transpose), solve, D2H of x and history"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{GRID}x{GRID}", "n": p.n, "nnz": p.nnz,
                       "iters_per_step": iters_per_step, "t_cycle": "ping-pong 1..5", "R": 40,
                       "tol": TOL, "l2": "flushed between steps (256 MiB write); working set "
                       "~0.23 GB > 129 MB L2", "parallelism": f"replicas x{world}"},
            "rel_res_after_step": last["rel_res"], "time_to_tol_s": None,
            "matvecs_per_s": world * sum(i["matvecs"] for i in infos) / (total_ms * 1e-3),
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_extra:   # the other configurations: at N = 1 only
        line["extra"] = extra_workloads(tacta, dev, stream, plan, b, min(args.steps, 5))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        one = oracle_rate(1, CPU_SAMPLE_ITERS)
        allc = oracle_rate(cores, CPU_SAMPLE_ITERS) if cores > 1 else one
        if one is None or allc is None:           # no child process: time it here
            v, dt, _ = cpu_baseline(p, CPU_SAMPLE_ITERS)
            one = allc = (v, dt)
        line["cpu_baseline"] = {
            "value": allc[0], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {CPU_SAMPLE_ITERS} F_t steps of the same solve ({allc[1]:.1f} s; numpy "
                      f"FP64 with its BLAS pool at {cores} threads; scipy's CSR products, most of the "
                      "work, run on one thread)",
            "host_cores": cores,
            "single_thread": {"value": one[0], "unit": UNIT, "cores": 1, "seconds": one[1]}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
