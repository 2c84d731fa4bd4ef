#!/usr/bin/env python
"""Benchmark: ms per shooting gradient (forward + adjoint) at N = 100,000,
Barnes-Hut against plain exact, on synthetic blob point clouds.

One step = one Barnes-Hut shooting gradient and one exact ("plain")
shooting gradient of the objective of Eq. 2 (T = 20 Euler steps forward, 20
adjoint steps back) on N = 100,000 points drawn from 8 anisotropic Gaussian
blobs in a 60 mm cube, sigma = 1.5 mm, threshold 3 sigma.  `value` is the
Barnes-Hut ms per gradient (the paper's method); the plain exact figure, the
speed-up and pair-interaction rates ride along.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --batched [--steps K] [--warmup W]

--batched measures the many-subject workload instead (64 bent-slab subjects,
N log-uniform in [5000, 40000], sigma = 2 mm, T = 20): ms per gradient of all
subjects for the batched exact and batched Barnes-Hut calls against plain
per-subject exact calls, one JSON line.

With --gpus N > 1 (launched by torch.distributed.run, one rank per GPU) each
rank computes its own replica of the workload (the shooting of one point set
does not shard without an exchange step); value aggregates all ranks'
gradients over the slowest rank's time.  --impl reference times the FP64 CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per shooting gradient (fwd+adjoint) at N=100k vs plain; pair-interactions/s"
UNIT = "ms/gradient"
WORKLOAD = "blobs100k"
THRESH = 3.0
# FP32 pipe: 128 lanes per SM per clock (one FADD/FMUL/FFMA lane-op each),
# 152 SMs, maximum SM clock 2070 MHz.
ALU_PEAK_OPS = 152 * 128 * 2.07e9
# Algorithmic FP32 ops per pair: the formulas' counts (forward 16; adjoint
# 40, the direct evaluation of its four sums).  The adjoint kernels issue 36:
# with beta stored scaled by 2 ln2 s in the adjoint pack, the sums need no
# constants (ISSUED_OPS_PER_PAIR, reported beside the roofline).
OPS_PER_PAIR = {"exact_fwd": 16, "exact_adj": 40, "bh_fwd": 16, "bh_adj": 40, "bh_walk": 16}
ISSUED_OPS_PER_PAIR = {"exact_fwd": 16, "exact_adj": 36, "bh_fwd": 16, "bh_adj": 36,
                       "bh_walk": 16}
# algorithmic bytes per point of one tree pass, averaged over the forward
# builds (about 250 B: FP32 positions and pack read, four sort passes, node
# boxes and records written) and the backward aggregations (about 200 B:
# both packs read, leaf and node records and pair sums written), which
# alternate in the class
TREE_BYTES_PER_POINT = 225.0
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the leaf-size and truncation variant lines (launch-list captures)")
    ap.add_argument("--batched", action="store_true",
                    help="measure the 64-subject batched workload (separate JSON line)")
    ap.add_argument("--sphere", action="store_true",
                    help="measure the 1M-point sphere workload: Barnes-Hut gradient, T = 40, "
                         "checkpoint every 6 steps (separate JSON line)")
    ap.add_argument("--probe", choices=["bh", "exact", "batched", "bhgrad"],
                    help="for profiler captures: two rounds of one forward and one adjoint "
                         "right-hand side at the workload's initial state (batched: one "
                         "exact gradient of the 64-subject workload; bhgrad: two Barnes-Hut "
                         "gradients, the benchmark's kernels), then exit")
    return ap.parse_args()


def workload():
    from paper_1907_04834_gb300 import inputs
    return inputs.config(WORKLOAD)


def config_dict(w, extra=None):
    d = {"workload": f"{WORKLOAD}: N={w.N} points from 8 anisotropic Gaussian blobs (std 2-6 mm) "
                     f"in a 60 mm cube, sigma={w.sigma} mm, T={w.T} Euler steps, lambda={w.lam}, "
                     f"Barnes-Hut threshold {THRESH:g} sigma",
         "N": w.N, "T": w.T, "sigma": w.sigma, "lambda": w.lam, "thresh_sigmas": THRESH,
         "step": "one Barnes-Hut gradient + one exact (plain) gradient, fwd + adjoint",
         "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.p = None
        self.lines = []
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if device_id:
                cmd += ["-i", device_id]
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------- dist
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_ranks(values, world, op="max"):
    """Reduce a list of floats over ranks (identity when world == 1)."""
    if world == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.cpu().tolist()


# --------------------------------------------------------------------- CPU baseline
def oracle_timing(w, bh_reps=2, rows=4000):
    """Times the FP64 oracle on a bounded sample: Barnes-Hut forward + adjoint
    right-hand side at full N (bh_reps times), exact forward + adjoint on
    `rows` sampled rows; extrapolates to ms per gradient (x T steps each)."""
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(0)
    al = rng.normal(size=w.q0.shape)
    be = rng.normal(scale=0.1, size=w.q0.shape)
    t0 = time.perf_counter()
    for _ in range(bh_reps):
        oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=THRESH)
        oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=1, thresh=THRESH)
    bh_step = (time.perf_counter() - t0) / bh_reps
    idx = np.sort(rng.choice(w.N, rows, replace=False))
    t0 = time.perf_counter()
    oracle.rhs_rows(w.q0, w.p0, w.sigma, idx)
    oracle.adj_rhs_rows(w.q0, w.p0, al, be, w.sigma, idx)
    ex_step = (time.perf_counter() - t0) * w.N / rows
    return {"bh_ms": 1e3 * bh_step * w.T, "exact_ms": 1e3 * ex_step * w.T,
            "cores": oracle.num_threads(),
            "sample": f"{bh_reps} x (one Barnes-Hut forward + one adjoint right-hand side at full "
                      f"N={w.N}), x T={w.T}; exact: forward + adjoint on {rows} sampled rows, "
                      f"x N/rows x T"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    w = workload()
    rng = np.random.default_rng(0)
    al = rng.normal(size=w.q0.shape)
    be = rng.normal(scale=0.1, size=w.q0.shape)

    def step():
        t0 = time.perf_counter()
        oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=THRESH)
        oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=1, thresh=THRESH)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    step_ms = 1e3 * sum(ts) / len(ts)
    ms = step_ms * w.T
    sample = (f"each step: one Barnes-Hut forward + one adjoint right-hand side of the FP64 oracle "
              f"at full N={w.N} (ms_per_step, measured); value extrapolates x T={w.T} to one "
              f"gradient")
    cfg = config_dict(w, {"parallelism": "host cores",
                          "step": "one Barnes-Hut forward + one adjoint right-hand side of the "
                                  "FP64 oracle at full N (a T-th of one gradient); value = "
                                  "ms_per_step x T"})
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- ours
def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(kernel_class):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kernel_class)
        if not d:
            return None
        src = os.path.join(ROOT, d["source"])
        if source_sha(src) != d["source_sha"]:
            return None
        return float(d["bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1907_04834_gb300 import native
    native.build()
    import paper_1907_04834_gb300 as gs
    w = workload()
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    q0, p0, X = t(w.q0), t(w.p0), t(w.X)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def bh_grad():
        return gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH)

    def plain_grad():
        return gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="exact")

    # this GPU's measured issue rates (gs_alu_peaks): FP32 FMA lane-ops/s,
    # FP32 lane-ops/s through packed f32x2 FMA, MUFU ex2/s
    alu = gs.alu_peaks(dev.index or 0)
    # interactions per step at t = 0 (the per-gradient count is estimated as 2T x this)
    _, _, cnt = gs.rhs(q0, p0, w.sigma, mode="bh", thresh=THRESH)
    bh_inter_step = cnt[0] + cnt[1]
    # the traversal's node visits at t = 0 (points taken + nodes reached), the
    # walk's warp iterations and the list entries it emits (gs_bh_tally)
    tal, (walk_iters, list_entries) = gs.bh_tally(q0, w.sigma, THRESH, with_stats=True)
    visits_step = int(tal[:, 0].sum() + tal[:, 4].sum())
    for _ in range(args.warmup):
        bh_grad()
        plain_grad()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = str(local)
    # Timed region: the gradients as a caller gets them (each one CUDA graph
    # replayed on the stream, the library's default).
    gs.timing(False)
    gs.timing_read()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(uuid)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        bh_grad()
        ev[k][1].record()
        plain_grad()
        ev[k][2].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    _, launches = gs.timing_read()
    # Kernel pass: the same steps again with CUDA events around every kernel
    # class inside the library (launched one by one: graphs are off while
    # kernel timing is on); the roofline and class shares come from here.
    gs.timing(True)
    gs.timing_read()
    for k in range(args.steps):
        flush.zero_()
        bh_grad()
        plain_grad()
    torch.cuda.synchronize()
    kern, _ = gs.timing_read()
    gs.timing(False)
    bh_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    pl_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    tot_bh, tot_pl = aggregate_ranks([sum(bh_ms), sum(pl_ms)], ws, "max")
    grads = args.steps * ws
    value = tot_bh / grads
    plain = tot_pl / grads
    step_ms = (tot_bh + tot_pl) / args.steps
    pair_bh = 2 * w.T * bh_inter_step
    pair_pl = 2 * w.T * w.N * w.N

    # roofline of the dominant kernel class in the timed region
    dom = max(kern, key=lambda k: kern[k][1])
    nl, ms = kern[dom]
    per_launch_s = ms / max(nl, 1) * 1e-3
    if dom == "tree_build":
        alg = TREE_BYTES_PER_POINT * w.N
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        roof = {"bound": "hbm", "achieved": alg / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s"}
    else:
        units = w.N * w.N if dom.startswith("exact") else bh_inter_step
        alg = OPS_PER_PAIR[dom] * units
        roof = {"bound": "alu", "achieved": alg / per_launch_s / 1e12,
                "peak": ALU_PEAK_OPS / 1e12, "unit": "Tops/s",
                "ops_per_pair": OPS_PER_PAIR[dom],
                "issued_ops_per_pair": ISSUED_OPS_PER_PAIR[dom],
                "issued_frac": ISSUED_OPS_PER_PAIR[dom] * units / per_launch_s / ALU_PEAK_OPS}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if roof["bound"] == "alu":
        # one MUFU ex2 per pair, against this run's measured ex2 rate
        roof["mufu"] = {"achieved": units / per_launch_s / 1e12, "peak": alu[2] / 1e12,
                        "unit": "T ex2/s", "frac": units / per_launch_s / alu[2],
                        "peak_kind": "measured (gs_alu_peaks)"}
        roof["frac_of_measured_f32x2"] = alg / per_launch_s / alu[1]
    roof["kernel"] = dom
    roof["launch_ms"] = per_launch_s * 1e3
    roof["share"] = ms / max(sum(v[1] for v in kern.values()), 1e-9)
    tr = measured_traffic(dom)
    roof["traffic"] = tr
    # every timed class against its own roof (the pair classes against the
    # FP32 pipe, the tree class -- forward builds and backward aggregations
    # alternate, TREE_BYTES_PER_POINT on average -- against HBM); the walk
    # issues compares and branches, no pair arithmetic, and has none
    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    class_roofs = {}
    for cls, (ncl, mcl) in kern.items():
        per = mcl / max(ncl, 1) * 1e-3
        if cls == "tree_build":
            gbs = TREE_BYTES_PER_POINT * w.N / per / 1e9
            class_roofs[cls] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                "unit": "GB/s", "frac": gbs / hbm_peak,
                                "bytes_per_point": TREE_BYTES_PER_POINT}
        elif cls in ("exact_fwd", "exact_adj", "bh_fwd", "bh_adj"):
            units = w.N * w.N if cls.startswith("exact") else bh_inter_step
            ach = OPS_PER_PAIR[cls] * units / per / 1e12
            class_roofs[cls] = {"bound": "alu", "achieved": ach, "peak": ALU_PEAK_OPS / 1e12,
                                "unit": "Tops/s", "frac": ach * 1e12 / ALU_PEAK_OPS,
                                "issued_frac": ISSUED_OPS_PER_PAIR[cls] * units / per
                                / ALU_PEAK_OPS,
                                "mufu_frac": units / per / alu[2]}
            if cls.startswith("bh"):
                # lanes evaluate every list entry of their warp; the share of
                # those lane-slots holding an interaction, and the issued
                # fraction per evaluated lane-slot
                slots = 32.0 * list_entries
                class_roofs[cls]["lane_slots_taken"] = bh_inter_step / slots
                class_roofs[cls]["issued_frac_per_lane_slot"] = (
                    ISSUED_OPS_PER_PAIR[cls] * slots / per / ALU_PEAK_OPS)
        elif cls == "bh_walk":
            # no arithmetic roof: the algorithmic work is the per-point
            # traversal's node visits, against the walk's lane-slots
            class_roofs[cls] = {"bound": "issue", "node_visits": visits_step,
                                "warp_iterations": walk_iters,
                                "visits_per_lane_slot": visits_step / (32.0 * walk_iters),
                                "visits_per_s": visits_step / per,
                                "ms_per_walk": per * 1e3}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(w, {"parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"}),
            "plain_ms_per_gradient": plain, "speedup_vs_plain": plain / value,
            "pair_interactions_per_s": {"bh": pair_bh * grads / (tot_bh * 1e-3),
                                        "plain": pair_pl * grads / (tot_pl * 1e-3)},
            "exact_equivalent_pairs_per_s_bh": pair_pl * grads / (tot_bh * 1e-3),
            "shooting_steps_per_s_bh": 2 * w.T * grads / (tot_bh * 1e-3),
            "bh_interactions_per_point_step": bh_inter_step / w.N,
            "roofline": roof,
            "kernels": {k: {"launch_groups": v[0], "ms": v[1]} for k, v in kern.items()},
            "class_rooflines": class_roofs,
            "gpu_launches": launches, "wall_s": wall, "clocks": ck,
            "alu_peaks_measured": {"fp32_fma_lane_ops_per_s": alu[0],
                                   "fp32_f32x2_lane_ops_per_s": alu[1], "mufu_ex2_per_s": alu[2],
                                   "derived_fp32_peak_lane_ops_per_s": ALU_PEAK_OPS}}

    if rank == 0 and not args.no_variants:
        # leaf-size variant picked by the autotuner on the initial state (a
        # declared variant of the approximation; `value` stays the paper's
        # leaf size 1), with both gradients' distance from the exact gradient
        best, tune_ms = gs.autotune(q0, p0, w.sigma, thresh=THRESH)
        _, g_ex, _ = plain_grad()
        _, g_bh, _ = bh_grad()
        tuned = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH,
                                      leaf_size=best)
        tuned()
        tms = []
        for _ in range(3):
            flush.zero_()
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record()
            _, g_tu, _ = tuned()
            b_ev.record()
            torch.cuda.synchronize()
            tms.append(a_ev.elapsed_time(b_ev))
        nrm = float(torch.linalg.norm(g_ex))
        line["bh_leaf_variant"] = {
            "leaf_size": best, "ms_per_gradient": statistics.median(tms),
            "autotune_ms_per_fwd_adj_step": {str(k): v for k, v in tune_ms.items()},
            "grad_rel_l2_vs_exact": float(torch.linalg.norm(g_tu - g_ex)) / nrm,
            "paper_leaf1_grad_rel_l2_vs_exact": float(torch.linalg.norm(g_bh - g_ex)) / nrm}
        # pure 3-sigma truncation (far field dropped), same threshold
        trunc = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="trunc",
                                      thresh=THRESH)
        trunc()
        tms = []
        for _ in range(3):
            flush.zero_()
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record()
            _, g_tr, _ = trunc()
            b_ev.record()
            torch.cuda.synchronize()
            tms.append(a_ev.elapsed_time(b_ev))
        line["trunc_variant"] = {"ms_per_gradient": statistics.median(tms),
                                 "grad_rel_l2_vs_exact":
                                 float(torch.linalg.norm(g_tr - g_ex)) / nrm}
        # semi-implicit symplectic Euler shooting (forward only): the cost of
        # its fixed-point passes, which reuse each step's tree and lists
        def shoot_ms(M):
            gs.shoot(q0, p0, w.sigma, w.T, mode="bh", thresh=THRESH, sympl_iters=M)
            ts = []
            for _ in range(3):
                flush.zero_()
                a_ev = torch.cuda.Event(enable_timing=True)
                b_ev = torch.cuda.Event(enable_timing=True)
                a_ev.record()
                gs.shoot(q0, p0, w.sigma, w.T, mode="bh", thresh=THRESH, sympl_iters=M)
                b_ev.record()
                torch.cuda.synchronize()
                ts.append(a_ev.elapsed_time(b_ev))
            return statistics.median(ts)
        line["sympl_variant"] = {"passes": 2, "bh_ms_per_shoot": shoot_ms(2),
                                 "explicit_bh_ms_per_shoot": shoot_ms(0)}
        # tile shape of the exact kernels (source splits J) picked by the
        # autotuner on the initial state, against the built-in choice: one
        # plain exact gradient each (J changes rounding only)
        (jf, ja), jms = gs.autotune_exact(q0, p0, w.sigma)

        def plain_ms():
            plain_grad()
            ts = []
            for _ in range(2):
                flush.zero_()
                a_ev = torch.cuda.Event(enable_timing=True)
                b_ev = torch.cuda.Event(enable_timing=True)
                a_ev.record()
                plain_grad()
                b_ev.record()
                torch.cuda.synchronize()
                ts.append(a_ev.elapsed_time(b_ev))
            return min(ts)
        builtin_ms = plain_ms()
        gs.set_option("exact_splits_fwd", jf)
        gs.set_option("exact_splits_adj", ja)
        try:
            tuned_ms = plain_ms()
        finally:
            gs.set_option("exact_splits_fwd", 0)
            gs.set_option("exact_splits_adj", 0)
        line["exact_tile_variant"] = {
            "splits_fwd": jf, "splits_adj": ja, "ms_per_gradient": tuned_ms,
            "builtin_ms_per_gradient": builtin_ms,
            "autotune_ms_per_fwd_adj_rhs": {str(k): v for k, v in jms.items()}}
    if rank == 0 and not args.no_variants:
        # the same workload with momenta 20x larger: points move by about
        # 0.8 kernel widths (median; 2 at the 90th percentile) over t in [0, 1], so the decisions
        # change from step to step
        p20 = 20.0 * p0
        dgrad = lambda: gs.shoot_grad(q0, p20, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH)
        dgrad()
        tms = []
        for _ in range(3):
            flush.zero_()
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record()
            dgrad()
            b_ev.record()
            torch.cuda.synchronize()
            tms.append(a_ev.elapsed_time(b_ev))
        q1d, _, _ = gs.shoot(q0, p20, w.sigma, w.T, mode="bh", thresh=THRESH)
        mv = torch.linalg.norm(q1d - q0, dim=1) / w.sigma
        line["deforming_variant"] = {
            "momenta": "20x the workload's", "ms_per_gradient": statistics.median(tms),
            "displacement_sigmas": {"median": float(mv.median()), "max": float(mv.max())}}
        line["batched"] = batched_summary(gs, torch, steps=1, warmup=1)
        line["sphere1m"] = sphere_summary(gs, torch, steps=2, warmup=1)
    if rank == 0 and args.e2e_steps > 0:
        # end to end through the C ABI with pinned host buffers (H2D + D2H inside)
        h = lambda a: torch.as_tensor(a, dtype=torch.float64).pin_memory()
        hq, hp, hX = h(w.q0), h(w.p0), h(w.X)
        gs.shoot_grad(hq, hp, hX, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH)
        es = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            E, g, q1 = gs.shoot_grad(hq, hp, hX, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH)
            es.append((time.perf_counter() - t0) * 1e3)
        line["e2e"] = {"value": statistics.median(es), "unit": UNIT,
                       "h2d_bytes_per_step": 3 * w.N * 3 * 8,
                       "d2h_bytes_per_step": (3 + 2 * w.N * 3) * 8}
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            ob = oracle_timing(w)
            line["cpu_baseline"] = {"value": ob["bh_ms"], "unit": UNIT, "cores": ob["cores"],
                                    "kind": "oracle", "sample": ob["sample"],
                                    "plain_value": ob["exact_ms"]}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_probe(args):
    import torch
    from paper_1907_04834_gb300 import native
    native.build()
    import paper_1907_04834_gb300 as gs
    w = workload()
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    q, p = t(w.q0), t(w.p0)
    gen = torch.Generator(device=dev).manual_seed(0)
    al = torch.randn(q.shape, dtype=torch.float64, device=dev, generator=gen)
    be = 0.1 * torch.randn(q.shape, dtype=torch.float64, device=dev, generator=gen)
    gs.set_option("graphs", 0)  # plain launches for the profiler
    if args.probe == "batched":
        import numpy as np
        from paper_1907_04834_gb300 import inputs
        ws, off = inputs.batch()
        cat = lambda k: t(np.concatenate([getattr(v, k) for v in ws]))
        gs.shoot_batched(cat("q0"), cat("p0"), cat("X"), off, ws[0].sigma, ws[0].T, ws[0].lam)
        torch.cuda.synchronize()
        print(json.dumps({"probe": "batched", "N": int(off[-1]), "ok": True}))
        return 0
    if args.probe == "bhgrad":
        X = t(w.X)
        for _ in range(2):
            gs.shoot_grad(q, p, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH)
        torch.cuda.synchronize()
        print(json.dumps({"probe": "bhgrad", "N": w.N, "ok": True}))
        return 0
    mode = "bh" if args.probe == "bh" else "exact"
    for _ in range(2):
        gs.rhs(q, p, w.sigma, mode=mode, thresh=THRESH)
        gs.adj_rhs(q, p, al, be, w.sigma, mode=mode, thresh=THRESH)
    torch.cuda.synchronize()
    print(json.dumps({"probe": args.probe, "N": w.N, "ok": True}))
    return 0


def _timed(torch, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def batched_summary(gs, torch, steps=1, warmup=1):
    """64 bent-slab subjects (N log-uniform in [5000, 40000], sigma = 2,
    T = 20): ms per gradient of all subjects, batched Barnes-Hut (one forest
    per step) against plain per-subject exact calls, and the Barnes-Hut
    gradient's relative L2 distance from the batched exact gradient."""
    import numpy as np
    from paper_1907_04834_gb300 import inputs
    ws, off = inputs.batch()
    dev = torch.device("cuda", torch.cuda.current_device())
    cat = lambda k: torch.as_tensor(np.concatenate([getattr(w, k) for w in ws]), device=dev)
    q0, p0, X = cat("q0"), cat("p0"), cat("X")
    sig, T, lam = ws[0].sigma, ws[0].T, ws[0].lam

    def plain():
        for k in range(len(ws)):
            sl = slice(int(off[k]), int(off[k + 1]))
            gs.shoot_grad(q0[sl], p0[sl], X[sl], sig, T, lam, mode="exact")

    bh = lambda: gs.shoot_batched(q0, p0, X, off, sig, T, lam, mode="bh", thresh=THRESH)
    ms_bh = _timed(torch, bh, steps, warmup)
    ms_pl = _timed(torch, plain, steps, warmup)
    _, gb = bh()
    _, ge = gs.shoot_batched(q0, p0, X, off, sig, T, lam, mode="exact")
    return {"ms_batched_bh": ms_bh, "ms_plain_per_subject_exact": ms_pl,
            "speedup_batched_bh_vs_plain": ms_pl / ms_bh,
            "bh_vs_exact_grad_rel_l2": float(torch.linalg.norm(gb - ge) / torch.linalg.norm(ge)),
            "workload": f"{len(ws)} bent-slab subjects, N log-uniform in [5000, 40000] (total "
                        f"{int(off[-1])}), sigma={sig} mm, T={T}, lambda={lam}",
            "steps": steps, "warmup": warmup}


def sphere_summary(gs, torch, steps=2, warmup=1):
    """sphere1m (N = 1,000,000, sigma = 1, T = 40): ms per Barnes-Hut
    gradient with the trajectory checkpointed every 6 steps."""
    from paper_1907_04834_gb300 import inputs
    w = inputs.config("sphere1m")
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    q0, p0, X = t(w.q0), t(w.p0), t(w.X)
    _, _, cnt = gs.rhs(q0, p0, w.sigma, mode="bh", thresh=THRESH)
    fn = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH,
                               ckpt_every=6)
    ms = _timed(torch, fn, steps, warmup)
    # the tree build at 10^6 points against HBM (kernel classes, one gradient)
    gs.timing(True)
    gs.timing_read()
    fn()
    torch.cuda.synchronize()
    kern, _ = gs.timing_read()
    gs.timing(False)
    nb, tb = kern["tree_build"]
    per = tb / max(nb, 1) * 1e-3
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    gbs = TREE_BYTES_PER_POINT * w.N / per / 1e9
    return {"ms_per_gradient": ms,
            "bh_interactions_per_point_step": (cnt[0] + cnt[1]) / w.N,
            "class_ms_per_gradient": {k: v[1] for k, v in kern.items() if v[0]},
            "tree_build": {"bound": "hbm", "us_per_pass": per * 1e6, "achieved": gbs,
                           "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                           "bytes_per_point": TREE_BYTES_PER_POINT},
            "workload": f"sphere1m: N={w.N}, sigma={w.sigma} mm, T={w.T}, checkpoint every 6",
            "steps": steps, "warmup": warmup}


def run_batched(args):
    """64 slab subjects: batched exact, batched Barnes-Hut and plain
    per-subject exact gradients, CUDA events around each call."""
    import numpy as np
    import torch
    from paper_1907_04834_gb300 import native, inputs
    native.build()
    import paper_1907_04834_gb300 as gs
    ws, off = inputs.batch()
    dev = torch.device("cuda", 0)
    cat = lambda k: torch.as_tensor(np.concatenate([getattr(w, k) for w in ws]), device=dev)
    q0, p0, X = cat("q0"), cat("p0"), cat("X")
    sig, T, lam = ws[0].sigma, ws[0].T, ws[0].lam
    ns = np.diff(off)

    def plain():
        for k in range(len(ws)):
            sl = slice(int(off[k]), int(off[k + 1]))
            gs.shoot_grad(q0[sl], p0[sl], X[sl], sig, T, lam, mode="exact")

    runs = {"batched_exact": lambda: gs.shoot_batched(q0, p0, X, off, sig, T, lam, mode="exact"),
            "batched_bh": lambda: gs.shoot_batched(q0, p0, X, off, sig, T, lam, mode="bh",
                                                   thresh=THRESH),
            "plain_per_subject_exact": plain}
    res = {}
    for name, fn in runs.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        res[name] = statistics.median(ts)
    Eb, gb = runs["batched_bh"]()
    Ee, ge = runs["batched_exact"]()
    line = {"mode": "batched", "unit": "ms per gradient of all subjects", "steps": args.steps,
            "warmup": args.warmup, "ms": res,
            "speedup_batched_bh_vs_plain": res["plain_per_subject_exact"] / res["batched_bh"],
            "speedup_batched_exact_vs_plain": res["plain_per_subject_exact"] / res["batched_exact"],
            "bh_vs_exact_grad_rel_l2": float(torch.linalg.norm(gb - ge) / torch.linalg.norm(ge)),
            "exact_pairs_per_s_batched": 2 * T * float(np.sum(ns.astype(float) ** 2))
            / (res["batched_exact"] * 1e-3),
            "config": {"workload": f"{len(ws)} bent-slab subjects, N log-uniform in [5000, 40000] "
                                   f"(total {int(off[-1])}), sigma={sig} mm, T={T}, lambda={lam}",
                       "dtype": "f32 pair sums, f64 state"}}
    print(json.dumps(line))
    return 0


def run_sphere(args):
    """N = 1,000,000 points on a bumpy 50 mm sphere, sigma = 1 mm, T = 40:
    Barnes-Hut gradient with the trajectory checkpointed every 6 steps (the
    paper's rule and the autotuned leaf size), CUDA events around each call."""
    import torch
    from paper_1907_04834_gb300 import native, inputs
    native.build()
    import paper_1907_04834_gb300 as gs
    w = inputs.config("sphere1m")
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    q0, p0, X = t(w.q0), t(w.p0), t(w.X)
    _, _, cnt = gs.rhs(q0, p0, w.sigma, mode="bh", thresh=THRESH)
    best, _ = gs.autotune(q0, p0, w.sigma, thresh=THRESH)
    res = {}
    for name, leaf in (("bh", 1), (f"bh_leaf{best}", best)):
        fn = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode="bh", thresh=THRESH,
                                   ckpt_every=6, leaf_size=leaf)
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record()
            fn()
            b_ev.record()
            torch.cuda.synchronize()
            ts.append(a_ev.elapsed_time(b_ev))
        res[name] = statistics.median(ts)
    line = {"mode": "sphere", "unit": "ms per gradient", "steps": args.steps,
            "warmup": args.warmup, "ms": res,
            "bh_interactions_per_point_step": (cnt[0] + cnt[1]) / w.N,
            "config": {"workload": f"sphere1m: N={w.N} points on a 50 mm sphere with 32 radial "
                                   f"bumps, sigma={w.sigma} mm, T={w.T}, lambda={w.lam}, "
                                   "checkpoint every 6 steps, Barnes-Hut threshold 3 sigma"}}
    print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.probe:
        return run_probe(args)
    if args.batched:
        return run_batched(args)
    if args.sphere:
        return run_sphere(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
