#!/usr/bin/env python
"""Benchmark: ENO-MR cell-updates/s per RK stage on one GB300.

Workload: 2D Euler (gamma = 1.4) four-quadrant Riemann problem on [0,1]^2,
interface at (0.8, 0.8), quadrant states drawn with seed = rank, 4096^2 cells,
ENO-MR order 9, transmissive boundaries, SSP-RK3 with the CFL 0.5 step
computed on the device.  One benchmark step = one SSP-RK3 step (3 stages);
the default 100 steps from t = 0 are the workload's whole run.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (test infrastructure, not the product path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ENO-MR cell-updates/s per RK stage"
UNIT = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--order", type=int, default=9)
    ap.add_argument("--cfl", type=float, default=0.5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--paper-runs", action="store_true",
                    help="also time the paper's 2D problems as whole runs (about 2.5 min)")
    ap.add_argument("--occupancy", choices=["auto", "high", "low"], default="auto",
                    help="sweep instance of the paper's 2D runs (enomr_set_occupancy)")
    ap.add_argument("--only", choices=["adjoint", "batched", "vortex", "paper"], default=None,
                    help="run one secondary measurement alone (profiling aid)")
    return ap.parse_args()


def config(a):
    return {"workload": "euler2d_quadrant_riemann", "grid": [a.n, a.n], "order": a.order,
            "cfl": a.cfl, "bc": "transmissive", "time_integrator": "SSP-RK3",
            "step": "one SSP-RK3 step = 3 RK stages", "seed": "rank",
            "run": f"{a.steps} SSP-RK3 steps from t = 0",
            "l2": "inputs larger than L2 (one state is %.0f MB)" % (4 * 8 * a.n * a.n / 1e6)}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=50):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.marks = {}

    def mark(self, name):
        """Remember the current sample count (start or end of a window)."""
        self.marks[name] = len(self.lines)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summary()

    def summary(self, start=None, end=None):
        """Median SM clock, max clock and throttle reasons of the samples
        between two marks (default: all samples)."""
        lo = self.marks.get(start, 0) if start else 0
        hi = self.marks.get(end, len(self.lines)) if end else len(self.lines)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[lo:hi]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "period_ms": self.period_ms}


# ---------------------------------------------------------------------------
# algorithmic FP64 work of one sweep launch (counted per interface; an FMA is
# two flops, an add, multiply, divide or square root one)
# ---------------------------------------------------------------------------
def sweep_work(order, C, sel, n_interfaces, counts, stage_epilogue=False):
    """Algorithmic work of one Euler sweep as (flops, FP64 operations).

    Operations are FP64-pipe operations of a minimal evaluation: fma, mul,
    add, div and rsqrt count 1 each (div and rsqrt as one operation, though
    the hardware evaluates them with several); flops count an fma as 2.
    Sign flips, |x|, min/max and compares, which the kernels do on the
    integer ALU, count 0.  (ops, flops) per part, C = 4 / C = 3:

    every cell that differs from its predecessor along the line (a cell
    equal to it repeats its values):
      the cell's primitives and normal flux        15, 18 / 12, 14
    every cell of a tile that is not on one state per line (in a tile on
    one state per line every flux difference is exactly zero):
      flux difference of the cell                  2C, 2C
      add of the other sweep's part, when the sweep carries the stage
                                                   C, C
    every cell, when the sweep carries the SSP-RK3 stage (the mean of the
    three stages: the first is U + dt D, 1 fma; the others 2 fma, 1 mul)
                                                   7C/3, 4C
    flat interfaces with bitwise-equal centre states (both sides take
    S(0,0) on one state U, whose flux R L F(U) = F(U) is the cell's flux):
      nothing more
    every other interface:
      Roe eigen-quantities and scaled rows of L    16, 19 / 15, 17
      back-projection F = R (f^+ + f^-)            19, 24 / 16, 19
    the Roe average, where the centre states differ 11, 14 / 8, 10
    other flat interfaces (both sides: three equal cell states at the
    side's centre, so IS_0 = 0 exactly and minmod returns v(0)):
      projection of the two centre cells           20, 40 / 12, 24 each
      per field: two split fmas and f^+ + f^-      3, 5
    the remaining interfaces:
      projection of the 2g-cell window             20, 40 / 12, 24 per cell
      per field: split of 2(2g-1) values and f^+ + f^-
      per window (2C): the baseline indicator      6, 8
        the indicators of the tested candidates up to the chosen one
                                                   |S|, 2|S|-1 each
        (none when IS_0 = 0), and the reconstruction on the chosen stencil
        (|S|, 2|S|-1) or the minmod fma (1, 2).
    sel: selection histogram counts[T+3] over all windows of the launch
    (flat interfaces included); counts: (flat, flat with equal centre
    states, equal centre states) interface counts, the number of cells
    that differ from their predecessor along the line and, optionally, the
    number of cells in tiles not on one state per line (sweep_counts;
    without it every cell counts as in such a tile).  The cell counts use
    n_interfaces (one interface per cell of a line, plus one)."""
    import oracle  # table sizes only
    n_flat, n_flat_eq, n_eq, n_distinct = counts[:4]
    n_busy = counts[4] if len(counts) > 4 else n_interfaces
    g = (order + 1) // 2
    T = oracle.num_tested(order)
    sizes = np.array([oracle.candidate(order, t)[0] + oracle.candidate(order, t)[1] + 1
                      for t in range(T)], dtype=np.float64)
    four = C == 4
    proj = np.array([20, 40] if four else [12, 24], dtype=np.float64)
    cell = np.array([15, 18] if four else [12, 14], dtype=np.float64)
    busy = np.array([2 * C, 2 * C], dtype=np.float64) + (C if stage_epilogue else 0)
    stage = np.array([7 * C / 3, 4 * C]) if stage_epilogue else np.zeros(2)
    eigen = (np.array([16, 19] if four else [15, 17])
             + np.array([19, 24] if four else [16, 19])).astype(np.float64)
    roe_avg = np.array([11, 14] if four else [8, 10], dtype=np.float64)
    w = float(n_distinct) * cell + float(n_busy) * busy + float(n_interfaces) * stage
    w += float(n_interfaces - n_flat_eq) * eigen
    w += float(n_interfaces - n_eq) * roe_avg
    w += float(n_flat - n_flat_eq) * (2 * proj + C * np.array([3, 5]))
    split = np.array([2 * (2 * g - 1) + 1, 4 * (2 * g - 1) + 1], dtype=np.float64)
    w += float(n_interfaces - n_flat) * (proj * 2 * g + C * split)
    cum = np.stack([np.cumsum(sizes), np.cumsum(2 * sizes - 1)], axis=1)  # walk to t
    cnt = np.asarray(sel, dtype=np.float64).copy()
    cnt[T + 2] -= 2 * C * n_flat  # the flat interfaces' windows
    base = np.array([6, 8], dtype=np.float64)
    for t in range(T):
        w += cnt[t] * (base + cum[t] + np.array([sizes[t], 2 * sizes[t] - 1]))
    # minmod outcomes: S(0,1) and S(1,0) come after a full walk; S(0,0) is
    # counted as the IS_0 = 0 shortcut (lower bound)
    w += (cnt[T] + cnt[T + 1]) * (base + cum[-1] + np.array([1, 2]))
    w += cnt[T + 2] * (base + np.array([1, 2]))
    return float(w[1]), float(w[0])


# Tile shapes of the 2D sweeps (cells along the line, lines): row sweep,
# column sweep.  Each tile writes TP - 1 cells of each of its lines and stages
# g cells beyond them on either side.
SWEEP_TILES = {0: (128, 2), 1: (64, 4)}


def busy_cells(U, axis, order):
    """Cells of a transmissive 2D sweep (axis 0: x, 1: y) in tiles that are
    not on one state per line: some line of the tile has two neighbouring
    staged cells that differ (ghost cells repeat the edge cell)."""
    import torch
    TP, NL = SWEEP_TILES[axis]
    g = (order + 1) // 2
    X = U if axis == 0 else U.transpose(1, 2)
    nl, n = X.shape[1], X.shape[2]
    d = (X[..., 1:] != X[..., :-1]).any(dim=0).to(torch.int32)        # cell c vs c - 1
    P = torch.nn.functional.pad(torch.cumsum(d, dim=1), (1, 0))       # P[:, c]: diffs in 1..c
    nseg = (n + TP - 2) // (TP - 1)
    x0 = torch.arange(nseg, device=X.device) * (TP - 1)
    a = (x0 - g).clamp(0, n - 1)
    b = (x0 + TP + g - 2).clamp(0, n - 1)
    varies = (P[:, b] - P[:, a]) > 0                                   # [line, tile]
    ngrp = (nl + NL - 1) // NL
    pad = ngrp * NL - nl
    if pad:
        varies = torch.cat([varies, varies[-1:].expand(pad, -1)], dim=0)  # clamped lines
    busy = varies.view(ngrp, NL, nseg).any(dim=1)                      # [group, tile]
    lines = torch.full((ngrp,), NL, device=X.device)
    lines[-1] = nl - (ngrp - 1) * NL
    cells = torch.minimum(x0 + TP - 1, torch.tensor(n, device=X.device)) - x0
    return int((busy.to(torch.int64) * lines[:, None] * cells[None, :]).sum().item())


def sweep_counts(U, axis, order):
    """flat_interfaces(U, axis) and busy_cells(U, axis, order): the counts
    sweep_work takes."""
    return flat_interfaces(U, axis) + (busy_cells(U, axis, order),)


def flat_interfaces(U, axis):
    """Interface counts of a transmissive 2D sweep (axis 0: x, 1: y):
    (flat, flat with bitwise-equal centre states, bitwise-equal centre
    states), flatness in the sense of the kernel's shortcut, and the number
    of cells that differ from their predecessor along the line (a line's
    first cell included)."""
    import torch
    X = U if axis == 0 else U.transpose(1, 2)
    Xp = torch.nn.functional.pad(X.unsqueeze(0), (3, 3, 0, 0), mode="replicate")[0]
    eq = (Xp[..., 1:] == Xp[..., :-1]).all(dim=0)      # eq[:, j]: padded cells j, j+1
    nI = X.shape[2] + 1
    e = [eq[:, o:o + nI] for o in range(5)]            # e_o: cells k-3+o, k-2+o
    flat = ((e[0] & e[1]) | (e[2] & e[3])) & ((e[3] & e[4]) | (e[1] & e[2]))
    same_prev = (X[..., 1:] == X[..., :-1]).all(dim=0)
    distinct = X.shape[1] + int((~same_prev).sum().item())
    return (int(flat.sum().item()), int((flat & e[2]).sum().item()), int(e[2].sum().item()),
            distinct)


KERNEL_SOURCES = ("enomr_sweep.cuh", "enomr_tma.cuh", "enomr_kernels.cuh", "enomr_common.cuh",
                  "gen_coeffs.py")


def kernel_source_digest():
    """sha256 over the sources that define the sweep kernels (code and tile
    shapes)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2311_15504_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kname, n, order):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary of this workload, or None when that summary was taken on other
    kernel sources (or does not cover this kernel and size)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                        f"euler2d_riemann_{n}_r{order}_launches.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    rec = {}
    for ln in lines:
        if ln.startswith("    ") or ":" not in ln:
            continue
        k, _, v = ln.partition(":")
        rec[k.strip().strip("`")] = v.strip().strip("`")
    if rec.get("kernel sources sha256") != kernel_source_digest():
        return None
    v = rec.get(f"dram bytes per launch {kname}")
    return float(v) if v else None


def batched_gain(enomr, workloads, dev, a, nprob=4096, order=9, reps=5):
    """4096 independent 1D Euler Riemann problems (sizes log-uniform in
    [128, 8192]): the persistent batched step (autotuned, captured in a CUDA
    graph) against one enomr_step per problem (the same kernels' arithmetic,
    all 4096 captured in one CUDA graph)."""
    import torch
    sizes, Us, hs = workloads.riemann_batch(nprob, seed=0)
    B = enomr.Batch(sizes, hs, order=order, bc=enomr.TRANSMISSIVE, device=dev)
    Ub = B.pack(Us)
    B.autotune(Ub, reps=2)
    tile, grid, per_item = B.config()
    cells = int(sizes.sum())

    def timed(graph):
        graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        B.step(Ub, a.cfl)
    torch.cuda.synchronize()
    gb = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb):
        B.step(Ub, a.cfl)
    ms_b = timed(gb)
    Up = B.pack(Us)
    singles = [enomr.Solver(enomr.EULER, int(n), order=order, dx=float(h),
                            bc=enomr.TRANSMISSIVE, device=dev) for n, h in zip(sizes, hs)]
    views = [B.view(Up, p) for p in range(nprob)]
    with torch.cuda.stream(side):
        for sp, v in zip(singles, views):
            sp.step(v, 0.0, a.cfl)
    torch.cuda.synchronize()
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp):
        for sp, v in zip(singles, views):
            sp.step(v, 0.0, a.cfl)
    ms_p = timed(gp)
    # the fair per-problem baseline: the same launches spread over 8 streams,
    # captured as 8 parallel branches of one graph (independent problems,
    # each with its own context)
    nbr = 8
    branches = [torch.cuda.Stream(device=dev) for _ in range(nbr)]
    gc = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gc):
        cap = torch.cuda.current_stream(dev)
        for b in branches:
            b.wait_stream(cap)
        for k, b in enumerate(branches):
            with torch.cuda.stream(b):
                for p_ in range(k, nprob, nbr):
                    singles[p_].step(views[p_], 0.0, a.cfl)
        for b in branches:
            cap.wait_stream(b)
    ms_c = timed(gc)
    # same arithmetic: after the same number of steps the two states agree bitwise
    Ub2, Up2 = B.pack(Us), B.pack(Us)
    with torch.cuda.stream(side):
        for _ in range(2):
            B.step(Ub2, a.cfl)
            for sp, p in zip(singles, range(nprob)):
                sp.step(B.view(Up2, p), 0.0, a.cfl)
    torch.cuda.synchronize()
    identical = bool(torch.equal(Ub2, Up2))
    for sp in singles:
        sp.close()
    B.close()
    return {"workload": f"{nprob} 1D Euler Riemann problems, sizes log-uniform [128, 8192] "
                        f"({cells} cells), order {order}, transmissive, CFL {a.cfl}",
            "batched": {"value": cells * 3 / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b,
                        "tile": tile, "grid": grid, "tiles_per_item": per_item,
                        "launches_per_step": 5},
            "per_problem_serial": {"value": cells * 3 / (ms_p * 1e-3), "unit": UNIT,
                                   "ms_per_step": ms_p, "launches_per_step": 7 * nprob,
                                   "form": "one stream, one CUDA graph"},
            "per_problem_concurrent": {"value": cells * 3 / (ms_c * 1e-3), "unit": UNIT,
                                       "ms_per_step": ms_c, "launches_per_step": 7 * nprob,
                                       "form": f"{nbr} parallel branches of one CUDA graph"},
            "gain": ms_c / ms_b, "gain_vs_serial": ms_p / ms_b,
            "gain_definition": "concurrent per-problem launches / persistent batched step",
            "bitwise_identical_after_2_steps": identical}


def adjoint_ratio(enomr, workloads, dev, n=1024, order=9, steps=200, cfl=0.5):
    """The adjoint workload: isentropic vortex n^2 (periodic, order 9),
    `steps` CFL steps through the differentiable rollout (per-step
    checkpoints; dt kept on the device and recomputed from each checkpoint
    in the backward pass), loss 1/2 ||rho(t) - rho_target||^2.  Times the
    forward rollout (steps + checkpoint copies) and the backward pass; the
    device memory in use at the peak (all checkpoints alive) is read from
    the driver, so the library's own scratch is included."""
    import torch
    U0, h, _ = workloads.isentropic_vortex(n)
    rng = np.random.Generator(np.random.PCG64(2024))
    Ut = U0.copy()
    Ut[0] += 1e-3 * rng.standard_normal((n, n))
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info(dev)
    s = enomr.Solver(enomr.EULER, (n, n), order=order, dx=h, dy=h, bc=enomr.PERIODIC,
                     device=dev)
    tgt_state = torch.from_numpy(Ut).to(dev)
    for _ in range(steps):
        s.step(tgt_state, 0.0, cfl)
    tgt = tgt_state[0].clone()
    del tgt_state
    # warm-up of both directions
    x = torch.from_numpy(U0).to(dev).requires_grad_(True)
    out = enomr.rollout(x, s, 2, cfl=cfl)
    (0.5 * ((out[0] - tgt) ** 2).sum()).backward()
    torch.cuda.synchronize()
    x = torch.from_numpy(U0).to(dev).requires_grad_(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    out = enomr.rollout(x, s, steps, cfl=cfl)
    loss = 0.5 * ((out[0] - tgt) ** 2).sum()
    e[1].record()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    loss.backward()
    e[2].record()
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1]) / steps
    bwd = e[1].elapsed_time(e[2]) / steps
    g_norm = float(x.grad.norm())
    s.close()
    return {"workload": f"isentropic vortex {n}^2 periodic, order {order}, {steps} CFL steps, "
                        "loss 1/2 ||rho(t) - rho_target||^2",
            "forward_ms_per_step": round(fwd, 4), "adjoint_ms_per_step": round(bwd, 4),
            "ratio": bwd / fwd, "forward_includes_checkpoint_copy": True,
            "device_bytes_at_peak": int(free0 - free1),
            "checkpoint_bytes": int(steps * U0.nbytes),
            "host_syncs_per_step": 0, "grad_norm": g_norm}


def probe_ops_peak(enomr, dev):
    """Measured FP64 throughput: the all-SM FMA-chain probe, in flop/s and
    in FP64 pipe operations/s (an fma is one operation, two flops)."""
    fl, _ = enomr.probe_fp64_fma(iters=20000, device=dev)
    return fl, fl / 2.0


def sweep_fracs(enomr, solver, U, order, n, cfl, peak_ops, steps=2, probe_ops=None):
    """The x and y sweeps of `steps` SSP-RK3 steps from state U, each timed
    live on the library's stream (mean ms per launch), against:
      frac (= frac_executed): the executed-work model (sweep_work with the
        state's flat-interface and distinct-cell counts) over the unit-count
        FP64 peak;
      frac_method: the method's per-interface work with every interface and
        every cell evaluated in full (no flat-interface or repeated-cell
        shortcut) over the same peak -- above 1 where the shortcuts skip
        most of the work;
      *_probe: the executed work over the measured FMA-probe rate;
      *_hbm_frac: the compulsory bytes over the measured copy bandwidth.
    Work from the selections and flat-interface counts of U."""
    import torch
    T = enomr.num_tested(order)
    nsx = 8 * n * (n + 1)
    sel = solver.selection(U)
    hx = torch.bincount(sel[:nsx].long(), minlength=T + 3).cpu().numpy()
    hy = torch.bincount(sel[nsx:].long(), minlength=T + 3).cpu().numpy()
    nint = n * (n + 1)
    work = {"x": (sweep_work(order, 4, hx, nint, sweep_counts(U, 0, order)),
                  sweep_work(order, 4, hx, nint, (0, 0, 0, n * n))),
            "y": (sweep_work(order, 4, hy, nint, sweep_counts(U, 1, order), stage_epilogue=True),
                  sweep_work(order, 4, hy, nint, (0, 0, 0, n * n), stage_epilogue=True))}
    out = {}
    for kind, key in ((1, "x"), (2, "y")):
        Uc = U.clone()
        solver.profile_begin(kind, 3 * steps)
        for _ in range(steps):
            solver.step(Uc, 0.0, cfl)
        nl, ms = solver.profile_end()
        avg = ms / max(nl, 1)
        (fl, ops), (mfl, mops) = work[key]
        out[key] = round(ops / (avg * 1e-3) / peak_ops, 4)
        out[key + "_ms"] = round(avg, 4)
        out[key + "_method"] = round(mops / (avg * 1e-3) / peak_ops, 4)
        if probe_ops:
            out[key + "_probe"] = round(ops / (avg * 1e-3) / probe_ops, 4)
        if ms > 0:  # the same launches against the measured copy bandwidth
            out[key + "_hbm_frac"] = hbm_side(n, kind - 1, avg)["frac"]
        del Uc
    return out


def scalar_work(order, sel, n, staged_ops):
    """Executed FP64 operations of one scalar (advection or Burgers) launch
    on n cells: per interface the staged split value (staged_ops), the
    baseline indicator (6), the indicators of the tested candidates up to
    the chosen one (|S| each), the reconstruction (2g-1 for a tested
    stencil, 1 for minmod), the flux difference (2) and the stage update
    (7/3: the mean of the three SSP-RK3 stages, U + dt D in the first with
    1 fma, 2 fma and 1 mul in the others); only the window that carries the
    flux (f^+ for a > 0, u > 0) is evaluated.  sel: histogram of that
    side's selections."""
    import oracle  # table sizes only
    g = (order + 1) // 2
    T = oracle.num_tested(order)
    sizes = np.array([oracle.candidate(order, t)[0] + oracle.candidate(order, t)[1] + 1
                      for t in range(T)], dtype=np.float64)
    cum = np.cumsum(sizes)
    cnt = np.asarray(sel, dtype=np.float64)
    w = float(n + 1) * (staged_ops + 6) + float(n) * (2 + 7 / 3)
    for t in range(T):
        w += cnt[t] * (cum[t] + (2 * g - 1))
    w += (cnt[T] + cnt[T + 1]) * (cum[-1] + 1) + cnt[T + 2] * 1
    return w


def paper_run(enomr, dev, name, U0, dx, dy, order, sides, gravity, gamma, cfl, t_end,
              occupancy="auto"):
    """One of the paper's 2D problems from t = 0 to t_end with CFL steps
    (each step reads its dt back to the host); host-timed whole run.  A run
    that turns non-physical stops and says so."""
    import torch
    ny, nx = U0.shape[1:]
    s = enomr.Solver(enomr.EULER, (ny, nx), order=order, dx=dx, dy=dy,
                     bc=enomr.TRANSMISSIVE, gamma=gamma, device=dev)
    if sides is not None:
        s.set_sides(sides)
    if gravity != (0.0, 0.0):
        s.set_body_force(*gravity)
    s.set_occupancy({"auto": enomr.OCCUPANCY_AUTO, "high": enomr.OCCUPANCY_HIGH,
                     "low": enomr.OCCUPANCY_LOW}[occupancy])
    U = torch.from_numpy(U0).to(dev)
    s.step(U.clone(), 1e-9)  # warm-up
    s.time = 0.0
    torch.cuda.synchronize()
    t, n = 0.0, 0
    t0 = time.perf_counter()
    while t < t_end and n < 200000:
        dt = min(s.cfl_dt(U, cfl), t_end - t)
        if not dt > 0.0:  # non-physical state: stop
            break
        s.step(U, dt=dt)
        t += dt
        n += 1
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    try:
        s.check_status()
        status = "ok"
    except enomr.EnomrError as e:
        status = str(e)
    s.close()
    return {"workload": f"{name}, order {order}, CFL {cfl}, t = 0 -> {t_end}",
            "steps": n, "t_reached": t, "status": status, "wall_s": round(el, 3),
            "occupancy": occupancy,
            "unit": UNIT, "value": nx * ny * 3 * n / el,
            "note": "host-timed whole run; each step reads its CFL dt back to the host"}


def hbm_side(n, dom, avg_ms):
    """The dominant sweep against HBM: its compulsory bytes per launch (x
    sweep: read U, write D; y sweep: read U, D and U^n, write the stage
    output, U^n = U in the first of the three stages) over its mean launch
    time, and that rate over the measured copy bandwidth."""
    state = 4 * 8 * n * n
    compulsory = 2 * state if dom == 0 else state * (3 + 4 + 4) / 3.0
    rate = compulsory / (avg_ms * 1e-3) / 1e9
    peak = None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            peak = json.load(f).get("hbm_gbs")
    return {"compulsory_bytes_per_launch": compulsory, "achieved_gbs": round(rate, 1),
            "peak_gbs": peak, "frac": round(rate / peak, 4) if peak else None,
            "peak_source": "measured copy bandwidth" if peak else None}


def end_to_end(s, U0, U, cells, a, nsnap=10):
    """The public step with host buffers: every step copies its input state
    from pinned host memory and reads its result back.  The inputs are
    snapshots of the timed trajectory (block j of steps/nsnap steps starts
    from the state at its first step), so the steps cost what the
    trajectory's steps cost.  The steps are independent problems, so the
    copies run double-buffered on two copy streams and overlap the compute of
    the neighbouring steps, as a caller streaming problems through one solver
    would run them.  The serial form (copy in, step, copy out on one stream)
    is timed beside it."""
    import torch
    dev = U.device
    m = -(-a.steps // nsnap)
    Ut = torch.from_numpy(U0).to(dev)
    snaps = []
    for k in range(a.steps):
        if k % m == 0:
            h = torch.empty(Ut.shape, dtype=Ut.dtype, pin_memory=True)
            h.copy_(Ut)
            snaps.append(h)
        s.step(Ut, 0.0, a.cfl)
    del Ut
    Uh_out = [torch.empty(U.shape, dtype=U.dtype, pin_memory=True) for _ in range(2)]
    bufs = [torch.empty_like(U) for _ in range(2)]
    comp = torch.cuda.current_stream(dev)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()  # noqa: E731
    loaded, stepped, freed = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for b in range(2):
        freed[b].record(comp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(a.steps):
        b = k % 2
        with torch.cuda.stream(s_in):
            s_in.wait_event(freed[b])           # the read-back of step k-2 is done
            bufs[b].copy_(snaps[k // m], non_blocking=True)
            loaded[b].record(s_in)
        comp.wait_event(loaded[b])
        s.step(bufs[b], 0.0, a.cfl)
        stepped[b].record(comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(stepped[b])
            Uh_out[b].copy_(bufs[b], non_blocking=True)
            freed[b].record(s_out)
    torch.cuda.synchronize()
    overlapped = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k in range(a.steps):
        bufs[0].copy_(snaps[k // m], non_blocking=True)
        s.step(bufs[0], 0.0, a.cfl)
        Uh_out[0].copy_(bufs[0], non_blocking=True)
    torch.cuda.synchronize()
    serial = time.perf_counter() - t0
    return {"value": cells * 3 * a.steps / serial, "unit": UNIT,
            "h2d_bytes_per_step": U.numel() * 8,
            "d2h_bytes_per_step": Uh_out[0].numel() * 8,
            "inputs": f"{len(snaps)} snapshots of the timed trajectory, each the input of "
                      f"{m} consecutive steps",
            "copies": "value: one problem at a time, copy in, step, copy out on one stream; "
                      "overlapped_value: the steps' copies double-buffered on two copy "
                      "streams, overlapping the neighbouring steps' compute; both host-timed "
                      "over all steps",
            "overlapped_value": cells * 3 * a.steps / overlapped}


def paper_runs(enomr, workloads, dev, R, occupancy="auto"):
    """The paper's 2D problems (Sec. 4.4), whole runs with their CFL steps."""
    out = {}
    U1, d1, _ = workloads.riemann2d_rp1(801)
    out["paper_rp1_801"] = paper_run(enomr, dev, "2D Riemann RP1, 801^2", U1, d1, d1, R,
                                     None, (0.0, 0.0), 1.4, 0.3, 1.0, occupancy)
    Ud_, ddx, ddy, dsides = workloads.double_mach(1200, 300)
    out["paper_double_mach"] = paper_run(enomr, dev, "double Mach reflection, 1200x300",
                                         Ud_, ddx, ddy, R, dsides, (0.0, 0.0), 1.4, 0.1, 0.2,
                                         occupancy)
    Ur_, rdx, rdy, rsides = workloads.rayleigh_taylor(200, 800)
    out["paper_rayleigh_taylor"] = paper_run(enomr, dev, "Rayleigh-Taylor, 200x800",
                                             Ur_, rdx, rdy, R, rsides, (0.0, 1.0),
                                             5.0 / 3.0, 0.3, 1.95, occupancy)
    return out


def aggregate_ranks(ms_local, cell_updates_per_rank, device):
    """Whole-job rate of independent replicas: the max over ranks of the
    timed region (ms) and all ranks' cell-updates divided by it."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    ms_max = float(t.item())
    return ms_max, world * cell_updates_per_rank / (ms_max * 1e-3)


def vortex_rate(enomr, workloads, dev, a):
    """Smooth workload (no flat windows): isentropic vortex, periodic, CFL
    steps; W warm-up steps, then K timed steps."""
    import torch
    Uv, hv, _ = workloads.isentropic_vortex(a.n)
    sv = enomr.Solver(enomr.EULER, (a.n, a.n), order=a.order, dx=hv, dy=hv,
                      bc=enomr.PERIODIC, device=dev)
    U = torch.from_numpy(Uv).to(dev)
    for _ in range(a.warmup):
        sv.step(U, 0.0, a.cfl)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(a.steps):
        sv.step(U, 0.0, a.cfl)
    f1.record()
    torch.cuda.synchronize()
    sv.check_status()
    sv.close()
    return {"workload": f"isentropic vortex {a.n}^2 periodic, order {a.order}",
            "value": a.n * a.n * 3 * a.steps / (f0.elapsed_time(f1) * 1e-3), "unit": UNIT,
            "ms_per_step": f0.elapsed_time(f1) / a.steps}


def timed_steps(solver, U, steps, dt=0.0, cfl=0.5):
    """ms of `steps` steps of solver on U (CUDA events on the current stream)."""
    import torch
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(steps):
        solver.step(U, dt, cfl)
    f1.record()
    torch.cuda.synchronize()
    return f0.elapsed_time(f1)


def rate_of(solver, Ustate, steps=2, dt=0.0, cfl=0.5):
    """cell-updates/s per RK stage of `steps` steps after one warm-up step."""
    import torch
    solver.step(Ustate, dt, cfl)
    torch.cuda.synchronize()
    ms = timed_steps(solver, Ustate, steps, dt, cfl)
    cells = Ustate[0].numel() if Ustate.dim() > 1 else Ustate.numel()
    return cells * 3 * steps / (ms * 1e-3)


def small_configs(enomr, workloads, dev):
    """The paper-sized 1D runs, which are latency-bound: advection N = 200
    (orders 5, 7, 9, the sine and the unit step, CFL 0.5) and the
    shock/entropy-wave interaction at N = 400, 1600, 6400 (orders 5, 9, 13,
    17, CFL steps on the device).  Each: microseconds per SSP-RK3 step and
    cell-updates/s per RK stage, from a plain stream of 200 steps and from a
    CUDA graph of 50 steps replayed 4 times (launch overhead removed)."""
    import torch

    def measure(solver, U, dt):
        for _ in range(3):
            solver.step(U, dt, 0.5)
        torch.cuda.synchronize()
        ms_stream = timed_steps(solver, U, 200, dt) / 200
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            solver.step(U, dt, 0.5)
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            for _ in range(50):
                solver.step(U, dt, 0.5)
        gr.replay()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(4):
            gr.replay()
        f1.record()
        torch.cuda.synchronize()
        ms_graph = f0.elapsed_time(f1) / 200
        cells = U.shape[-1]
        return {"us_per_step_stream": round(ms_stream * 1e3, 2),
                "us_per_step_graph": round(ms_graph * 1e3, 2),
                "value_graph": cells * 3 / (ms_graph * 1e-3)}

    out = {"config1_advection_200": {}, "config2_shock_entropy": {}, "unit": UNIT}
    for R in (5, 7, 9):
        for kind in ("sine", "step"):
            u, h = (workloads.advection_sine(200) if kind == "sine"
                    else workloads.advection_step(200))
            sa = enomr.Solver(enomr.ADVECTION, 200, order=R, dx=h, bc=enomr.PERIODIC, device=dev)
            out["config1_advection_200"][f"R{R}_{kind}"] = measure(
                sa, torch.from_numpy(u).to(dev), 0.5 * h)
            sa.close()
    for N in (400, 1600, 6400):
        for R in (5, 9, 13, 17):
            U, h = workloads.shock_entropy(N)
            se = enomr.Solver(enomr.EULER, N, order=R, dx=h, bc=enomr.TRANSMISSIVE, device=dev)
            out["config2_shock_entropy"][f"N{N}_R{R}"] = measure(se, torch.from_numpy(U).to(dev),
                                                                 0.0)
            se.close()
    return out


def scalar_fracs(enomr, workloads, dev, peak_ops, hbm_peak):
    """Scalar advection (sin(pi x)) and Burgers (1 + 0.5 sin^3(pi x)) at
    N = 2^24, orders 5, 9, 17: rate, the kernel's mean launch time, its
    executed FP64 work (scalar_work) over the unit-count peak, and its
    compulsory bytes (read U^(s) and U^n, write the stage: 24 B per cell)
    over the measured copy bandwidth."""
    import torch
    N = 1 << 24
    out = {}
    for name, eq, make, staged in (("advection_2p24", enomr.ADVECTION, workloads.advection_sine, 1),
                                   ("burgers_2p24", enomr.BURGERS, workloads.burgers_sine3, 2)):
        vals = {}
        for R in (5, 9, 17):
            u, h = make(N)
            sv = enomr.Solver(eq, N, order=R, dx=h, bc=enomr.PERIODIC, device=dev)
            ud = torch.from_numpy(u).to(dev)
            dt = 0.5 * h if eq == enomr.ADVECTION else 0.0
            rate = rate_of(sv, ud, steps=4, dt=dt)
            sel = sv.selection(ud)
            T = enomr.num_tested(R)
            hist = torch.bincount(sel[:N + 1].long(), minlength=T + 3).cpu().numpy()
            ops = scalar_work(R, hist, N, staged)
            sv.profile_begin(1, 12)
            timed_steps(sv, ud, 4, dt)
            nl, ms = sv.profile_end()
            avg = ms / max(nl, 1)
            vals[str(R)] = {"value": rate, "kernel_ms": round(avg, 4),
                            "fp64_op_frac": round(ops / (avg * 1e-3) / peak_ops, 4),
                            "hbm_frac": (round(24.0 * N / (avg * 1e-3) / 1e9 / hbm_peak, 4)
                                         if hbm_peak else None)}
            sv.close()
        out[name] = {"workload": f"{name.split('_')[0]}, N = 2^24, periodic, SSP-RK3",
                     "unit": UNIT, "values": vals}
    return out


def per_order_vortex(enomr, workloads, dev, n, cfl, peak_ops, probe_ops):
    """The long path at every order: the isentropic vortex (no flat windows)
    on n^2 with the library's setting for smooth data (low-occupancy sweeps,
    TMA staging): rate (1 warm-up + 2 timed steps) and both sweeps'
    fractions; `value_default` is the rate with the default settings."""
    import torch
    Uv, hv, _ = workloads.isentropic_vortex(n)
    out = {}
    for R in enomr.ORDERS:
        sv = enomr.Solver(enomr.EULER, (n, n), order=R, dx=hv, dy=hv, bc=enomr.PERIODIC,
                          device=dev)
        U = torch.from_numpy(Uv).to(dev)
        default = rate_of(sv, U.clone(), cfl=cfl)
        sv.set_occupancy(enomr.OCCUPANCY_LOW)
        sv.set_staging(enomr.STAGING_TMA)
        out[str(R)] = {"value": rate_of(sv, U.clone(), cfl=cfl), "value_default": default,
                       **sweep_fracs(enomr, sv, U, R, n, cfl, peak_ops, probe_ops=probe_ops)}
        sv.close()
        del U
    return {"workload": f"isentropic vortex {n}^2 periodic (every interface on the long path)",
            "setting": "enomr_set_occupancy LOW + enomr_set_staging TMA (the smooth-data "
                       "setting); value_default: automatic settings",
            "unit": UNIT, "orders": out}


def riemann_sizes(enomr, workloads, dev, cfl, steps=20):
    """The four-quadrant Riemann workload at 1024^2 and 2048^2 (orders 9
    and 17): rate of `steps` CFL steps from t = 0 after one warm-up step."""
    import torch
    out = {}
    for n in (1024, 2048):
        U0, dx, dy = workloads.riemann2d(n, n, seed=0)
        for R in (9, 17):
            sk = enomr.Solver(enomr.EULER, (n, n), order=R, dx=dx, dy=dy,
                              bc=enomr.TRANSMISSIVE, device=dev)
            U = torch.from_numpy(U0).to(dev)
            sk.step(U.clone(), 0.0, cfl)
            ms = timed_steps(sk, U, steps, cfl=cfl)
            out[f"{n}_R{R}"] = {"value": n * n * 3 * steps / (ms * 1e-3),
                                "ms_per_step": round(ms / steps, 4)}
            sk.close()
    return {"unit": UNIT, "run": f"{steps} CFL steps from t = 0", "values": out}


def staging_ab(enomr, s, U0, dev, steps, cfl):
    """The same trajectory (`steps` CFL steps from t = 0) with the sweeps'
    tiles staged by TMA (the library's default where the state allows it)
    and with plain loads: each sweep's mean launch time and the step time.
    Both give the same bits."""
    import torch
    out = {}
    for name, mode in (("tma", enomr.STAGING_TMA), ("loads", enomr.STAGING_LOADS)):
        s.set_staging(mode)
        r = {}
        for kind, key in ((1, "x_ms"), (2, "y_ms")):
            U = torch.from_numpy(U0).to(dev)
            s.profile_begin(kind, 3 * steps)
            for _ in range(steps):
                s.step(U, 0.0, cfl)
            nl, ms = s.profile_end()
            r[key] = round(ms / max(nl, 1), 4)
        U = torch.from_numpy(U0).to(dev)
        r["step_ms"] = round(timed_steps(s, U, steps, cfl=cfl) / steps, 4)
        out[name] = r
    s.set_staging(enomr.STAGING_AUTO)
    out["tma_vs_loads_step"] = round(out["loads"]["step_ms"] / out["tma"]["step_ms"], 4)
    return out


def main_ours(a):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_15504_gb300 import enomr, workloads

    clk = ClockSampler(local)
    clk.start()
    n, R = a.n, a.order
    U0, dx, dy = workloads.riemann2d(n, n, seed=rank)
    s = enomr.Solver(enomr.EULER, (n, n), order=R, dx=dx, dy=dy, bc=enomr.TRANSMISSIVE,
                     device=dev)
    U = torch.from_numpy(U0).to(dev)
    for _ in range(a.warmup):
        s.step(U, 0.0, a.cfl)
    U.copy_(torch.from_numpy(U0))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s.profile_begin(1, 3 * a.steps)  # x sweep: timed live during the run
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clk.mark("timed_start")
    e0.record()
    for _ in range(a.steps):
        s.step(U, 0.0, a.cfl)
    e1.record()
    torch.cuda.synchronize()
    time.sleep(0.12)  # let the sampler take the region's last samples
    clk.mark("timed_end")
    ms = e0.elapsed_time(e1)
    nx_launch, x_ms = s.profile_end()
    s.check_status()
    cells = n * n
    ms_max, value = aggregate_ranks(ms, cells * 3 * a.steps, dev)
    launches_per_step = 1 + 3 + 2 * 3  # dt, 3 alpha reductions, 2 sweeps x 3 stages

    extras = {}
    U_final = U
    if rank == 0 and not a.no_extras:
        # y sweep and alpha, timed over the same trajectory right after the run
        Uy = torch.from_numpy(U0).to(dev)
        s.profile_begin(2, 3 * a.steps)
        for _ in range(a.steps):
            s.step(Uy, 0.0, a.cfl)
        ny_launch, y_ms = s.profile_end()
        Uy.copy_(torch.from_numpy(U0))
        s.profile_begin(3, 3 * a.steps)
        for _ in range(a.steps):
            s.step(Uy, 0.0, a.cfl)
        na_launch, a_ms = s.profile_end()
        del Uy
        # algorithmic work of a sweep: selection histograms and flat-interface
        # counts of the step states of the same trajectory (U^n of every
        # sampled step stands in for its three stage states), averaged
        T = enomr.num_tested(R)
        nsx = 8 * n * (n + 1)
        every = max(1, a.steps // 20)
        Us = torch.from_numpy(U0).to(dev)
        hx = np.zeros(T + 3)
        hy = np.zeros(T + 3)
        cx = np.zeros(5)
        cy = np.zeros(5)
        ns = 0
        for it in range(a.steps):
            if it % every == 0:
                sel = s.selection(Us)
                hx += torch.bincount(sel[:nsx].long(), minlength=T + 3).cpu().numpy()
                hy += torch.bincount(sel[nsx:].long(), minlength=T + 3).cpu().numpy()
                cx += np.array(sweep_counts(Us, 0, R))
                cy += np.array(sweep_counts(Us, 1, R))
                ns += 1
            s.step(Us, 0.0, a.cfl)
        hx, hy, cx, cy = hx / ns, hy / ns, cx / ns, cy / ns
        del Us
        nint = n * (n + 1)
        wx = sweep_work(R, 4, hx, nint, cx)
        wy = sweep_work(R, 4, hy, nint, cy, stage_epilogue=True)
        mx = sweep_work(R, 4, hx, nint, (0, 0, 0, n * n))
        my = sweep_work(R, 4, hy, nint, (0, 0, 0, n * n), stage_epilogue=True)
        extras["flat_interface_fraction"] = [cx[0] / nint, cy[0] / nint]
        extras["distinct_cell_fraction"] = [cx[3] / (n * n), cy[3] / (n * n)]
        probe, probe_ops = probe_ops_peak(enomr, dev)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        clocks_t = clk.summary("timed_start", "timed_end")
        mhz = clocks_t.get("sm_mhz") or clocks_t.get("sm_max_mhz") or 2070.0
        # 2 FP64 lanes per SM per clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
        # peak_sustained = 2 / SM / cycle; DMUL and DADD take the same slots), at the
        # median SM clock of the timed region
        peak_ops = 2.0 * sms * mhz * 1e6
        x_avg = x_ms / max(nx_launch, 1)
        y_avg = y_ms / max(ny_launch, 1)
        if x_avg >= y_avg:
            dom, avg, (fl, ops), (mfl, mops) = 0, x_avg, wx, mx
        else:
            dom, avg, (fl, ops), (mfl, mops) = 1, y_avg, wy, my
        kname = f"k_sweep_tma<{R},{dom}>"
        achieved = ops / (avg * 1e-3)
        extras["roofline"] = {
            "bound": "alu", "pipe": "fp64", "kernel": kname,
            "achieved": round(achieved / 1e9, 2), "peak": round(peak_ops / 1e9, 2),
            "unit": "GFP64op/s", "frac": round(achieved / peak_ops, 4),
            "frac_executed": round(achieved / peak_ops, 4),
            "frac_method": round(mops / (avg * 1e-3) / peak_ops, 4),
            "frac_definitions": {
                "frac_executed": "the work the kernel executes (flat interfaces on one state "
                                 "take the cell's flux, repeated cells copy their "
                                 "representative's values, tiles on one state per line "
                                 "skip the flux difference), over the unit-count peak",
                "frac_method": "the method's per-interface work with every interface and "
                               "cell evaluated in full, over the same peak; above 1 where "
                               "the shortcuts skip most of it"},
            "peak_source": (f"unit counts x clock: 2 FP64 ops/clk/SM x {sms} SMs x "
                            f"{mhz:.0f} MHz (median SM clock of the timed region)"),
            "op_definition": "fma, mul, add, div, rsqrt = 1 FP64 operation each",
            "fp64_fma_probe_tflops": round(probe / 1e12, 4),
            "frac_of_probe": round(achieved / probe_ops, 4),
            "traffic": recorded_traffic(kname, n, R),
            "avg_launch_ms": round(avg, 4), "algorithmic_ops_per_launch": ops,
            "method_ops_per_launch": mops,
            "algorithmic_flops_per_launch": fl,
            "achieved_tflops": round(fl / (avg * 1e-3) / 1e12, 4),
            "x_sweep_ms": round(x_avg, 4), "y_sweep_ms": round(y_avg, 4),
            "x_sweep_frac": round(wx[1] / (x_avg * 1e-3) / peak_ops, 4),
            "y_sweep_frac": round(wy[1] / (y_avg * 1e-3) / peak_ops, 4),
            "x_sweep_frac_method": round(mx[1] / (x_avg * 1e-3) / peak_ops, 4),
            "y_sweep_frac_method": round(my[1] / (y_avg * 1e-3) / peak_ops, 4),
            "alpha_ms": round(a_ms / max(na_launch, 1), 4),
            "hbm": hbm_side(n, dom, avg)}
        extras["selection_histogram_x"] = [round(float(v)) for v in hx]
        extras["work_samples"] = ns
        extras["staging_ab"] = staging_ab(enomr, s, U0, dev, min(a.steps, 10), a.cfl)
        per_order, per_order_frac = {}, {}
        for Rk in enomr.ORDERS:
            sk = enomr.Solver(enomr.EULER, (n, n), order=Rk, dx=dx, dy=dy,
                              bc=enomr.TRANSMISSIVE, device=dev)
            Uk = torch.from_numpy(U0).to(dev)
            per_order[str(Rk)] = rate_of(sk, Uk, cfl=a.cfl)
            per_order_frac[str(Rk)] = sweep_fracs(enomr, sk, Uk, Rk, n, a.cfl, peak_ops,
                                                  probe_ops=probe_ops)
            sk.close()
            del Uk
        extras["per_order_riemann"] = {"unit": UNIT, "values": per_order,
                                       "fp64_op_frac": per_order_frac,
                                       "run": "1 warm-up + 2 timed steps from t = 0; "
                                              "fractions over the next 2 steps"}
        extras["per_order_vortex"] = per_order_vortex(enomr, workloads, dev, n, a.cfl, peak_ops,
                                                      probe_ops)
        extras["riemann_sizes"] = riemann_sizes(enomr, workloads, dev, a.cfl)
    if rank == 0 and not a.no_extras and a.paper_runs:
        extras.update(paper_runs(enomr, workloads, dev, R, a.occupancy))
    if rank == 0 and not a.no_extras:
        hbm_peak = hbm_side(n, 0, 1.0)["peak_gbs"]
        extras.update(scalar_fracs(enomr, workloads, dev, peak_ops, hbm_peak))
        extras["small_configs"] = small_configs(enomr, workloads, dev)
        extras["batched"] = batched_gain(enomr, workloads, dev, a)
        extras["adjoint"] = {"n512": adjoint_ratio(enomr, workloads, dev, n=512),
                             "n1024": adjoint_ratio(enomr, workloads, dev, n=1024)}
        extras["e2e"] = end_to_end(s, U0, U, cells, a)
    clocks_all = clk.stop()
    clocks = clk.summary("timed_start", "timed_end")
    clocks["whole_run"] = clocks_all

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic (seeded four-quadrant Riemann states)",
               "config": config(a), "clocks": clocks,
               "gpu_launches": launches_per_step * a.steps}
        out.update(extras)
        if not a.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(a)
            out["parity"] = parity_check(a, enomr, s, U_final, dx, dy)
        print(json.dumps(out), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure)
# ---------------------------------------------------------------------------
def _oracle_problem(a, m):
    """The same workload on an m x m grid (m = n: the full grid)."""
    import oracle
    from paper_2311_15504_gb300 import workloads
    U0, dx, dy = workloads.riemann2d(m, m, seed=0)
    P = oracle.Problem(oracle.EQ_EULER2D, a.order, m, m, dx=dx, dy=dy,
                       bc=oracle.BC_TRANSMISSIVE)
    return P, U0


def _oracle_rate_estimate(a):
    """seconds per cell of one oracle RHS with all threads (512^2 probe)."""
    P, U0 = _oracle_problem(a, 512)
    t0 = time.perf_counter()
    P.rhs(U0)
    return (time.perf_counter() - t0) / (512 * 512)


def cpu_baseline(a, budget_s=20.0):
    import oracle
    per_cell = _oracle_rate_estimate(a)
    m = a.n
    while 3 * per_cell * m * m > budget_s and m > 256:
        m //= 2
    P, U0 = _oracle_problem(a, m)
    dt = P.cfl_dt(U0, a.cfl)
    t0 = time.perf_counter()
    P.step_ssprk3(U0, dt)
    el = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same step on one host thread, on a grid a quarter of the size
    # (results are bitwise the same for any thread count)
    m1 = max(m // 4, 128)
    P1, U1 = _oracle_problem(a, m1)
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        P1.step_ssprk3(U1, P1.cfl_dt(U1, a.cfl))
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    return {"value": m * m * 3 / el, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"one oracle SSP-RK3 step (3 stages) of the same workload on a "
                      f"{m}x{m} grid ({el:.1f} s wall)",
            "single_thread": {"value": m1 * m1 * 3 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"one step on a {m1}x{m1} grid ({el1:.1f} s wall)"}}


def parity_check(a, enomr, s, U, dx, dy):
    """The CUDA path against the oracle on the final state of the timed run
    (seed 0, the full grid; part of the CPU leg): selection flips of one
    right-hand side (every interface, field and side of both sweeps) and the
    largest difference of the right-hand side against the oracle re-run
    with the CUDA path's selections, relative to max(||L||, ||F||/h)."""
    import oracle
    t0 = time.perf_counter()
    sel = s.selection(U).cpu().numpy()
    rhs = s.rhs(U).cpu().numpy()
    Uh = U.cpu().numpy()
    ref = oracle.rhs_euler2d(Uh, dx, dy, a.order, bc=oracle.BC_TRANSMISSIVE, want_sel=True)
    flips = int((ref["sel"] != sel).sum())
    forced = oracle.rhs_euler2d(Uh, dx, dy, a.order, bc=oracle.BC_TRANSMISSIVE, forced=sel)["rhs"]
    rho, mx, my, E = Uh
    u, v = mx / rho, my / rho
    p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    fscale = max(float(np.abs(mx).max()), float(np.abs(my).max()),
                 float(np.abs(mx * u + p).max()), float(np.abs(my * v + p).max()),
                 float(np.abs((E + p) * u).max()), float(np.abs((E + p) * v).max()))
    lnorm = float(np.abs(forced).max())
    err = float(np.abs(rhs - forced).max())
    return {"state": f"final state of the timed run ({a.steps} steps, seed 0, {a.n}^2)",
            "selection_flips": flips, "selections": int(sel.size),
            "rhs_max_abs_diff": err,
            "rhs_rel_diff": err / max(lnorm, fscale / min(dx, dy)),
            "rhs_rel_diff_vs_L": err / lnorm if lnorm > 0 else 0.0,
            "wall_s": round(time.perf_counter() - t0, 1)}


def main_reference(a):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    per_cell = _oracle_rate_estimate(a)
    budget = 150.0 / max(a.steps + a.warmup, 1)  # seconds per step
    m = a.n
    while 3 * per_cell * m * m > budget and m > 128:
        m //= 2
    P, U0 = _oracle_problem(a, m)
    U = U0.copy()
    dt = P.cfl_dt(U0, a.cfl)
    for _ in range(a.warmup):
        U = P.step_ssprk3(U, dt)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        U = P.step_ssprk3(U, dt)
    el = time.perf_counter() - t0
    value = m * m * 3 * a.steps / el
    cores = oracle.num_threads()
    sample = (f"each step: one oracle SSP-RK3 step of the workload on a {m}x{m} grid "
              f"(full size {a.n}x{a.n}); fixed dt")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": el * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(a),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main_only(a):
    import torch
    from paper_2311_15504_gb300 import enomr, workloads
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if a.only == "adjoint":
        out = adjoint_ratio(enomr, workloads, dev, n=a.n, steps=a.steps)
    elif a.only == "vortex":
        out = vortex_rate(enomr, workloads, dev, a)
    elif a.only == "paper":
        out = paper_runs(enomr, workloads, dev, a.order, a.occupancy)
    else:
        out = batched_gain(enomr, workloads, dev, a)
    print(json.dumps({"only": a.only, **out}), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.only:
        main_only(args)
    elif args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)
