"""Benchmark of the GB300 Fock-exchange path: band-pair applications per second.

One step = one full pass of the exchange path over the beta-boron-sized
workload (96^3 grid, Gamma-centred 2x2x2 mesh, 160 occupied / 192 target
bands: 1,966,080 band pairs): sphere->grid of every orbital, the three fused
band-pair passes for every (k, q, target batch, occupied batch), grid->sphere
of V_x c and the E_x reduction, all through the C ABI (xx_energy).

Printed as one JSON line (rank 0):
  value      band pairs / s with inputs resident in HBM (CUDA events, K steps)
  e2e        the same through the public API with pinned host buffers: H2D of
             the orbitals and occupations, xx_energy, D2H of V_x c and E_x
  roofline   the dominant kernel's algorithmic bytes per launch over its mean
             launch duration (events on its stream during the timed steps),
             against the measured HBM copy bandwidth
  cpu_baseline  the FP64 CPU oracle, as it stands, on a bounded sample
  fp64       the all-FP64 GPU path on one target k-point at the production batch
             shape, with its ALU fraction against the measured FP64 FMA rate
  parity     the CUDA path (both precisions) against the oracle on the
             cpu_baseline sample
  real_gamma    the real-orbital Gamma path against the general path on the same
                cell at the Gamma point only (real orbitals, 30,720 pairs)
  exact_grid    the same workload with the plan on the smallest grid on which the
                operator is exact (60^3; same V_x c and E_x up to rounding)
  alpha_boron   the alpha-boron-sized workload (48^3, 64 k-points, 1.77 M pairs)
  sweep_cells   six uneven Gamma cells in one launch per band-pair pass, against
                one plan per cell on concurrent streams
  --impl reference  times the oracle as the reference arm.
Multi-GPU (torchrun): one workload sharded over the ranks by k-point blocks
{k, q} (xx_set_shard): every step, rank 0 broadcasts the orbitals (NCCL), each
rank applies the blocks it owns, the partial V_x c are all-reduced and the E_x
shares summed in rank order; strong scaling, value = the workload's pairs / the
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "band-pair exchange applications/s and % HBM roofline, FP32-mixed vs FP64 GPU"
UNIT = "band-pair applications/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.index = index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_beta_boron_96.json")


def kernel_source_hash():
    """Hash of the sources of the single-cell kernels (the passes, their FFT building
    blocks and launchers, and the per-length translation units; not the host loops of
    xx_api.cu nor the batched multi-cell kernels): recorded DRAM traffic per launch is
    only valid for these kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1111_0716_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in ("xx_launch.cuh", "xx_kernels.cuh", "xx_fft.cuh",
                                             "xx_roots.cuh")] + \
        glob.glob(os.path.join(csrc, "xx_n*.cu"))
    for f in sorted(files):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, batch):
    """DRAM bytes per transformed band pair of a pass from the committed ncu summary,
    or None when stale (other kernel sources or another batch shape)."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash() or list(d.get("batch", [])) != list(batch):
        return None
    return d.get("bytes_per_pair", {}).get(kernel)


def batch_schedule(nk, n_occ, n_tgt, TA, TJ, G_max=1, sym=True, cross=True, owned=None):
    """The band-pair launches of one xx_energy call with shared grids, in the
    host loop's order: (kind, targets, occupied) with kind "full" (passes A, B,
    C) or "mirrored" (passes A, B, C and the role-swapped pass C).  G_max is the
    plan's q_per_batch: that many k-points' whole occupied sets share a batch;
    target batches are cut at n_occ (the split of the grids' layout).  owned(k, q):
    whether the plan's shard owns block {k, q} (None: every block)."""
    out = []
    T = min(TA, TJ)
    sym = sym and n_occ > 1
    own = owned or (lambda k, q: True)

    def run_q(q_lo, q_hi, a_lo, a_hi, mirrored):
        if a_lo >= a_hi:
            return
        q0 = q_lo
        while q0 < q_hi:
            G = min(G_max, q_hi - q0)
            cut = n_occ if a_lo < n_occ < a_hi else a_hi
            for lo, hi in ((a_lo, cut), (cut, a_hi)):
                for a0 in range(lo, hi, TA):
                    ta = min(TA, hi - a0)
                    jstep = n_occ if G > 1 else TJ
                    for j0 in range(0, n_occ, jstep):
                        nj = min(jstep, n_occ - j0)
                        out.append(("mirrored" if mirrored else "full", ta, G * nj))
            q0 += G

    for k in range(nk):
        def run_owned(q_lo, q_hi, a_lo, a_hi, mirrored):
            q = q_lo
            while q < q_hi:
                if not own(k, q):
                    q += 1
                    continue
                q_end = q + 1
                while q_end < q_hi and own(k, q_end):
                    q_end += 1
                run_q(q, q_end, a_lo, a_hi, mirrored)
                q = q_end

        if not sym:
            run_owned(0, nk, 0, n_tgt, False)
            continue
        if own(k, k):
            for i0 in range(0, n_occ, T):
                for j0 in range(i0, n_occ, T):
                    out.append(("mirrored" if j0 > i0 else "full", min(T, n_occ - i0),
                                min(T, n_occ - j0)))
            run_q(k, k + 1, n_occ, n_tgt, False)
        if cross:
            run_owned(0, k, n_occ, n_tgt, False)
            run_owned(k + 1, nk, 0, n_occ, True)
            run_owned(k + 1, nk, n_occ, n_tgt, False)
        else:
            run_owned(0, k, 0, n_tgt, False)
            run_owned(k + 1, nk, 0, n_tgt, False)
    return out


def pass_bytes_per_step(wl, schedule, elem=8):
    """Algorithmic HBM bytes of each band-pair pass over one step.

    Per transformed band pair each pass streams one grid of N^3 complex values
    in and one out (16 B per grid point in FP32 complex): pass A reads u_j and
    writes the codensity transform, pass B reads and writes it, pass C reads it
    and u_j (the role-swapped pass C reads it and u_a).  Per launch and target
    (per occupied band for the role-swapped pass C): pass A reads u_a, pass C
    reads the FP64 accumulator and writes it back (32 B/pt).
    """
    n3 = wl.grid[0] ** 3
    a = b = c = 0
    for kind, ta, tj in schedule:
        a += (2 * elem * ta * tj + elem * ta) * n3
        b += 2 * elem * ta * tj * n3
        c += (2 * elem * ta * tj + 32 * ta) * n3
        if kind == "mirrored":
            c += (2 * elem * ta * tj + 32 * tj) * n3
    return {"pass_a": a, "pass_b": b, "pass_c": c}


def distribute_orbitals(c):
    """Rank 0's orbital coefficients (complex tensor) to every rank."""
    import torch
    import torch.distributed as dist
    dist.broadcast(torch.view_as_real(c), src=0)


def combine_shards(vx, ex, ex_parts):
    """Sum the ranks' partial V_x c (in place, every rank) and their E_x shares,
    the shares added in rank order so the total does not depend on the
    collective's reduction order (ex_parts: one 2-vector per rank, scratch)."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(torch.view_as_real(vx))
    dist.all_gather(ex_parts, ex)
    ex.copy_(ex_parts[0])
    for part in ex_parts[1:]:
        ex.add_(part)


def run_oracle_sample(wl, n_occ_sample, want_vx=False):
    """The FP64 oracle on target (k=0, a=0), all q, the first n_occ_sample occupied bands."""
    from oracle import oracle
    t0 = time.perf_counter()
    vx = oracle.apply(wl, sel=[(0, 0)], c_occ=wl.c_occ[:, :n_occ_sample],
                      w_occ=wl.w_occ[:, :n_occ_sample])
    dt = time.perf_counter() - t0
    pairs = wl.nk * n_occ_sample
    if want_vx:
        return pairs / dt, dt, pairs, oracle.num_threads(), vx
    return pairs / dt, dt, pairs, oracle.num_threads()


# Nominal flops of one transformed band pair on an N^3 grid pruned to P = 4 n_max + 1
# frequencies per axis: the line transforms the passes run (pass A: N^2 x-lines and
# N P y-lines; pass B: P^2 forward and P^2 inverse z-lines; pass C: N P y-lines and
# N^2 x-lines) at the usual 5 L log2 L flops per length-L transform, plus the
# pointwise work (codensity 6, kernel multiply 2 per kept frequency, u_j multiply and
# weighted accumulate 8 flops per point).
def flops_per_pair(N, P):
    import math
    line = 5.0 * N * math.log2(N)
    a = N * (N + P) * line + 6.0 * N ** 3
    b = 2.0 * P * P * line + 2.0 * P ** 3
    c = N * (N + P) * line + 8.0 * N ** 3
    return {"pass_a": a, "pass_b": b, "pass_c": c}


def reference_arm(args, rank, world):
    """The oracle timed as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    from paper_1111_0716_gb300 import synth
    wl = synth.beta_boron()
    n_s = args.oracle_occ
    for _ in range(args.warmup):
        run_oracle_sample(wl, max(1, n_s // 4))
    rates, total = [], 0.0
    for _ in range(args.steps):
        r, dt, pairs, cores = run_oracle_sample(wl, n_s)
        rates.append(r)
        total += dt
    value = float(np.sum([args.steps * wl.nk * n_s])) / total
    sample = ("target (k=0, a=0) x 8 q x %d occupied bands = %d pairs of the 96^3 beta-boron "
              "workload per step" % (n_s, wl.nk * n_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name + " (beta-boron-sized rhombohedral cell)", "grid": 96,
                       "nk": wl.nk, "n_occ": wl.n_occ,
                       "n_tgt": wl.n_tgt, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """beta-boron 96^3, target k=0, 64 targets x 80 occupied bands x 8 q (40960 pairs),
    in the benchmark's batch shape (64 targets x 80 occupied per launch)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import synth, xx
    if args.profile_alpha:
        wa = synth.alpha_boron()
        plan = xx.Plan.from_workload(wa, precision=xx.XX_FP32_MIXED)
        c = torch.from_numpy(wa.c_tgt).cuda()
        wo, wt = torch.from_numpy(wa.w_occ).cuda(), torch.from_numpy(wa.w_tgt).cuda()
        l0 = 0
        for step in range(2):
            if step == 1:
                l0 = plan.info()["kernel_launches"]
            plan.energy(c, wo, c, wt, shared=True)
        torch.cuda.synchronize()
        info = plan.info()
        plan.close()
        print(json.dumps({"profile_case": wa.name, "pairs_per_step": wa.pair_count(),
                          "launches_first_step": l0, "launches_second_step": info["kernel_launches"] - l0,
                          "batch": [info["targets_per_batch"], info["occupied_per_batch"]],
                          "q_per_batch": info["q_per_batch"]}))
        return
    wl = synth.beta_boron()
    if args.profile_grid:
        wl = wl.replace(grid=(args.profile_grid,) * 3)
    prec = xx.XX_FP64 if args.precision == "fp64" else xx.XX_FP32_MIXED
    if args.profile_shared:
        # the first two k-points with shared grids: k = q tiles, the pair-symmetric
        # block (0, 1) (passes A, B, C and the role-swapped pass C at 64 x 80) and
        # the targets past the occupied set
        nb = 16 if args.profile_small else wl.coeff.shape[1]
        sub = wl.replace(kfrac=wl.kfrac[:2], npw=wl.npw[:2], miller=wl.miller[:2],
                         coeff=wl.coeff[:2, :nb], w=wl.w[:2, :nb], n_occ=min(wl.n_occ, nb),
                         n_tgt=min(wl.n_tgt, nb))
        plan = xx.Plan.from_workload(sub, precision=prec)
        c = torch.from_numpy(sub.c_tgt).cuda()
        ex, vx = plan.energy(c, torch.from_numpy(sub.w_occ).cuda(), c,
                             torch.from_numpy(sub.w_tgt).cuda(), shared=True)
        torch.cuda.synchronize()
        info = plan.info()
        plan.close()
        print(json.dumps({"profile_case": sub.name + " (k-points 0, 1)", "pairs": sub.pair_count(),
                          "transformed": info["pairs_transformed"],
                          "batch": [info["targets_per_batch"], info["occupied_per_batch"]],
                          "workspace_gb": info["peak_workspace_bytes"] / 1e9}))
        return
    plan = xx.Plan.from_workload(wl, precision=prec)
    nt, no = (16, 16) if args.profile_small else (64, 80)
    if args.profile_small:
        # the bench's occupied width: 80 columns (the whole sets of 5 q-points), so the
        # FP64 accumulator update is spread over as many pairs as in the bench
        plan.set_batch(16, 80)
    co = torch.from_numpy(wl.c_occ[:, :no].copy()).cuda()
    wo = torch.from_numpy(wl.w_occ[:, :no].copy()).cuda()
    ct = torch.from_numpy(wl.c_tgt[:1, :nt].copy()).cuda()
    plan.apply_range(0, 1, co, wo, ct)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    print(json.dumps({"profile_case": wl.name, "pairs": nt * no * wl.nk,
                      "batch": [info["targets_per_batch"], info["occupied_per_batch"]],
                      "workspace_gb": info["peak_workspace_bytes"] / 1e9}))


def real_gamma_leg(xx, torch, stream, reps=3):
    """E_x step on the Gamma-only cell with real orbitals: general path (k = q pair
    symmetry) against the real-orbital path (two occupied bands per transform)."""
    from paper_1111_0716_gb300 import synth
    wl = synth.real_beta_cell()
    c = torch.from_numpy(wl.c_tgt.copy()).cuda()
    wo = torch.from_numpy(wl.w_occ.copy()).cuda()
    wt = torch.from_numpy(wl.w_tgt.copy()).cuda()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for real in (False, True):
        plan = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED)
        plan.set_real_gamma(real)
        ex, vx = plan.energy(c, wo, c, wt, shared=True, stream=stream)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            g0.record(stream)
            plan.energy(c, wo, c, wt, vx_out=vx, ex_out=ex, shared=True, stream=stream)
            g1.record(stream)
            torch.cuda.synchronize()
            ts.append(g0.elapsed_time(g1) / 1e3)
        plan.sync(timeout_s=60.0, stream=stream)
        out[real] = (float(np.median(ts)), float(ex[0].item()))
        plan.close()
    pairs = wl.pair_count()
    return {"value": pairs / out[True][0], "unit": UNIT, "general_path": pairs / out[False][0],
            "E_x_rel_diff": abs(out[True][1] - out[False][1]) / abs(out[False][1]),
            "sample": "%s: 1 k-point, %d occupied x %d targets = %d pairs, FP32-mixed, median of %d"
                      % (wl.name, wl.n_occ, wl.n_tgt, pairs, reps)}


def exact_grid_leg(xx, torch, wl, stream, e_ref, reps=2):
    """The same workload on the smallest grid on which the operator is exact
    (N >= 4 n_max + 1: 60^3 for this basis), through the same xx_energy call."""
    n = xx.xx_exact_grid(wl.n_max())
    small = wl.replace(grid=(n,) * 3)
    plan = xx.Plan.from_workload(small, precision=xx.XX_FP32_MIXED)
    c = torch.from_numpy(small.c_tgt).cuda()
    wo = torch.from_numpy(small.w_occ).cuda()
    wt = torch.from_numpy(small.w_tgt).cuda()
    ex, vx = plan.energy(c, wo, c, wt, shared=True, stream=stream)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(reps):
        plan.energy(c, wo, c, wt, vx_out=vx, ex_out=ex, shared=True, stream=stream)
    g1.record(stream)
    torch.cuda.synchronize()
    plan.sync(timeout_s=60.0, stream=stream)
    t = g0.elapsed_time(g1) / 1e3 / reps
    e = float(ex[0].item())
    plan.close()
    return {"value": wl.pair_count() / t, "unit": UNIT, "grid": n,
            "E_x_rel_diff_vs_%d" % wl.grid[0]: abs(e - e_ref) / abs(e_ref),
            "sample": "%s with the plan created on the %d^3 grid (4 n_max + 1 = %d), FP32-mixed, "
                      "mean of %d steps" % (wl.name, n, 4 * int(wl.n_max().max()) + 1, reps)}


def alpha_boron_leg(xx, torch, stream, hbm, reps=2):
    """The alpha-boron-sized workload (48^3, MP 4x4x4 = 64 k-points, 18 occupied / 24
    target bands: 1,769,472 pairs) through xx_energy with shared grids."""
    from paper_1111_0716_gb300 import synth
    wl = synth.alpha_boron()
    plan = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED)
    c = torch.from_numpy(wl.c_tgt).cuda()
    wo = torch.from_numpy(wl.w_occ).cuda()
    wt = torch.from_numpy(wl.w_tgt).cuda()
    ex, vx = plan.energy(c, wo, c, wt, shared=True, stream=stream)
    torch.cuda.synchronize()
    p0 = plan.info()["pairs_transformed"]
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(reps):
        plan.energy(c, wo, c, wt, vx_out=vx, ex_out=ex, shared=True, stream=stream)
    g1.record(stream)
    torch.cuda.synchronize()
    plan.sync(timeout_s=60.0, stream=stream)
    info = plan.info()
    t = g0.elapsed_time(g1) / 1e3 / reps
    plan.close()
    TA, TJ = info["targets_per_batch"], info["occupied_per_batch"]
    sched = batch_schedule(wl.nk, wl.n_occ, wl.n_tgt, TA, TJ, info["q_per_batch"])
    if sum(a * b for _, a, b in sched) * reps != info["pairs_transformed"] - p0:
        raise RuntimeError("launch schedule model disagrees with the library (alpha-boron)")
    path_bytes = sum(pass_bytes_per_step(wl, sched).values())
    return {"value": wl.pair_count() / t, "unit": UNIT, "ms_per_step": 1e3 * t,
            "path_roofline": {"achieved": path_bytes / t / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": path_bytes / t / 1e9 / hbm},
            "sample": "%s: 48^3, 64 k-points, 18 occupied x 24 targets = %d pairs, FP32-mixed, "
                      "mean of %d steps" % (wl.name, wl.pair_count(), reps)}


def sweep_leg(xx, torch, stream, reps=3):
    """The six uneven sweep cells (32^3 ... 80^3, 16 ... 96 bands, Gamma; 17,472 pairs):
    one launch per band-pair pass over all cells (xx_run_batched) against one plan per
    cell on concurrent streams (xx_run_many), FP32-mixed."""
    from paper_1111_0716_gb300 import synth
    cells = [synth.sweep_cell(i) for i in range(len(synth.SWEEP_GRIDS))]
    plans, jobs = [], []
    for wl in cells:
        plan = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED, workspace_cap=48 << 30)
        c = torch.from_numpy(wl.c_tgt).cuda()
        jobs.append({"plan": plan, "c_occ": c, "ld_occ": c.shape[1],
                     "w_occ": torch.from_numpy(wl.w_occ).cuda(), "c_tgt": c,
                     "w_tgt": torch.from_numpy(wl.w_tgt).cuda(), "vx_out": torch.empty_like(c),
                     "ex_out": torch.empty(2, dtype=torch.float64, device="cuda")})
        plans.append(plan)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for name, fn in (("batched", xx.xx_run_batched), ("streams", xx.xx_run_many)):
        fn(jobs, stream=stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            g0.record(stream)
            fn(jobs, stream=stream)
            g1.record(stream)
            torch.cuda.synchronize()
            ts.append(g0.elapsed_time(g1) / 1e3)
        out[name] = float(np.median(ts))
    for plan in plans:
        plan.sync(timeout_s=60.0, stream=stream)
        plan.close()
    pairs = sum(wl.pair_count() for wl in cells)
    return {"value": pairs / out["batched"], "unit": UNIT, "streams_same_cells": pairs / out["streams"],
            "ms_batched": 1e3 * out["batched"], "ms_streams": 1e3 * out["streams"],
            "sample": "six Gamma cells 32^3 ... 80^3 with 16 ... 96 bands (%d pairs), FP32-mixed, "
                      "one launch per band-pair pass over all cells vs one plan per cell on its own "
                      "stream, median of %d" % (pairs, reps)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-occ", type=int, default=40,
                    help="occupied bands in the oracle sample (pairs = 8 x this; 40 bands take "
                         "about 10 s on 16 cores)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 slice")
    ap.add_argument("--no-real", action="store_true", help="skip the real-orbital Gamma leg")
    ap.add_argument("--no-exact-grid", action="store_true",
                    help="skip the smallest-exact-grid leg")
    ap.add_argument("--no-alpha", action="store_true", help="skip the alpha-boron-sized leg")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the six-cell sweep leg (one launch per pass vs streams)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one slice of the workload (k=0, 64 targets x 80 occupied bands, "
                         "all q: one launch per pass in the benchmark's batch shape) once and "
                         "exit: the case ncu captures")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of --profile-case")
    ap.add_argument("--profile-small", action="store_true",
                    help="with --profile-case: 16 targets x 16 occupied bands (a few GB on the "
                         "device, for multi-pass ncu captures); with --profile-shared: 16 bands "
                         "at each of the two k-points")
    ap.add_argument("--profile-shared", action="store_true",
                    help="with --profile-case: xx_energy on the first two k-points with shared "
                         "grids (pair-symmetric batches, role-swapped pass C; about 25 GB)")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="with --profile-case: run the case on this FFT grid instead of 96^3 "
                         "(any supported length >= 4 n_max + 1 = 57, e.g. 60)")
    ap.add_argument("--profile-alpha", action="store_true",
                    help="with --profile-case: two steps of the alpha-boron-sized workload (48^3, "
                         "64 k-points) through xx_energy with shared grids, the first of which "
                         "builds the grids and kernel tables")
    ap.add_argument("--with-vjp", action="store_true",
                    help="also time the vector-Jacobian product (xx_apply_vjp, both orbital "
                         "sets) on 16 target bands of every k-point")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.profile_case:
        profile_case(args)
        return

    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import synth, xx

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.beta_boron()
    pairs = wl.pair_count()
    plan = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED)
    if world > 1:
        plan.set_shard(rank, world)
    stream = torch.cuda.current_stream()
    # rank 0 holds the orbitals; the others receive them every step
    c = torch.from_numpy(wl.c_tgt).cuda() if rank == 0 else \
        torch.empty(wl.c_tgt.shape, dtype=torch.complex128, device="cuda")
    w = torch.from_numpy(wl.w_tgt).cuda()
    vx = torch.empty_like(c)
    ex = torch.empty(2, dtype=torch.float64, device="cuda")

    # the occupied orbitals are the leading n_occ target bands (ld = n_tgt)
    w_occ = torch.from_numpy(wl.w_occ).cuda()

    ex_parts = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in range(world)]

    def step():
        if world > 1:
            distribute_orbitals(c)
        xx.xx_energy(plan.handle, c, c.shape[1], w_occ, wl.n_occ, c, w, c.shape[1], vx, ex)
        if world > 1:
            combine_shards(vx, ex, ex_parts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.profile(True)
    plan.profile_read(reset=True)
    launches0 = plan.info()["kernel_launches"]
    pairs0 = plan.info()["pairs_transformed"]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    launches = plan.info()["kernel_launches"] - launches0
    pairs_step_transformed = plan.info()["pairs_transformed"] - pairs0
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    info = plan.info()
    e_x = float(ex[0].item())
    if world > 1:
        tt = torch.tensor([t], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    value = pairs * args.steps / t

    # end to end through the public API with pinned host buffers
    c_h = torch.from_numpy(wl.c_tgt).pin_memory()
    w_h = torch.from_numpy(wl.w_tgt).pin_memory()
    wo_h = torch.from_numpy(wl.w_occ).pin_memory()
    vx_h = torch.empty(vx.shape, dtype=vx.dtype).pin_memory()
    ex_h = torch.empty(2, dtype=torch.float64).pin_memory()

    def e2e_step():
        if rank == 0:
            c.copy_(c_h, non_blocking=True)
        w.copy_(w_h, non_blocking=True)
        w_occ.copy_(wo_h, non_blocking=True)
        step()
        if rank == 0:
            vx_h.copy_(vx, non_blocking=True)
            ex_h.copy_(ex, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 2))
    e2e_step()
    torch.cuda.synchronize()
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    t_e2e = f0.elapsed_time(f1) / 1e3
    if world > 1:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    h2d = c.numel() * 16 + (w.numel() + w_occ.numel()) * 8
    d2h = vx.numel() * 16 + 16

    # roofline of the dominant kernel: algorithmic bytes over its event-timed
    # device time during the timed steps, against the measured HBM copy rate
    hbm, peak_kind = peaks()
    TA, TJ = info["targets_per_batch"], info["occupied_per_batch"]
    owner = xx.xx_shard_blocks(wl.nk, wl.n_occ, wl.n_tgt, world)

    def owned(k, q):
        k, q = min(k, q), max(k, q)
        return owner[k * wl.nk - k * (k - 1) // 2 + (q - k)] == rank
    sched = batch_schedule(wl.nk, wl.n_occ, wl.n_tgt, TA, TJ, info["q_per_batch"], owned=owned)
    transformed = sum(ta * tj for _, ta, tj in sched)
    if transformed * args.steps != pairs_step_transformed:
        raise RuntimeError("launch schedule model (%d pairs) disagrees with the library (%d)"
                           % (transformed * args.steps, pairs_step_transformed))
    model = pass_bytes_per_step(wl, sched)
    dom = max(("pass_a", "pass_b", "pass_c"), key=lambda k: prof[k][0])
    ms_tot, n_l = prof[dom]
    mean_s = ms_tot / 1e3 / max(n_l, 1)
    bytes_per_launch = model[dom] * args.steps / max(n_l, 1)
    achieved = bytes_per_launch / mean_s / 1e9 if mean_s > 0 else 0.0
    path_bytes = sum(model.values()) * args.steps
    # DRAM bytes per launch from the recorded bytes per pair: the pairs the class's
    # launches process (a mirrored batch's role-swapped pass C re-reads its pairs)
    per_pair = recorded_traffic(dom, [TA, TJ])
    class_pairs = sum(ta * tj * (2 if (dom == "pass_c" and kind == "mirrored") else 1)
                      for kind, ta, tj in sched)
    traffic = per_pair * class_pairs * args.steps / max(n_l, 1) if per_pair else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "frac_kind": "model bytes (algorithmic) / time",
                "peak_kind": peak_kind, "traffic": traffic,
                "dram_frac": (traffic / mean_s / 1e9 / hbm) if traffic and mean_s > 0 else None,
                "bytes_per_launch": bytes_per_launch, "mean_launch_ms": mean_s * 1e3,
                "launches": n_l,
                "path": {"achieved": path_bytes / t / 1e9, "frac": path_bytes / t / 1e9 / hbm,
                         "bytes_per_logical_pair_per_point": path_bytes / args.steps / pairs / (96 ** 3)}}
    # ALU view of the same kernel: nominal flops of its transforms and pointwise work
    # over its event-timed launches, against the measured FP32 FMA rate
    P1 = 4 * int(wl.n_max().max()) + 1
    fpp = flops_per_pair(96, P1)
    kflops = 0.0
    for kind, ta, tj in sched:
        kflops += fpp[dom] * ta * tj * (2 if (dom == "pass_c" and kind == "mirrored") else 1)
    fp32_peak = xx.xx_measure_fma_rate(xx.XX_FP32_MIXED) if rank == 0 else None
    if fp32_peak:
        alu = kflops * args.steps / max(n_l, 1) / mean_s / 1e12 if mean_s > 0 else 0.0
        roofline["alu"] = {"achieved": alu, "peak": fp32_peak, "unit": "TFLOP/s", "frac": alu / fp32_peak,
                           "peak_kind": "measured FP32 FMA rate (xx_measure_fma_rate)",
                           "flops_per_pair": fpp[dom]}
    shares = {k: v[0] for k, v in prof.items() if v[1]}
    tot = sum(shares.values()) or 1.0
    kernel_share = {k: round(v / tot, 4) for k, v in shares.items()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + " (beta-boron-sized rhombohedral cell)", "grid": 96,
                       "nk": wl.nk, "n_occ": wl.n_occ, "n_tgt": wl.n_tgt,
                       "pairs_per_step": pairs,
                       "parallelism": ("1 GPU" if world == 1 else
                                       "%d GPUs, k-point blocks {k, q} sharded, orbitals broadcast "
                                       "and V_x c all-reduced every step (NCCL)" % world),
                       "precision": "FP32 FFTs and products, FP64 "
                       "accumulation, kernel table and reductions",
                       "pairs_counted": "logical (k, a, q, j) applications; each occupied pair "
                       "of the blocks (k, q) and (q, k) is transformed once (W_qj,ka = "
                       "conj W_ka,qj): %d transforms per step" % (pairs_step_transformed // args.steps),
                       "batch": [TA, TJ], "l2": "inputs larger than L2 (orbital grids %.1f GB)"
                       % (wl.nk * wl.n_tgt * 96 ** 3 * 8 / 1e9), "E_x": e_x},
            "e2e": {"value": pairs * e2e_steps / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roofline, "kernel_time_share": kernel_share,
            "peak_workspace_gb": info["peak_workspace_bytes"] / 1e9}
    if clk:
        line["clocks"] = clk

    if rank == 0 and world == 1 and not args.no_fp64:
        # all-FP64 GPU path on one target k-point at the production batch shape: target
        # k=0, 64 target bands x all 160 occupied bands x 8 q (81,920 pairs)
        p64 = xx.Plan.from_workload(wl, precision=xx.XX_FP64)
        nt, no = 64, wl.n_occ
        ct = torch.from_numpy(wl.c_tgt[:1, :nt].copy()).cuda()
        co = torch.from_numpy(wl.c_occ[:, :no].copy()).cuda()
        wo = torch.from_numpy(wl.w_occ[:, :no].copy()).cuda()
        v64 = torch.empty_like(ct)
        p64.apply_range(0, 1, co, wo, ct, v64)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        p64.apply_range(0, 1, co, wo, ct, v64)
        g1.record(stream)
        torch.cuda.synchronize()
        t64 = g0.elapsed_time(g1) / 1e3
        info64 = p64.info()
        p_slice = nt * wl.nk * no
        # same slice in mixed precision for the like-for-like ratio
        p32 = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED)
        v32 = torch.empty_like(ct)
        p32.apply_range(0, 1, co, wo, ct, v32)
        torch.cuda.synchronize()
        g0.record(stream)
        p32.apply_range(0, 1, co, wo, ct, v32)
        g1.record(stream)
        torch.cuda.synchronize()
        t32 = g0.elapsed_time(g1) / 1e3
        fp64_peak = xx.xx_measure_fma_rate(xx.XX_FP64)
        fl = sum(fpp.values()) * p_slice
        line["fp64"] = {"value": p_slice / t64, "unit": UNIT,
                        "fp32_mixed_same_slice": p_slice / t32,
                        "batch": [info64["targets_per_batch"], info64["occupied_per_batch"]],
                        "alu": {"achieved": fl / t64 / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                                "frac": fl / t64 / 1e12 / fp64_peak,
                                "peak_kind": "measured FP64 FMA rate (xx_measure_fma_rate)",
                                "flops_per_pair": sum(fpp.values())},
                        "fp32_mixed_alu_frac_same_slice": fl / t32 / 1e12 / fp32_peak if fp32_peak else None,
                        "sample": "target k=0, %d target x %d occupied bands x 8 q = %d pairs, "
                                  "no pair symmetry (separate occupied array)" % (nt, no, p_slice)}
        p64.close()
        p32.close()

    if rank == 0 and world == 1 and not args.no_real:
        line["real_gamma"] = real_gamma_leg(xx, torch, stream)

    if rank == 0 and world == 1 and not args.no_exact_grid:
        line["exact_grid"] = exact_grid_leg(xx, torch, wl, stream, e_x)

    if rank == 0 and world == 1 and not args.no_sweep:
        line["sweep_cells"] = sweep_leg(xx, torch, stream)

    if rank == 0 and world == 1 and not args.no_alpha:
        line["alpha_boron"] = alpha_boron_leg(xx, torch, stream, hbm)

    if rank == 0 and args.with_vjp:
        nt = 16
        ct = torch.from_numpy(wl.c_tgt[:, :nt].copy()).cuda()
        co = torch.from_numpy(wl.c_occ.copy()).cuda()
        wo = torch.from_numpy(wl.w_occ.copy()).cuda()
        ybar = torch.from_numpy(np.ascontiguousarray(wl.c_tgt[:, nt:2 * nt])).cuda()
        pv = xx.Plan.from_workload(wl, precision=xx.XX_FP32_MIXED)
        fwd = pv.apply(co, wo, ct)
        pv.vjp(co, wo, ct, ybar)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        pv.apply(co, wo, ct, vx_out=fwd)
        g1.record(stream)
        torch.cuda.synchronize()
        t_f = g0.elapsed_time(g1) / 1e3
        g0.record(stream)
        pv.vjp(co, wo, ct, ybar)
        g1.record(stream)
        torch.cuda.synchronize()
        t_v = g0.elapsed_time(g1) / 1e3
        pv.close()
        p_slice = wl.nk * nt * wl.nk * wl.n_occ
        line["vjp"] = {"value": p_slice / t_v, "unit": UNIT, "forward_same_slice": p_slice / t_f,
                       "sample": "%d target bands x 8 k x 160 occupied x 8 q = %d pairs; the VJP "
                                 "returns dL/dc_tgt* and dL/dc_occ*" % (nt, p_slice)}

    if rank == 0 and world == 1 and not args.no_baseline:
        r, dt, p_s, cores, vx_o = run_oracle_sample(wl, args.oracle_occ, want_vx=True)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "target (k=0, a=0) x 8 q x %d occupied = %d pairs, %.1f s"
                                % (args.oracle_occ, p_s, dt)}
        # parity on the same sample: the CUDA path in both precisions against the oracle
        no = args.oracle_occ
        co = torch.from_numpy(wl.c_occ[:, :no].copy()).cuda()
        wo = torch.from_numpy(wl.w_occ[:, :no].copy()).cuda()
        ct = torch.from_numpy(wl.c_tgt[:1, :1].copy()).cuda()
        ref = np.asarray(vx_o).reshape(-1)
        c0 = wl.c_tgt[0, 0]
        d_ref = np.vdot(c0, ref).real
        par = {"sample": "target (k=0, a=0) x 8 q x %d occupied (the cpu_baseline sample)" % no}
        for name, prec in (("fp32_mixed", xx.XX_FP32_MIXED), ("fp64", xx.XX_FP64)):
            pp = xx.Plan.from_workload(wl, precision=prec)
            got = pp.apply_range(0, 1, co, wo, ct).cpu().numpy().reshape(-1)
            pp.close()
            par[name] = {"max_dVx_over_max_Vx": float(np.abs(got - ref).max() / np.abs(ref).max()),
                         "c_Vx_c_rel": float(abs(np.vdot(c0, got).real - d_ref) / abs(d_ref))}
        line["parity"] = par
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
