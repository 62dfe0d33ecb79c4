"""Throughput of the polarizable FMM energy + forces step on one GB300 (atoms/s).

Workload: the 30,000-site protein-density globule (Gaussian profile, sigma
15 A, 0.1 sites/A^3), charges N(0, 0.35) e neutralised, polarizabilities
U(0.3, 2.5) A^3, expansion order p = 6, octree depth 4.

One step = the whole hot path on a persistent context: rebuild the octree
from HBM-resident positions and run the static pass (fmm_update_positions),
solve the induced dipoles from mu = alpha E^q to the relative residual
tolerance (fmm_solve_induced_dipoles), then one more FMM pass for energy,
forces and parameter gradients (fmm_energy_forces).  The headline `value` is
MIXED precision; the all-FP64 GPU form is timed beside it and the relative RMS
force error of MIXED against FP64 is reported.

The inputs (1.2 MB) are far smaller than L2, so L2 is flushed (a 256 MB write)
before every timed step, outside the step's CUDA-event interval.

--impl reference times the CPU oracle (test infrastructure) on the host cores
on the same workload instead.
"""
from __future__ import annotations

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

METRIC = "atoms/s polarizable FMM energy+forces, mixed vs FP64, at ≤1e-5 RMS force err"
WORKLOAD_INDEX = 2
TOL = {"mixed": 1e-6, "fp64": 1e-8}


def tol_for(mode, n):
    """PCG tolerance (relative residual).  FP64: 1e-8.  MIXED: 1e-6 up to 1e5
    sites, 3e-7 above: the force error against FP64 grows with the system
    (1.2e-5 at 1e-6 on the 4M shell, 1.5e-6 at 1e-7), and every MIXED line must
    stay within the 1e-5 relative RMS force gate."""
    if mode == "fp64":
        return TOL["fp64"]
    return TOL["mixed"] if n <= 100_000 else 3e-7
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernels, from one ncu capture of the workload named in the key (the
# command and the figures are in profiles/); the line reports null for any
# other kernel, workload or mode
TRAFFIC = {                                              # profiles/launches_globule30k_mixed.md
    ("leaf_dipole", "globule", 30000, "mixed"): 1579000,
    ("m2l", "globule", 30000, "mixed"): 2108000,
    ("p2m", "globule", 30000, "mixed"): 1150000,
    ("l2p", "globule", 30000, "mixed"): 5003000,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--m2l", default="auto", choices=["auto", "simt", "tensor", "ffma"])
    ap.add_argument("--pol-frac", type=float, default=1.0,
                    help="fraction of the sites that keep their polarizability (a seeded random subset; the "
                         "others get alpha = 0)")
    ap.add_argument("--dipole-tree", action="store_true",
                    help="solve for the dipoles on a second tree over the polarizable sites (Sec. III)")
    ap.add_argument("--workload", default="globule30k",
                    choices=["globule30k", "cube1k", "ring300k", "globule100k", "shell250k", "shell1M", "shell4M"],
                    help="workload (the default is the one the headline metric is quoted on)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel from the host (no CUDA graphs; for kernel profilers)")
    ap.add_argument("--only-main", action="store_true",
                    help="time the headline mode only (no FP64 leg, profiling, e2e or CPU leg): for ncu captures")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# algorithmic work of one pass (counted from the tree, not from the kernels)
# ---------------------------------------------------------------------------

def ncoef(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def m2l_flops_per_box_pair(p):
    # 2 flops per retained term of F_n += sum_{|m| <= p-|n|} D_{n+m} M_m
    return 2 * sum((s + 1) * (s + 2) // 2 * ncoef(p - s) for s in range(p + 1))


def tc_inputs(p):
    """Inputs that go through the tensor cores: all of them (rounded up to 8) for
    p = 7, 8; at most the first 40 for p <= 6, whose higher-degree inputs feed so
    few outputs that the M2L evaluates them with FP32 FMAs instead."""
    kp = (ncoef(p) + 7) // 8 * 8
    return kp if p > 6 else min(kp, 40)


def tc_issued_macs_per_row(p):
    """MACs per tile row, offset and product issued by the tensor-core M2L: one
    MMA per input step of 8, whose N is the prefix of outputs that step feeds
    (|n| <= p - degree of the step's first input), rounded up to 16."""
    deg = lambda i: next(s for s in range(p + 1) if i < ncoef(s))
    total = 0
    for k in range(tc_inputs(p) // 8):
        dmax = p - deg(8 * k)
        nout = ncoef(dmax) if dmax >= 0 else 0
        total += max(16, (nout + 15) // 16 * 16) * 8
    return total


def simt_fmas_per_row(p):
    """FP32 FMAs per tile row and offset of the M2L's CUDA-core part: inputs from
    tc_inputs(p) on, for every output they can feed (|n| + |m| <= p)."""
    deg = lambda i: next(s for s in range(p + 1) if i < ncoef(s))
    nc = ncoef(p)
    return sum(1 for m in range(tc_inputs(p), nc) for nn in range(nc) if deg(nn) + deg(m) <= p)


def load_peaks():
    try:
        j = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), float(j.get("bf16_tflops_sustained", j["bf16_tflops"])), \
            "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def m2m_flops_per_box(p):
    """Upward shift of one box (three one-axis convolutions, k <= n_d terms per
    coefficient and axis, FMA = 2) plus the 2^-|n| scaling."""
    total = 0
    for s_ in range(p + 1):
        for x in range(s_, -1, -1):
            for y in range(s_ - x, -1, -1):
                z = s_ - x - y
                total += 2 * (x + y + z) + 1
    return total


def l2l_flops_per_level(p):
    """Downward shift of one box per level: three one-axis passes, p - |n| terms
    each (FMA = 2), plus the 2^-(|n|+1) scaling and the partial-sum add."""
    total = 0
    for s_ in range(p + 1):
        total += (s_ + 1) * (s_ + 2) // 2 * (3 * 2 * (p - s_) + 2)
    return total


def radix_passes(depth):
    return (3 * depth + 7) // 8


def m2l_kernel(p, mixed, impl):
    """The M2L kernel the library runs: FP32 FMAs on the CUDA cores (MIXED, p <= 6,
    auto or ffma), tcgen05 TF32 (MIXED otherwise, unless simt), or the SIMT kernel."""
    if not mixed:
        return "simt"
    if impl in ("auto", "ffma") and p <= 6:
        return "ffma"
    return "simt" if impl == "simt" else "tensor"


def family_work(w, n, near_pairs, box_pairs, nbox, mixed, iterations, m2l_impl="auto"):
    """Algorithmic work of one launch of each kernel family (flops or bytes),
    with the bound it is measured against.  Counted from the tree and the
    operators, not from the kernels."""
    p, d = w.p, w.depth
    nc = ncoef(p)
    rsz = 4 if mixed else 8
    leaves = nbox[d]
    inner = sum(nbox[l] for l in range(3, d + 1))  # boxes shifted to their parent
    alu = "fp32" if mixed else "fp64"
    out = {
        # per solver pass: dipole field of the sources, 34 flops per ordered pair
        "leaf_dipole": (near_pairs * 34, "alu", alu, "34 flops per ordered near pair (dipole -> field)"),
        "m2l": (box_pairs * m2l_flops_per_box_pair(p),
                "tensor" if m2l_kernel(p, mixed, m2l_impl) == "tensor" else "alu",
                {"tensor": "tf32", "ffma": "fp32", "simt": alu}[m2l_kernel(p, mixed, m2l_impl)],
                f"{m2l_flops_per_box_pair(p)} flops per box pair (sum over |n|+|m| <= p of 2)"),
        # P2M of the dipoles (8 flops per site and coefficient) and M2M of every box below level 2
        "p2m": (n * nc * 8 + inner * m2m_flops_per_box(p), "alu", alu,
                "P2M 8 flops per site and coefficient + M2M per shifted box"),
        # L2L of the leaf's ancestors from level 3 and L2P of the field (|n| <= p-1: 3 FMA + 2 mul)
        "l2p": (n * ncoef(p - 1) * 10 + leaves * (d - 2) * l2l_flops_per_level(p), "alu", alu,
                "L2P of E (10 flops per site and coefficient of order <= p-1) + L2L per leaf and level"),
        # static pass: charge -> potential and field (20 flops per pair) + L2P of Phi, E
        "leaf_static": (near_pairs * 20 + n * nc * 11 + leaves * (d - 2) * l2l_flops_per_level(p), "alu", alu,
                        "20 flops per pair (charge -> Phi, E) + L2P + L2L"),
        # force pass: charges and dipoles -> Phi, E, grad E (95 flops per pair) + L2P of 10 outputs
        "leaf_full": (near_pairs * 95 + n * nc * 23 + leaves * (d - 2) * l2l_flops_per_level(p), "alu", alu,
                      "95 flops per pair (charge + dipole -> Phi, E, grad E) + L2P + L2L"),
        # tree: bounding box (24 B), keys (24 in, 8 out), radix passes (24 B each), the
        # gather of positions, charges, polarizabilities and the packed copies (~120 B)
        "tree": (n * (24 + 32 + 24 * radix_passes(d) + 120), "hbm", "hbm",
                 f"{24 + 32 + 24 * radix_passes(d) + 120} B per site per tree build"),
        # PCG vectors: update (reads alpha, d, Ad, mu, r; writes mu, r, z) and direction
        # (reads z, d; writes d and its packed copy), float64
        "solver": (n * (176 + 72 + 4 * rsz), "hbm", "hbm", f"{176 + 72 + 4 * rsz} B per site per PCG iteration"),
        # energies and gradients: reads q, alpha, mu, Phi^q, E^q, Phi, E, grad E, perm; writes F, dU/dq, dU/dalpha
        "assemble": (n * 196, "hbm", "hbm", "196 B per site (assembly reads and writes)"),
    }
    return out


def _morton3(x, y, z):
    key = np.zeros(x.shape, dtype=np.int64)
    for b in range(10):
        key |= (((x >> b) & 1) << (3 * b)) | (((y >> b) & 1) << (3 * b + 1)) | (((z >> b) & 1) << (3 * b + 2))
    return key


def tree_work(pos, depth, lo, side):
    """Near-field pairs (ordered, i != j, adjacent leaves), far-field box pairs
    (the 189-offset interaction lists, occupied sources only), tensor-core tiles,
    and the entries of the FP32 CUDA-core M2L: per group of 32 boxes of one
    octant class (levels >= 2 coarse first, Morton order within a level), the
    offsets with at least one occupied source."""
    ns = 1 << depth
    h = side / ns
    cell = np.clip(np.floor((pos - lo) / h).astype(np.int64), 0, ns - 1)
    lin = cell[:, 0] + ns * (cell[:, 1] + ns * cell[:, 2])
    cnt = np.bincount(lin, minlength=ns ** 3).reshape(ns, ns, ns).transpose(2, 1, 0)  # [x][y][z]
    pad = np.pad(cnt, 1)
    nb = np.zeros_like(cnt)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                nb += pad[1 + dx:1 + dx + ns, 1 + dy:1 + dy + ns, 1 + dz:1 + dz + ns]
    near_pairs = int(np.sum(cnt * nb) - pos.shape[0])
    box_pairs = 0
    class_rows = np.zeros(8, dtype=np.int64)
    offsets = [(ox, oy, oz) for oz in range(-3, 4) for oy in range(-3, 4) for ox in range(-3, 4)
               if max(abs(ox), abs(oy), abs(oz)) > 1]
    present = [[] for _ in range(8)]  # per class: [rows, 343-grid offsets] occupancy of the source
    for l in range(2, depth + 1):
        m = 1 << l
        occ = np.zeros((m, m, m), dtype=bool)
        c = cell >> (depth - l)
        occ[c[:, 0], c[:, 1], c[:, 2]] = True
        tx, ty, tz = np.nonzero(occ)
        order = np.argsort(_morton3(tx, ty, tz), kind="stable")
        tx, ty, tz = tx[order], ty[order], tz[order]
        cls = (tx & 1) + 2 * (ty & 1) + 4 * (tz & 1)
        class_rows += np.bincount(cls, minlength=8)
        pres = np.zeros((tx.shape[0], len(offsets)), dtype=bool)
        for j, (ox, oy, oz) in enumerate(offsets):
            ok = np.ones(tx.shape, dtype=bool)
            for t, o in ((tx, ox), (ty, oy), (tz, oz)):
                b = t & 1
                ok &= (o >= b - 3) & (o <= b + 2)
            sx, sy, sz = tx - ox, ty - oy, tz - oz
            ok &= (sx >= 0) & (sy >= 0) & (sz >= 0) & (sx < m) & (sy < m) & (sz < m)
            ok[ok] &= occ[sx[ok], sy[ok], sz[ok]]
            box_pairs += int(ok.sum())
            pres[:, j] = ok
        for k in range(8):
            present[k].append(pres[cls == k])
    tc_tiles = int(sum((r + 127) // 128 for r in class_rows))
    ffma_entries = 0
    for k in range(8):
        pk = np.concatenate(present[k]) if present[k] else np.zeros((0, len(offsets)), dtype=bool)
        for g in range(0, pk.shape[0], 32):
            ffma_entries += int(pk[g:g + 32].any(axis=0).sum())
    return near_pairs, box_pairs, tc_tiles, ffma_entries


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.out = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        return run_reference(args)
    if world > 1:
        import torch
        import torch.distributed as tdist

        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()


WORKLOADS = {"globule30k": (2, None), "cube1k": (1, None), "ring300k": (3, None), "globule100k": (4, None),
             "shell250k": (5, 250000), "shell1M": (5, 1000000), "shell4M": (5, 4000000)}


def max_over_ranks(total_ms, dist, device):
    """The job's time is the slowest rank's: MAX all-reduce of the timed
    interval (a no-op on one rank)."""
    if not dist:
        return total_ms
    import torch
    import torch.distributed as tdist

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, n, steps, total_ms):
    """Whole-job atoms/s: every rank runs an independent replica of n sites."""
    return world * n * steps / (total_ms / 1e3)


def workload_extra(args):
    """The workload name's suffix for the polarizable fraction and the dipole tree."""
    extra = f" pol_frac={args.pol_frac:g}" if args.pol_frac < 1.0 else ""
    return extra + (" dipole_tree" if args.dipole_tree else "")


def make_workload(name, pol_frac=1.0):
    """The named workload; with pol_frac < 1 only that fraction of the sites (a
    seeded random subset) keeps its polarizability, the others get alpha = 0."""
    import synth

    idx, n = WORKLOADS[name]
    w = synth.workload(idx, n=n)
    if pol_frac < 1.0:
        rng = np.random.Generator(np.random.PCG64(4242))
        off = rng.random(w.n) >= pol_frac
        w.alpha[off] = 0.0
    return w


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_1408_6527_gb300 import PolFMM
    import synth

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
    w = make_workload(args.workload, args.pol_frac)
    n = w.n
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    pos_d, q_d, a_d = dev(w.pos), dev(w.q), dev(w.alpha)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make(mode, src=None, profile=False, max_iter=500):
        s = src if src is not None else (pos_d, q_d, a_d)
        return PolFMM(*s, p=w.p, depth=w.depth, mode=mode, max_iter=max_iter, m2l=args.m2l, profile=profile,
                      graphs=not args.no_graphs, dipole_tree=args.dipole_tree)

    def step(ctx, mode, pos, tol=None):
        ctx.update_positions(pos)
        ctx.reset_dipoles()
        info = ctx.solve(tol_for(mode, n) if tol is None else tol)
        out = ctx.energy_forces()
        return info, out

    def timed(ctx, mode, steps, warmup, sample_clocks=False, tol=None):
        for _ in range(warmup):
            step(ctx, mode, pos_d, tol)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local_rank) if sample_clocks else None
        total_ms, iters = 0.0, []
        l0 = ctx.launch_count()
        info = out = None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info, out = step(ctx, mode, pos_d, tol)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            iters.append(info["iterations"])
        launches = ctx.launch_count() - l0
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        clocks = sampler.stop() if sampler else None
        return total_ms, iters, launches, info, out, clocks

    ctx = make(args.mode)
    total_ms, iters, launches, info, out, clocks = timed(ctx, args.mode, args.steps, args.warmup, True)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    F_main = out["F"].detach().cpu().numpy()
    mu_main = ctx.dipoles().detach().cpu().numpy()
    U_main = out["U"]
    lo, side = ctx.root_box()
    ctx.close()
    if rank != 0:
        return None
    ms_per_step = total_ms / args.steps
    value = job_value(world, n, args.steps, total_ms)
    if args.only_main:
        return {"metric": METRIC, "value": round(value, 1), "unit": "atoms/s", "ms_per_step": round(ms_per_step, 4),
                "iterations": iters[-1], "gpu_launches": int(launches), "only_main": True}

    # the other precision on the same workload
    other = "fp64" if args.mode == "mixed" else "mixed"
    ctx2 = make(other)
    t2, it2, _, info2, out2, _ = timed(ctx2, other, max(2, args.steps // 2), 1)
    F_other = out2["F"].detach().cpu().numpy()
    mu_other = ctx2.dipoles().detach().cpu().numpy()
    U_other = out2["U"]
    ctx2.close()
    res = {args.mode: (U_main, F_main, mu_main), other: (U_other, F_other, mu_other)}
    F64, Fmx = res["fp64"][1], res["mixed"][1]
    rms_err = rel_rms(Fmx, F64)
    errors_vs_fp64 = {"energy_rel": abs(res["mixed"][0] - res["fp64"][0]) / abs(res["fp64"][0]),
                      "forces_rel_rms": rms_err, "dipoles_rel_rms": rel_rms(res["mixed"][2], res["fp64"][2])}
    n2 = max(2, args.steps // 2)

    # the paper's timing protocol: exactly 10 dipole iterations per step
    ctx10 = make(args.mode, max_iter=10)
    t10, it10, _, _, _, _ = timed(ctx10, args.mode, max(2, args.steps // 2), 1, tol=0.0)
    ctx10.close()
    n10 = max(2, args.steps // 2)

    # per-kernel CUDA-event durations, recorded on the launching stream over
    # separately profiled steps of the same workload (kernels one at a time, no
    # graph and no near/far overlap: the shares are proportions, the sum exceeds
    # the graph-launched step)
    from paper_1408_6527_gb300 import measure_peak
    ctxp = make(args.mode, profile=True)
    for _ in range(2):
        step(ctxp, args.mode, pos_d)
    ctxp.profile_reset()
    nprof = 3
    prof_iters = 0
    for _ in range(nprof):
        flush.zero_()
        info_p, _ = step(ctxp, args.mode, pos_d)
        prof_iters += info_p["iterations"]
    fams = ["tree", "p2m", "m2m", "m2l", "l2l", "leaf_dipole", "l2p", "leaf_static", "leaf_full", "solver",
            "assemble"]
    prof = {f: ctxp.profile(f) for f in fams}
    nbox = ctxp.tree_info()["boxes"]
    ctxp.close()
    prof_total = sum(v[0] for v in prof.values())

    # roofline of every kernel family against its own measured peak
    near_pairs, box_pairs, tc_tiles, ffma_entries = tree_work(w.pos, w.depth, lo, side)
    hbm_peak, bf16_burst, bf16_sust, peak_src = load_peaks()
    p = w.p
    mixed = args.mode == "mixed"
    stream_ptr = torch.cuda.current_stream().cuda_stream
    fp32_peak = measure_peak("fp32", stream_ptr)
    fp64_peak = measure_peak("fp64", stream_ptr)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peaks = {
        "fp32": (fp32_peak, "TFLOP/s", f"measured FP32 FMA chains on all {props.multi_processor_count} SMs"),
        "fp64": (fp64_peak, "TFLOP/s", f"measured FP64 FMA chains on all {props.multi_processor_count} SMs"),
        # a kernel timed on its own: the burst cuBLAS figure, scaled to TF32 by the nominal ratio
        "tf32": (bf16_burst * 1.1 / 2.25, "TFLOP/s",
                 f"TF32 dense = {peak_src} burst bf16 {bf16_burst} x nominal TF32/BF16 1.1/2.25"),
        "hbm": (hbm_peak, "GB/s", f"{peak_src} HBM copy"),
    }
    work = family_work(w, n, near_pairs, box_pairs, nbox, mixed, prof_iters / nprof, args.m2l)
    roofs = {}
    for fam, (units, bound, pk, note) in work.items():
        ms, nl = prof[fam]
        if nl == 0:
            continue
        dur_s = ms / nl / 1e3
        if fam == "solver":  # one family launch per kernel: count the work per PCG iteration
            dur_s = ms / max(prof_iters, 1) / 1e3
        peak, unit, peak_note = peaks[pk]
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        achieved = units / dur_s / scale
        r = {"kernel": fam, "bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": unit,
             "frac": round(achieved / peak, 5),
             "traffic": TRAFFIC.get((fam, w.name, n, args.mode)),
             "peak_note": peak_note, "work_note": note,
             "avg_launch_ms": round(ms / nl, 4), "launches_per_step": round(nl / nprof, 2),
             ("algorithmic_bytes_per_unit" if bound == "hbm" else "algorithmic_flops_per_launch"): int(units),
             "share_of_step": round(ms / prof_total, 4)}
        if fam == "m2l" and m2l_kernel(p, mixed, args.m2l) == "tensor":
            # what the kernel issues: three TF32 products over the block-sparse MMA
            # schedule on every tile row, present or not
            issued = 3 * 2 * 128 * tc_issued_macs_per_row(p) * tc_tiles * 189
            r["issued_tensor_tflops"] = round(issued / dur_s / 1e12, 3)
            r["issued_tensor_frac"] = round(issued / dur_s / 1e12 / peaks["tf32"][0], 5)
        if fam == "m2l" and m2l_kernel(p, mixed, args.m2l) == "ffma":
            # what the kernel issues: every lane of a group runs the whole
            # contraction for each offset where any of the group's sources exists
            issued = 32 * m2l_flops_per_box_pair(p) * ffma_entries
            r["issued_fp32_tflops"] = round(issued / dur_s / 1e12, 3)
            r["issued_fp32_frac"] = round(issued / dur_s / 1e12 / peaks["fp32"][0], 5)
            r["lane_fill"] = round(box_pairs / (32 * ffma_entries), 4) if ffma_entries else None
        roofs[fam] = r
    dom = max(roofs, key=lambda f: prof[f][0]) if roofs else None
    roof = roofs.get(dom)

    # e2e: the same step through the public API with pinned host buffers
    pos_h = torch.from_numpy(w.pos.copy()).pin_memory()
    ctxh = PolFMM(w.pos, w.q, w.alpha, p=w.p, depth=w.depth, mode=args.mode, max_iter=500, m2l=args.m2l,
                  dipole_tree=args.dipole_tree)
    for _ in range(args.warmup):
        step(ctxh, args.mode, pos_h)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        step(ctxh, args.mode, pos_h)
        e2e_s += time.perf_counter() - s0
    ctxh.close()
    e2e = {"value": round(world * n * args.steps / e2e_s, 1), "unit": "atoms/s",
           "h2d_bytes_per_step": 3 * n * 8, "d2h_bytes_per_step": 5 * n * 8 + 24}

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "atoms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.mode == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"{w.name} {n} sites p={w.p} depth={w.depth} {args.mode}" + workload_extra(args),
                   "n_sites": n, "p": w.p,
                   "depth": w.depth, "mode": args.mode, "tol": tol_for(args.mode, n), "m2l": args.m2l,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before every step (256 MB write, outside the step interval)"},
        "iterations": iters[-1], "converged": bool(info["converged"]),
        "fmm_passes_per_step": iters[-1] + 3,
        "atoms_per_s_per_pass": round(value * (iters[-1] + 3), 1),
        "fixed_10_iterations": {"value": round(world * n * n10 / (t10 / 1e3), 1), "ms_per_step": round(t10 / n10, 4),
                                "iterations": it10[-1]},
        "rms_force_err_mixed_vs_fp64": rms_err,
        "errors_mixed_vs_fp64": {k: float(f"{v:.3e}") for k, v in errors_vs_fp64.items()},
        other: {"value": round(n * n2 / (t2 / 1e3), 1), "ms_per_step": round(t2 / n2, 4), "iterations": it2[-1]},
        "gpu_launches": int(launches),
        "kernel_ms_per_step": {f: round(v[0] / nprof, 4) for f, v in prof.items()},
        "kernel_ms_note": "CUDA events around each launch in separately profiled steps (kernels serialised, no "
                          "graph, no near/far overlap): proportions, whose sum exceeds the graph-launched step",
        "kernel_share": {f: round(v[0] / prof_total, 4) for f, v in prof.items()} if prof_total > 0 else None,
        "roofline": roof, "roofline_kernels": roofs, "clocks": clocks, "e2e": e2e,
        "tree": {"near_pairs": near_pairs, "m2l_box_pairs": box_pairs, "tc_tiles": tc_tiles,
                 "ffma_entries": ffma_entries, "boxes": nbox},
        "peaks": {k: {"value": round(v[0], 2), "unit": v[1], "source": v[2]} for k, v in peaks.items()},
    }
    if world == 1 and not args.no_cpu:
        cb, ref = cpu_baseline(w, lo, side, return_result=True)
        result["cpu_baseline"] = cb
        # both GPU modes against the FP64 oracle on the same tree (same p, root box, depth)
        result["errors_vs_oracle"] = {
            mode: {"energy_rel": float(f"{abs(U - ref['U']) / abs(ref['U']):.3e}"),
                   "forces_rel_rms": float(f"{rel_rms(F, ref['F']):.3e}"),
                   "dipoles_rel_rms": float(f"{rel_rms(mu, ref['mu']):.3e}")}
            for mode, (U, F, mu) in res.items()}
        result["errors_vs_oracle"]["oracle"] = f"CPU FMM, FP64, PCG to {TOL['fp64']:g}, same tree"
    return result


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def cpu_baseline(w, lo, side, tol=None, return_result=False):
    """The CPU oracle as it stands on the host cores: one complete step on the
    full workload (FMM static pass, PCG with FMM matrix-vector products to the
    FP64 tolerance, force pass)."""
    import oracle

    tol = tol if tol is not None else TOL["fp64"]
    t0 = time.perf_counter()
    out = oracle.polarizable_energy(w.pos, w.q, w.alpha, method="fmm", p=w.p, depth=w.depth, root=(lo, side),
                                    tol=tol, max_iter=500)
    dt = time.perf_counter() - t0
    cb = {"value": round(w.n / dt, 1), "unit": "atoms/s", "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"one complete step of the full {w.n}-site workload (FP64 CPU FMM p={w.p} depth={w.depth}, "
                    f"{out['iterations']} PCG iterations to {tol:g}, force pass): {dt:.2f} s"}
    return (cb, out) if return_result else cb


def run_reference(args):
    import synth
    import oracle

    w = make_workload(args.workload, args.pol_frac)
    lo, side = oracle.root_box(w.pos)
    tol = tol_for(args.mode, w.n)
    for _ in range(args.warmup):
        cpu_baseline(w, lo, side, tol)
    total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.polarizable_energy(w.pos, w.q, w.alpha, method="fmm", p=w.p, depth=w.depth, root=(lo, side),
                                  tol=tol, max_iter=500)
        total += time.perf_counter() - t0
    value = w.n * args.steps / total
    cores = oracle.num_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "atoms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{w.name} {w.n} sites p={w.p} depth={w.depth} {args.mode}" + workload_extra(args), "n_sites": w.n,
                   "p": w.p, "depth": w.depth, "mode": args.mode, "tol": tol},
        "cpu_baseline": {"value": round(value, 2), "unit": "atoms/s", "cores": cores, "kind": "oracle",
                         "sample": "each step one complete oracle step of the full workload"},
        "e2e": {"value": round(value, 2), "unit": "atoms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
