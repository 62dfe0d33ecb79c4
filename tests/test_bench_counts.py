"""The work counts behind the benchmark's roofline figures, against brute
force: M2L flops per box pair, tensor-core MACs issued per tile row, near-field
pairs and far-field box pairs of the octree; and the tolerance rule."""
import itertools

import numpy as np

import bench
import oracle
import synth


def test_m2l_flops_per_box_pair_counts_the_retained_terms():
    # F_n += sum_{|m| <= p - |n|} D_{n+m} M_m: one multiply-add per (n, m) with |n| + |m| <= p
    for p in range(1, 9):
        mis = [t for t in itertools.product(range(p + 1), repeat=3) if sum(t) <= p]
        pairs = sum(1 for n in mis for m in mis if sum(n) + sum(m) <= p)
        assert bench.m2l_flops_per_box_pair(p) == 2 * pairs
    assert bench.m2l_flops_per_box_pair(6) == 1848


def test_tensor_core_macs_issued_per_row():
    """Inputs in degree order in steps of 8; each step is one MMA whose N is the
    number of outputs it can feed (|n| <= p - degree of the step's first input),
    rounded up to 16, with K = 8."""
    for p in range(2, 9):
        deg = [int(d) for d in oracle.multi_indices(p).sum(1)]  # degree order, as the kernel stores them
        nc = len(deg)
        macs = 0
        kt = nc if p > 6 else min(nc, 40)  # p <= 6: the inputs from 40 on are FP32 FMAs
        for k0 in range(0, kt, 8):
            feeds = sum(1 for d in deg if d <= p - deg[k0])
            macs += max(16, -(-feeds // 16) * 16) * 8
        assert bench.tc_issued_macs_per_row(p) == macs
    assert bench.tc_issued_macs_per_row(6) == 8 * (96 + 48 + 32 + 16 + 16)
    assert bench.tc_issued_macs_per_row(8) == 8 * sum(
        max(16, -(-sum(1 for d in [int(v) for v in oracle.multi_indices(8).sum(1)] if d <= 8 - dk) // 16) * 16)
        for dk in [int(v) for v in oracle.multi_indices(8).sum(1)][::8])


def test_cuda_core_part_of_the_m2l_covers_the_rest():
    """Tensor-core inputs x their outputs + the CUDA-core FMAs = every retained
    term |n| + |m| <= p."""
    for p in range(1, 7):
        mis = [t for t in itertools.product(range(p + 1), repeat=3) if sum(t) <= p]
        deg = sorted(sum(t) for t in mis)
        kt = min((len(mis) + 7) // 8 * 8, 40)
        terms = sum(1 for dm in deg[:kt] for dn in deg if dn + dm <= p)
        assert terms + bench.simt_fmas_per_row(p) == bench.m2l_flops_per_box_pair(p) // 2
    assert bench.simt_fmas_per_row(6) == 16 * 4 + 28


def test_shift_flop_counts():
    """M2M: per coefficient n, three one-axis convolutions of n_x, n_y, n_z terms
    and one scaling; L2L per level: three passes of p - |n| terms, one scaling
    and one add."""
    for p in range(1, 9):
        mis = [t for t in itertools.product(range(p + 1), repeat=3) if sum(t) <= p]
        assert bench.m2m_flops_per_box(p) == sum(2 * sum(t) + 1 for t in mis)
        assert bench.l2l_flops_per_level(p) == sum(3 * 2 * (p - sum(t)) + 2 for t in mis)


def test_tree_work_counts_pairs_by_brute_force():
    w = synth.workload(1)
    lo, side = oracle.root_box(w.pos)
    depth = 3
    near, boxes, _, _ = bench.tree_work(w.pos, depth, lo, side)
    cells = oracle.leaf_cells(w.pos, depth, lo, side).astype(np.int64)
    # ordered site pairs i != j in adjacent (or the same) leaves
    adj = np.abs(cells[:, None, :] - cells[None, :, :]).max(axis=2) <= 1
    assert near == int(adj.sum()) - w.n
    # box pairs at each level >= 2: occupied target and source, not adjacent, parents adjacent
    total = 0
    for l in range(2, depth + 1):
        occ = sorted({tuple(c) for c in (cells >> (depth - l)).tolist()})
        for t in occ:
            for s in occ:
                d = max(abs(a - b) for a, b in zip(t, s))
                dp = max(abs((a >> 1) - (b >> 1)) for a, b in zip(t, s))
                total += d > 1 and dp <= 1
    assert boxes == total


def test_tolerance_rule():
    assert bench.tol_for("fp64", 10 ** 6) == 1e-8
    assert bench.tol_for("mixed", 100_000) == 1e-6
    assert bench.tol_for("mixed", 100_001) == 3e-7


def test_tree_work_counts_ffma_entries_by_brute_force():
    """Entries of the FP32 CUDA-core M2L: boxes of levels >= 2 per octant class
    (coarse levels first, Morton order within a level) in groups of 32; a group
    has an entry for each offset of its class at which any member's source
    box is occupied."""
    w = synth.workload(1)
    lo, side = oracle.root_box(w.pos)
    depth = 3
    _, _, _, entries = bench.tree_work(w.pos, depth, lo, side)
    cells = oracle.leaf_cells(w.pos, depth, lo, side).astype(np.int64)

    def morton(t):
        return sum(((t[a] >> b) & 1) << (3 * b + a) for b in range(8) for a in range(3))

    rows = {k: [] for k in range(8)}
    occ = {}
    for l in range(2, depth + 1):
        occ[l] = {tuple(c) for c in (cells >> (depth - l)).tolist()}
        for t in sorted(occ[l], key=morton):
            rows[(t[0] & 1) + 2 * (t[1] & 1) + 4 * (t[2] & 1)].append((l, t))
    total = 0
    for k in range(8):
        b = (k & 1, (k >> 1) & 1, (k >> 2) & 1)
        offs = [o for o in itertools.product(range(-3, 4), repeat=3)
                if max(map(abs, o)) > 1 and all(bd - 3 <= od <= bd + 2 for od, bd in zip(o, b))]
        assert len(offs) == 189
        for g in range(0, len(rows[k]), 32):
            grp = rows[k][g:g + 32]
            total += sum(any(tuple(t[a] - o[a] for a in range(3)) in occ[l] for l, t in grp) for o in offs)
    assert entries == total


def test_polarizable_fraction_workload():
    """--pol-frac keeps alpha on a seeded random subset of about that fraction
    of the sites and zeroes it elsewhere; positions and charges are unchanged."""
    full = bench.make_workload("cube1k")
    w = bench.make_workload("cube1k", 0.3)
    again = bench.make_workload("cube1k", 0.3)
    kept = w.alpha > 0
    assert abs(kept.mean() - 0.3) < 0.05
    assert np.array_equal(w.alpha[kept], full.alpha[kept]) and np.all(w.alpha[~kept] == 0.0)
    assert np.array_equal(w.pos, full.pos) and np.array_equal(w.q, full.q)
    assert np.array_equal(again.alpha, w.alpha)


def test_workload_name_carries_the_options():
    class A:
        pol_frac, dipole_tree = 1.0, False
    assert bench.workload_extra(A) == ""
    A.pol_frac, A.dipole_tree = 0.3, True
    assert bench.workload_extra(A) == " pol_frac=0.3 dipole_tree"
