"""Adaptive kd-tree FMM of Sec. III, on the CPU in FP64.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the plain reference for
the paper's own tree and walk. It composes the single-box operators of the C
oracle (P2M, M2M, M2L, L2L, L2P of Sec. II.B and the direct sums of Sec. II.A),
whose pins are in ``tests/test_oracle_pins.py``; its own pins are in
``tests/test_oracle_kdtree.py``.

Tree (Sec. III). A cell's particles are split across the longest dimension of
the cell's bounding volume, at the geometric centre of the particles along
that dimension. The recursion stops when a cell holds at most ``n_bucket``
particles (8 in the paper). Each cell stores:
- the geometric centre z of its particles;
- the tightest box enclosing them, padded when the cell holds fewer than three
  particles;
- r_enc, the distance from z to the box's farthest corner;
- its multipole coefficients M and field tensor coefficients F.
Multipoles are formed at the leaves and shifted up to the root.

Walk (Sec. III, Eq. mac). A stack of node pairs starts with (root, root). Each
pair taken from the stack is treated as follows.
- Direct sums are used when the two nodes together hold fewer than
  ``n_direct`` particles (about 64 in the paper), or when both are leaves.
- Otherwise, if theta |z_A - z_B| > r_enc,A + r_enc,B, the pair interacts
  through its multipoles, mutually: both nodes receive field tensors.
- Otherwise the node with the larger r_enc is split: its two children are
  paired with the other node. If that node is a leaf, the other node is split
  instead.
- A self pair that is not summed directly pushes the three unique
  combinations of its children.
After the walk the field tensors are shifted down to the leaves and evaluated
at the particles.

Readings where the paper leaves a choice:
- The "bounding volume" whose longest dimension is split is the tight box of
  the cell's particles.
- A self pair counts its particles once against ``n_direct``.
- The "small padding" of cells with fewer than three particles is ``pad`` Å on
  every side.
- When node B is split against A != B, the printed example also pushes
  B_left B_right. That pair is B's own self interaction, which the walk
  already reaches through (B, B); pushing it here as well would count those
  pairs twice. Only (A, B_left) and (A, B_right) are pushed.
"""
from __future__ import annotations

import numpy as np

from . import direct_fields, l2l, l2p, m2l, m2m, ncoef, p2m


class Cell:
    __slots__ = ("idx", "z", "lo", "hi", "r_enc", "children", "M", "F")

    def __init__(self, idx, pos, pad):
        self.idx = idx
        pts = pos[idx]
        self.z = pts.mean(axis=0)
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        if len(idx) < 3:
            lo, hi = lo - pad, hi + pad
        self.lo, self.hi = lo, hi
        corners = np.array([[a, b, c] for a in (lo[0], hi[0]) for b in (lo[1], hi[1]) for c in (lo[2], hi[2])])
        self.r_enc = float(np.max(np.linalg.norm(corners - self.z, axis=1)))
        self.children = ()
        self.M = None
        self.F = None

    @property
    def leaf(self):
        return not self.children

    @property
    def n(self):
        return len(self.idx)


def build_tree(pos, n_bucket=8, pad=1e-3):
    """kd-tree of Sec. III: returns the root Cell; every Cell lists its
    particles' indices, leaves hold at most n_bucket of them."""
    pos = np.asarray(pos, dtype=np.float64)

    def split(idx):
        cell = Cell(idx, pos, pad)
        if len(idx) <= n_bucket:
            return cell
        pts = pos[idx]
        extent = pts.max(axis=0) - pts.min(axis=0)
        d = int(np.argmax(extent))
        if extent[d] <= 0.0:  # coincident particles: nothing to split
            return cell
        c = pts[:, d].mean()
        left = idx[pts[:, d] < c]
        right = idx[pts[:, d] >= c]
        cell.children = (split(left), split(right))
        return cell

    return split(np.arange(pos.shape[0]))


def cells(root):
    """All cells, parents before children."""
    out, stack = [], [root]
    while stack:
        c = stack.pop()
        out.append(c)
        stack.extend(c.children)
    return out


def walk(root, theta, n_direct=64):
    """The dual-tree walk of Sec. III. Returns the direct pairs and the
    multipole pairs as lists of (A, B) cells; a self pair has A is B."""
    direct, multipole = [], []
    stack = [(root, root)]
    while stack:
        a, b = stack.pop()
        if a is b:
            if a.leaf or a.n < n_direct:
                direct.append((a, a))
            else:
                l, r = a.children
                stack.extend([(l, l), (r, r), (l, r)])
            continue
        if a.n + b.n < n_direct or (a.leaf and b.leaf):
            direct.append((a, b))
            continue
        if theta * np.linalg.norm(a.z - b.z) > a.r_enc + b.r_enc:
            multipole.append((a, b))
            continue
        big, small = (a, b) if a.r_enc >= b.r_enc else (b, a)
        if big.leaf:
            big, small = small, big
        c1, c2 = big.children
        stack.extend([(small, c1), (small, c2)])
    return direct, multipole


def _zero(v, shape):
    return np.zeros(shape) if v is None else v


def _leaf_multipole(p, z, x, q, mu, dl):
    """P2M of a leaf. With dl > 0 each point dipole enters as the pair of
    Sec. II.C: charges +q_mu at x + dl mu/|mu| and -q_mu at x - dl mu/|mu|,
    q_mu = |mu| / (2 dl), so that mu = 2 q_mu dl; dl = 0 takes the analytic
    point-dipole multipole (the dl -> 0 limit)."""
    if dl <= 0.0:
        return p2m(p, z, x, q, mu)
    norm = np.linalg.norm(mu, axis=1)
    has = norm > 0.0
    u = mu[has] / norm[has, None]
    qm = norm[has] / (2.0 * dl)
    pts = np.concatenate([x, x[has] + dl * u, x[has] - dl * u])
    chg = np.concatenate([q, qm, -qm])
    return p2m(p, z, pts, chg, None)


def kdtree_fields(pos, q=None, mu=None, p=5, theta=0.5, n_bucket=8, n_direct=64, pad=1e-3, dipole_dl=0.0):
    """Phi, E and G = grad E at every site by the kd-tree FMM of Sec. III.
    dipole_dl > 0 builds the multipoles of the dipoles from the +-q pairs of
    Sec. II.C at that separation; the direct sums always use the dipoles
    themselves, as the paper does."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    qv = _zero(None if q is None else np.asarray(q, dtype=np.float64), n)
    mv = _zero(None if mu is None else np.asarray(mu, dtype=np.float64), (n, 3))
    root = build_tree(pos, n_bucket, pad)
    allc = cells(root)
    nc = ncoef(p)
    # upward pass: P2M at the leaves about their centres, M2M to the parents
    for c in reversed(allc):
        if c.leaf:
            c.M = _leaf_multipole(p, c.z, pos[c.idx], qv[c.idx], mv[c.idx], dipole_dl)
        else:
            c.M = sum(m2m(p, c.z - ch.z, ch.M) for ch in c.children)
        c.F = np.zeros(nc)
    direct, multipole = walk(root, theta, n_direct)
    phi, E, G = np.zeros(n), np.zeros((n, 3)), np.zeros((n, 6))
    # multipole interactions, accumulated for both nodes (momentum)
    for a, b in multipole:
        a.F += m2l(p, a.z - b.z, b.M)
        b.F += m2l(p, b.z - a.z, a.M)
    # direct interactions with the explicit charges and dipoles
    for a, b in direct:
        if a is b:
            r = direct_fields(pos[a.idx], qv[a.idx], mv[a.idx])
            phi[a.idx] += r["phi"]
            E[a.idx] += r["E"]
            G[a.idx] += r["G"]
            continue
        for t, s in ((a, b), (b, a)):
            # sources s, then the targets t as silent sites
            P = np.concatenate([pos[s.idx], pos[t.idx]])
            Q = np.concatenate([qv[s.idx], np.zeros(t.n)])
            MU = np.concatenate([mv[s.idx], np.zeros((t.n, 3))])
            r = direct_fields(P, Q, MU, targets=np.arange(s.n, s.n + t.n))
            phi[t.idx] += r["phi"]
            E[t.idx] += r["E"]
            G[t.idx] += r["G"]
    # downward pass: L2L to the children, L2P at the leaf particles
    for c in allc:
        for ch in c.children:
            ch.F += l2l(p, ch.z - c.z, c.F)
        if c.leaf:
            for i in c.idx:
                ph, dph, ddph = l2p(p, pos[i] - c.z, c.F)
                phi[i] += ph
                E[i] -= dph
                G[i] -= ddph
    return {"phi": phi, "E": E, "G": G}
