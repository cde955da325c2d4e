"""O_fdm: a plain FP64 CPU implementation of the fast directional method.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with, imported by, or imports the CUDA path.

G. Of, R. Watschinger, "Complexity Analysis of a Fast Directional
Matrix-Vector Multiplication".  The code follows the paper's order:

  Sect. 2.1, Alg. 1        uniform box cluster trees        ClusterTree
  Sect. 2.2, Def. 1        admissibility (A1), (A3)         admissibility()
  Sect. 2.3, Alg. 2, Def.2 block tree, L+ and L-            BlockTree
  Sect. 2.4, Eq. (11)      largest high-frequency level     default_l_hf()
  Sect. 2.4, Alg. 3        direction sets D^(l)              Directions
  Sect. 2.4, Def. 3        direction map dir_(l)            Directions.dir()
  Sect. 2.6, Def. 5        active / inherited directions    FDMOracle._direction_sets()
  Sect. 2.2, Eqs. (4)-(10) interpolation, L_{t,c}, A_{c,txs}
  Sect. 2.5, Eq. (13)      transfer matrices E_{t',c}
  Sect. 2.6, Alg. 4        the product g = A v              FDMOracle.apply()
  Sect. 2.7                8 reference E_{t'}, one A per    mode="reuse"
                           reference configuration
  Sect. 2.7 (closing)      A ~ U V^* by partially pivoted   mode="aca"
                           ACA (oracle/aca.py)

Readings where the paper is silent or garbled:
  R1  Eq. (4) prints cos((2 nu - 1)/(2 pi (m+1))); the misplaced pi is read as
      cos((2 nu - 1) pi / (2 (m+1))), the Chebyshev points of the first kind.
  R2  "order" o = m + 1 nodes per axis; multi-index k = nu_x + o nu_y + o^2 nu_z.
  R3  Both trees share one root cube; its lower faces count as closed, so a
      point on them lies in the lowest box (all other boxes are (a, b]).
  R4  Children are numbered bx + 2 by + 4 bz (bit = 1: upper half), so Alg. 1's
      depth-first order lists every level in Morton order.
  R5  Alg. 1 refines a box iff it holds more than n_max points AND its level is
      below max_depth (n_max = 0: refine every non-empty box down to max_depth).
  R6  diam and dist of Def. 1 are those of the closed boxes.
  R7  The ray-face tie rule of Def. 3 is evaluated on m_t - m_s itself
      (psi_Q is scale invariant; m_t - m_s is exact in FP64 for dyadic boxes).
  R8  Faces 1..6 are -x, +x, -y, +y, -z, +z; a face's free axes (u, v) are the
      other two axes in increasing order; Alg. 3 numbers the four sub-faces of a
      face 2 h_u + h_v (h = 0: lower half).
  R9  Source-side active directions use the same orientation c_(l)(t, s).
  R10 Eq. (13) uses l both as level and as column index; read E[k, l].
  R11 A coincident target/source pair contributes 0 (the zero diagonal of
      Sect. 4, generalised).
  R12 l_hf default: the largest level l <= p with kappa * w_l > 2 (w_l the box
      side), else -1; it gives the paper's l_hf = k - 4 for every k of Sect. 4.
"""
import math

import numpy as np

from .aca import aca_partial

FOUR_PI = 4.0 * math.pi


# --------------------------------------------------------------------------
# Kernel, Eqs. (1)-(3)
# --------------------------------------------------------------------------
def helmholtz(x, y, kappa):
    """f(x, y) = exp(i kappa |x-y|) / (4 pi |x-y|), Eq. (1); 0 where x == y (R11).

    x, y broadcast against each other over leading axes; last axis has size 3.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    same = np.all(x == y, axis=-1)
    rs = np.where(same, 1.0, r)
    f = np.exp(1j * kappa * rs) / (FOUR_PI * rs)
    return np.where(same, 0.0 + 0.0j, f)


def helmholtz_c(x, y, kappa, c):
    """f_c(x, y) = exp(i kappa (|x-y| - <x-y, c>)) / (4 pi |x-y|), Eq. (3)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    return np.exp(1j * kappa * (r - d @ np.asarray(c, dtype=np.float64))) / (FOUR_PI * r)


# --------------------------------------------------------------------------
# Chebyshev interpolation, Eq. (4) with reading R1
# --------------------------------------------------------------------------
def cheb_nodes(order):
    """Reference nodes cos((2 nu - 1) pi / (2 (m+1))), nu = 1 .. m+1 (R1)."""
    nu = np.arange(1, order + 1, dtype=np.float64)
    return np.cos((2.0 * nu - 1.0) * math.pi / (2.0 * order))


def lagrange_1d(order, t):
    """1-D Lagrange polynomials of the reference nodes at t: shape t.shape + (order,)."""
    r = cheb_nodes(order)
    t = np.asarray(t, dtype=np.float64)
    out = np.empty(t.shape + (order,), dtype=np.float64)
    for nu in range(order):
        v = np.ones_like(t)
        for mu in range(order):
            if mu != nu:
                v = v * (t - r[mu]) / (r[nu] - r[mu])
        out[..., nu] = v
    return out


def box_nodes(lo, hi, order):
    """Tensor nodes xi_{t,k} of box [lo, hi], k = nu_x + o nu_y + o^2 nu_z: (n, 3)."""
    r = cheb_nodes(order)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ax = [(lo[i] + hi[i]) / 2.0 + (hi[i] - lo[i]) / 2.0 * r for i in range(3)]
    zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def box_lagrange(lo, hi, order, pts):
    """L_{t,k}(x) (tensor Lagrange polynomials of box t) at points: (m, n).

    lo, hi: (3,) or (m, 3) box bounds belonging to each point.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    mid = (lo + hi) / 2.0
    half = (hi - lo) / 2.0
    t = (pts - mid) / half
    lx = lagrange_1d(order, t[:, 0])
    ly = lagrange_1d(order, t[:, 1])
    lz = lagrange_1d(order, t[:, 2])
    m = pts.shape[0]
    return (lz[:, :, None, None] * ly[:, None, :, None] * lx[:, None, None, :]).reshape(m, order ** 3)


# --------------------------------------------------------------------------
# Alg. 1: uniform box cluster tree
# --------------------------------------------------------------------------
class ClusterTree:
    """Uniform box cluster tree of Alg. 1 (with readings R3 - R5).

    Boxes get ids in the order Alg. 1 creates them (depth first, children in
    R4 order).  Per box: level, integer coordinates ijk on the level grid,
    bounds lo/hi, the ascending index set t^ (idx), parent and children.
    """

    def __init__(self, points, root_lo, root_side, n_max, max_depth):
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        if not np.all(np.isfinite(pts)):
            raise ValueError("points must be finite")
        root_lo = np.asarray(root_lo, dtype=np.float64).reshape(3)
        root_hi = root_lo + float(root_side)
        if pts.shape[0] and (np.any(pts < root_lo) or np.any(pts > root_hi)):
            raise ValueError("points outside the root box")
        self.points = pts
        self.root_lo = root_lo
        self.root_side = float(root_side)
        self.n_max = int(n_max)
        self.max_depth = int(max_depth)
        self.level, self.ijk, self.lo, self.hi = [], [], [], []
        self.idx, self.parent, self.children = [], [], []
        if pts.shape[0] == 0:
            raise ValueError("empty point set")
        root = self._add(0, np.zeros(3, dtype=np.int64), root_lo, root_hi,
                         np.arange(pts.shape[0], dtype=np.int64), -1)
        self._refine(root)
        self.nboxes = len(self.level)
        self.depth = max(self.level)
        self.by_level = [[] for _ in range(self.depth + 1)]
        for b, lv in enumerate(self.level):
            self.by_level[lv].append(b)
        self.is_leaf = [len(ch) == 0 for ch in self.children]
        self.leaves = [b for b in range(self.nboxes) if self.is_leaf[b]]
        self.key_to_box = {}
        for b in range(self.nboxes):
            self.key_to_box[(self.level[b],) + tuple(int(v) for v in self.ijk[b])] = b
        # Python-float copies of the bounds for the scalar admissibility test.
        self._lo_t = [tuple(float(v) for v in a) for a in self.lo]
        self._hi_t = [tuple(float(v) for v in a) for a in self.hi]

    def _add(self, level, ijk, lo, hi, idx, parent):
        self.level.append(level)
        self.ijk.append(ijk)
        self.lo.append(lo)
        self.hi.append(hi)
        self.idx.append(idx)
        self.parent.append(parent)
        self.children.append([])
        return len(self.level) - 1

    def _refine(self, b):
        """RefineCluster of Alg. 1."""
        idx = self.idx[b]
        if idx.size > self.n_max and self.level[b] < self.max_depth:
            lo, hi = self.lo[b], self.hi[b]
            c = (lo + hi) / 2.0                 # centre of the box
            upper = self.points[idx] > c        # (c_i, b_i] is the upper half
            q = upper[:, 0].astype(np.int64) + 2 * upper[:, 1] + 4 * upper[:, 2]
            for k in range(8):
                sel = idx[q == k]
                if sel.size >= 1:               # only non-empty children
                    bits = np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1], dtype=np.int64)
                    clo = np.where(bits == 1, c, lo)
                    chi = np.where(bits == 1, hi, c)
                    ch = self._add(self.level[b] + 1, 2 * self.ijk[b] + bits,
                                   clo, chi, sel, b)
                    self.children[b].append(ch)
                    self._refine(ch)

    def midpoint(self, b):
        return (self.lo[b] + self.hi[b]) / 2.0

    def leaf_of_point(self):
        """Array: leaf box id of every point."""
        out = np.empty(self.points.shape[0], dtype=np.int64)
        for b in self.leaves:
            out[self.idx[b]] = b
        return out


# --------------------------------------------------------------------------
# Def. 1: directional admissibility, (A1) and (A3)
# --------------------------------------------------------------------------
def admissibility(lo_t, hi_t, lo_s, hi_s, kappa, eta2):
    """(A1, A3) for the closed axis-parallel boxes t and s (Def. 1, R6)."""
    diam_t = math.sqrt(sum((hi_t[i] - lo_t[i]) ** 2 for i in range(3)))
    diam_s = math.sqrt(sum((hi_s[i] - lo_s[i]) ** 2 for i in range(3)))
    gap2 = 0.0
    for i in range(3):
        g = max(0.0, lo_s[i] - hi_t[i], lo_t[i] - hi_s[i])
        gap2 += g * g
    dist = math.sqrt(gap2)
    dmax = max(diam_t, diam_s)
    a1 = dmax <= eta2 * dist
    a3 = kappa * dmax * dmax <= eta2 * dist
    return a1, a3


# --------------------------------------------------------------------------
# Alg. 2 / Def. 2: block tree
# --------------------------------------------------------------------------
class BlockTree:
    """Leaves of the block tree of Alg. 2, split into L+ and L- (Def. 2).

    target_keep: optional boolean list over target boxes.  When given, the
    recursion only descends into blocks (t, s) whose t is kept: the blocks of
    Alg. 2 whose row set can meet the kept rows (used to evaluate selected rows
    of the product).  With target_keep=None this is Alg. 2 unchanged.
    """

    def __init__(self, tt, ts, kappa, eta2, target_keep=None):
        self.adm = []    # L+ : list of (t, s)
        self.near = []   # L- : list of (t, s)
        lo_t, hi_t, lo_s, hi_s = tt._lo_t, tt._hi_t, ts._lo_t, ts._hi_t
        stack = [(0, 0)]
        while stack:
            t, s = stack.pop()
            if target_keep is not None and not target_keep[t]:
                continue
            a1, a3 = admissibility(lo_t[t], hi_t[t], lo_s[s], hi_s[s], kappa, eta2)
            if tt.is_leaf[t] or ts.is_leaf[s]:
                (self.adm if (a1 and a3) else self.near).append((t, s))
                continue
            if not (a1 and a3):
                # push in reverse so that pairs are visited in the paper's order
                for t2 in reversed(tt.children[t]):
                    for s2 in reversed(ts.children[s]):
                        stack.append((t2, s2))
            else:
                self.adm.append((t, s))

    def stats(self, tt, ts):
        """N_C, N_SC, nearfield entries and their share (Table 1 quantities)."""
        n_c = len(self.adm)
        stored = set()
        for (t, s) in self.adm:
            d = tt.ijk[t] - ts.ijk[s]
            stored.add((tt.level[t], int(d[0]), int(d[1]), int(d[2])))
        nf_entries = 0
        for (t, s) in self.near:
            nf_entries += tt.idx[t].size * ts.idx[s].size
        total = tt.points.shape[0] * ts.points.shape[0]
        return {"N_C": n_c, "N_SC": len(stored), "near_blocks": len(self.near),
                "nf_entries": nf_entries, "nf_percent": 100.0 * nf_entries / total}


# --------------------------------------------------------------------------
# Sect. 2.4: high-frequency levels, Alg. 3 directions, Def. 3 direction map
# --------------------------------------------------------------------------
def default_l_hf(kappa, root_side, p):
    """Reading R12 of Eq. (11): largest l <= p with kappa * w_l > 2, else -1."""
    l_hf = -1
    for lv in range(p + 1):
        if kappa * (root_side / 2.0 ** lv) > 2.0:
            l_hf = lv
    return l_hf


_FACES0 = [(0, -1.0), (0, 1.0), (1, -1.0), (1, 1.0), (2, -1.0), (2, 1.0)]


class Directions:
    """D^(l) of Alg. 3 and the map dir_(l) of Def. 3 for levels 0 .. p.

    Directions are referred to by their index j (0-based) in D^(l); on
    low-frequency levels D^(l) = {0} has the single index 0 (the zero vector).
    """

    def __init__(self, l_hf, p):
        self.l_hf = int(l_hf)
        self.p = int(p)
        self.faces = {}
        self.vectors = {}
        for lv in range(self.l_hf + 1, self.p + 1):
            self.vectors[lv] = np.zeros((1, 3))
        if self.l_hf >= 0:
            faces = []
            for axis, sign in _FACES0:
                faces.append((axis, sign, -1.0, 1.0, -1.0, 1.0))
            self.faces[self.l_hf] = faces
            for lv in range(self.l_hf - 1, -1, -1):
                new = []
                for (axis, sign, ulo, uhi, vlo, vhi) in self.faces[lv + 1]:
                    um, vm = (ulo + uhi) / 2.0, (vlo + vhi) / 2.0
                    for hu in (0, 1):          # sub-face 2 h_u + h_v (R8)
                        for hv in (0, 1):
                            new.append((axis, sign,
                                        (ulo, um)[hu], (um, uhi)[hu],
                                        (vlo, vm)[hv], (vm, vhi)[hv]))
                self.faces[lv] = new
            for lv in range(0, self.l_hf + 1):
                vecs = []
                for (axis, sign, ulo, uhi, vlo, vhi) in self.faces[lv]:
                    u, v = [a for a in range(3) if a != axis]
                    mid = np.zeros(3)
                    mid[axis] = sign
                    mid[u] = (ulo + uhi) / 2.0
                    mid[v] = (vlo + vhi) / 2.0
                    vecs.append(mid / np.linalg.norm(mid))   # normalised midpoint
                self.vectors[lv] = np.array(vecs)

    def count(self, lv):
        return self.vectors[lv].shape[0]

    def vector(self, lv, j):
        return self.vectors[lv][j]

    def dir(self, lv, v):
        """dir_(l)(v) of Def. 3, as an index into D^(l)."""
        if lv > self.l_hf:
            return 0
        v = np.asarray(v, dtype=np.float64)
        m = float(np.max(np.abs(v)))
        if m == 0.0:
            raise ValueError("dir_(l)(0) on a high-frequency level is never needed")
        psi = v / m
        for j, (axis, sign, ulo, uhi, vlo, vhi) in enumerate(self.faces[lv]):
            u, w = [a for a in range(3) if a != axis]
            if (psi[axis] == sign and ulo <= psi[u] <= uhi
                    and vlo <= psi[w] <= vhi):
                return j                       # smallest j whose face holds psi
        raise AssertionError("no face contains psi")


# --------------------------------------------------------------------------
# The oracle
# --------------------------------------------------------------------------
class FDMOracle:
    """Alg. 4 over the trees of Alg. 1, the partition of Alg. 2 and the
    directions of Alg. 3 / Def. 3 / Def. 5, all in FP64.

    Parameters mirror the paper: points P_T, P_S, wave number kappa, order
    o = m + 1, eta2, l_hf (None: reading R12), n_max and max_depth (R5), and the
    common root cube (root_lo, root_side) (R3).
    """

    def __init__(self, targets, sources, kappa, order, root_lo, root_side,
                 max_depth, n_max=0, eta2=5.0, l_hf=None):
        self.kappa = float(kappa)
        self.order = int(order)
        self.n = self.order ** 3
        self.eta2 = float(eta2)
        self.tt = ClusterTree(targets, root_lo, root_side, n_max, max_depth)
        self.ts = ClusterTree(sources, root_lo, root_side, n_max, max_depth)
        p_min = min(self.tt.depth, self.ts.depth)
        p_max = max(self.tt.depth, self.ts.depth)
        self.l_hf = default_l_hf(self.kappa, float(root_side), p_min) if l_hf is None else int(l_hf)
        self.dirs = Directions(self.l_hf, p_max)
        self.ref_nodes = cheb_nodes(self.order)
        self._c_cache = {}
        self._child_dir_cache = {}

    # ---------------------------------------------------------------- pieces
    def block_tree(self, target_keep=None):
        return BlockTree(self.tt, self.ts, self.kappa, self.eta2, target_keep)

    def c_of_block(self, t, s):
        """c_(l)(t, s) of Def. 3 (index into D^(l)), evaluated on m_t - m_s (R7).

        m_t - m_s depends only on the level and the integer box offset, so the
        value is cached per (level, offset).
        """
        lv = self.tt.level[t]
        d = self.tt.ijk[t] - self.ts.ijk[s]
        key = (lv, int(d[0]), int(d[1]), int(d[2]))
        c = self._c_cache.get(key)
        if c is None:
            c = self.dirs.dir(lv, self.tt.midpoint(t) - self.ts.midpoint(s))
            self._c_cache[key] = c
        return c

    def child_dir(self, lv, c):
        """dir_(l+1)(c) for c in D^(l), cached."""
        key = (lv, c)
        c2 = self._child_dir_cache.get(key)
        if c2 is None:
            c2 = self.dirs.dir(lv + 1, self.dirs.vector(lv, c))
            self._child_dir_cache[key] = c2
        return c2

    def _direction_sets(self, blocks):
        """Def. 5: D(t) u D^(t) for target boxes and D(s) u D^(s) for source boxes."""
        tt, ts, dirs = self.tt, self.ts, self.dirs
        act_t = [set() for _ in range(tt.nboxes)]
        act_s = [set() for _ in range(ts.nboxes)]
        for (t, s) in blocks.adm:
            c = self.c_of_block(t, s)
            act_t[t].add(c)
            act_s[s].add(c)          # same orientation on the source side (R9)

        def closure(tree, act):
            full = [None] * tree.nboxes
            for lv in range(tree.depth + 1):
                for b in tree.by_level[lv]:
                    inh = set()
                    if lv > 0:
                        par = tree.parent[b]
                        for c in full[par]:
                            inh.add(self.child_dir(lv - 1, c))
                    full[b] = act[b] | inh
            return full
        return closure(tt, act_t), closure(ts, act_s)

    def _dir_pair(self, lv, c):
        """(c vector at level lv, c' = dir_(lv+1)(c) and its vector at lv+1)."""
        cv = self.dirs.vector(lv, c)
        c2 = self.child_dir(lv, c)
        return cv, c2, self.dirs.vector(lv + 1, c2)

    def transfer_matrix(self, tree, child, cv, c2v):
        """E_{t',c}[k, l] = exp(i kappa <xi_{t',k}, c - c'>) L_{t,l}(xi_{t',k}), Eq. (13)."""
        par = tree.parent[child]
        xi = box_nodes(tree.lo[child], tree.hi[child], self.order)
        lag = box_lagrange(tree.lo[par], tree.hi[par], self.order, xi)
        return np.exp(1j * self.kappa * (xi @ (cv - c2v)))[:, None] * lag

    def coupling_matrix(self, t, s, cv):
        """A_{c,t x s}[j, k] = f_c(xi_{t,j}, xi_{s,k}), Eq. (9)."""
        xt = box_nodes(self.tt.lo[t], self.tt.hi[t], self.order)
        xs = box_nodes(self.ts.lo[s], self.ts.hi[s], self.order)
        return helmholtz_c(xt[:, None, :], xs[None, :, :], self.kappa, cv)

    def interpolation_matrix(self, tree, b, cv):
        """L_{t,c}[j, k] = L_{t,k}(x_j) exp(i kappa <x_j, c>), Eqs. (6), (10)."""
        pts = tree.points[tree.idx[b]]
        lag = box_lagrange(tree.lo[b], tree.hi[b], self.order, pts)
        return lag * np.exp(1j * self.kappa * (pts @ cv))[:, None]

    # ----------------------------------------------------------------- Alg. 4
    def apply(self, x, rows=None, mode="reuse", aca_tol=1e-8):
        """g = A v by Alg. 4.  Returns g at `rows` (all target rows when None).

        mode="literal": every L, E and A matrix is formed for its own block
        from Eqs. (9), (10), (13), in Alg. 4's loop order.
        mode="reuse": Sect. 2.7 -- each coupling matrix is formed once per
        level and box offset, each E_{t'} once per level and octant, and the
        diagonal directional part E^d is applied separately; the M2L updates
        that share a stored matrix are applied as one matrix product.
        mode="aca": as "reuse", with every stored coupling matrix replaced by
        its partially pivoted ACA U V^* to relative tolerance aca_tol (Sect.
        2.7, closing remark); the ranks are left in self.last_aca_ranks.
        With rows given, only the blocks of Alg. 2 whose target box contains a
        requested row (or an ancestor of one) are formed and applied.
        """
        if mode not in ("literal", "reuse", "aca"):
            raise ValueError(mode)
        tt, ts, dirs = self.tt, self.ts, self.dirs
        kappa, n = self.kappa, self.n
        v = np.asarray(x, dtype=np.complex128).reshape(-1)
        assert v.shape[0] == ts.points.shape[0]

        keep = None
        if rows is not None:
            rows = np.asarray(rows, dtype=np.int64)
            leaf_of = tt.leaf_of_point()
            keep = [False] * tt.nboxes
            for b in set(int(leaf_of[r]) for r in rows):
                while b >= 0 and not keep[b]:
                    keep[b] = True
                    b = tt.parent[b]
        blocks = self.block_tree(keep)
        dset_t, dset_s = self._direction_sets(blocks)

        # slots: one vector of n coefficients per (box, direction)
        vt = {}   # (s, c) -> source moments tilde v_{s,c}
        gt = {}   # (t, c) -> local coefficients tilde g_{t,c}

        # ---- forward transformation: S2M (lines for leaves of T_S)
        s2m_slots = [(s, c) for s in ts.leaves for c in sorted(dset_s[s])]
        if mode == "literal":
            for (s, c) in s2m_slots:
                cv = dirs.vector(ts.level[s], c)
                lmat = self.interpolation_matrix(ts, s, cv)
                vt[(s, c)] = lmat.conj().T @ v[ts.idx[s]]
        else:
            self._s2m_vectorised(s2m_slots, v, vt)

        # ---- forward transformation: M2M, levels p(T_S)-1 .. 0
        eref_s = {}
        for lv in range(ts.depth - 1, -1, -1):
            if mode == "reuse":
                self._m2m_level_reuse(lv, dset_s, vt, eref_s)
                continue
            for s in ts.by_level[lv]:
                if ts.is_leaf[s]:
                    continue
                for c in sorted(dset_s[s]):
                    cv, c2, c2v = self._dir_pair(lv, c)
                    acc = np.zeros(n, dtype=np.complex128)
                    for s2 in ts.children[s]:
                        emat = self.transfer_matrix(ts, s2, cv, c2v)
                        acc += emat.conj().T @ vt[(s2, c2)]
                    vt[(s, c)] = acc

        # ---- multiplication phase: M2L
        for t in range(tt.nboxes):
            for c in dset_t[t]:
                gt[(t, c)] = np.zeros(n, dtype=np.complex128)
        if mode == "literal":
            by_t = {}
            for (t, s) in blocks.adm:
                by_t.setdefault(t, []).append(s)
            for t in range(tt.nboxes):
                for s in by_t.get(t, ()):
                    c = self.c_of_block(t, s)
                    cv = dirs.vector(tt.level[t], c)
                    gt[(t, c)] += self.coupling_matrix(t, s, cv) @ vt[(s, c)]
        else:
            groups = {}
            aca_ranks = {}
            self.last_aca_ranks = aca_ranks
            for (t, s) in blocks.adm:
                d = tt.ijk[t] - ts.ijk[s]
                key = (tt.level[t], int(d[0]), int(d[1]), int(d[2]))
                groups.setdefault(key, []).append((t, s))
            for key, pairs in groups.items():
                t0, s0 = pairs[0]
                c = self.c_of_block(t0, s0)
                cv = dirs.vector(tt.level[t0], c)
                amat = self.coupling_matrix(t0, s0, cv)   # reference configuration
                vin = np.stack([vt[(s, c)] for (_, s) in pairs], axis=1)
                if mode == "aca":
                    u, w = aca_partial(amat, aca_tol)
                    aca_ranks[key] = u.shape[1]
                    out = u @ (w.conj().T @ vin)
                else:
                    out = amat @ vin
                for i, (t, _) in enumerate(pairs):
                    gt[(t, c)] += out[:, i]

        # ---- backward transformation: L2L, levels 0 .. p(T_T)-1
        eref_t = {}
        for lv in range(0, tt.depth):
            for t in tt.by_level[lv]:
                if tt.is_leaf[t] or (keep is not None and not keep[t]):
                    continue
                for c in sorted(dset_t[t]):
                    cv, c2, c2v = self._dir_pair(lv, c)
                    for t2 in tt.children[t]:
                        if keep is not None and not keep[t2]:
                            continue
                        if mode == "literal":
                            emat = self.transfer_matrix(tt, t2, cv, c2v)
                        else:
                            emat = self._transfer_reuse(tt, t2, cv, c2v, eref_t)
                        gt[(t2, c2)] += emat @ gt[(t, c)]

        # ---- backward transformation: L2T
        g = np.zeros(tt.points.shape[0], dtype=np.complex128)
        for t in tt.leaves:
            if keep is not None and not keep[t]:
                continue
            for c in sorted(dset_t[t]):
                cv = dirs.vector(tt.level[t], c)
                lmat = self.interpolation_matrix(tt, t, cv)
                g[tt.idx[t]] += lmat @ gt[(t, c)]

        # ---- nearfield evaluation
        for (t, s) in blocks.near:
            it = tt.idx[t]
            isrc = ts.idx[s]
            amat = helmholtz(tt.points[it][:, None, :], ts.points[isrc][None, :, :], kappa)
            g[it] += amat @ v[isrc]

        self.last_blocks = blocks
        if rows is None:
            return g
        return g[rows]

    # --------------------------------------------------------- reuse helpers
    def _transfer_reuse(self, tree, child, cv, c2v, cache):
        """E_{t',c} = E^d_{t',c} E_{t'} with E_{t'} one of 8 reference matrices
        per level (Sect. 2.7); E^d is the diagonal directional part."""
        lv = tree.level[child]
        octant = tuple(int(b) for b in (tree.ijk[child] & 1))
        key = (lv, octant)
        if key not in cache:
            par = tree.parent[child]
            xi = box_nodes(tree.lo[child], tree.hi[child], self.order)
            cache[key] = box_lagrange(tree.lo[par], tree.hi[par], self.order, xi)
        xi = box_nodes(tree.lo[child], tree.hi[child], self.order)
        ed = np.exp(1j * self.kappa * (xi @ (cv - c2v)))
        return ed[:, None] * cache[key]

    def _reference_transfer(self, tree, child, cache):
        """Non-directional part E_{t'} of the child's octant (Sect. 2.7)."""
        lv = tree.level[child]
        octant = tuple(int(b) for b in (tree.ijk[child] & 1))
        key = (lv, octant)
        if key not in cache:
            par = tree.parent[child]
            xi = box_nodes(tree.lo[child], tree.hi[child], self.order)
            cache[key] = box_lagrange(tree.lo[par], tree.hi[par], self.order, xi)
        return cache[key]

    def _m2m_level_reuse(self, lv, dset_s, vt, cache, chunk=4096):
        """M2M of one level with E_{s',c}^* = E_{s'}^T (E^d_{s',c})^*: for every
        non-leaf s on level lv and c in D(s) u D^(s),
        tilde v_{s,c} = sum_{s'} E_{s',c}^* tilde v_{s',c'}  (Alg. 4, Eq. 13)."""
        ts, n, kappa = self.ts, self.n, self.kappa
        r = self.ref_nodes
        offs = np.stack(np.meshgrid(r, r, r, indexing="ij")[::-1], axis=-1).reshape(n, 3)
        parents = []
        items = {}   # reference matrix key -> list of (parent slot, child key, c - c', child box)
        for s in ts.by_level[lv]:
            if ts.is_leaf[s]:
                continue
            for c in sorted(dset_s[s]):
                cv, c2, c2v = self._dir_pair(lv, c)
                ps = len(parents)
                parents.append((s, c))
                for s2 in ts.children[s]:
                    octant = tuple(int(b) for b in (ts.ijk[s2] & 1))
                    self._reference_transfer(ts, s2, cache)
                    items.setdefault((lv + 1, octant), []).append((ps, (s2, c2), cv - c2v, s2))
        acc = np.zeros((len(parents), n), dtype=np.complex128)
        for key, lst in items.items():
            eref = cache[key]
            for i0 in range(0, len(lst), chunk):
                part = lst[i0:i0 + chunk]
                ps = np.array([it[0] for it in part], dtype=np.int64)
                u = np.stack([vt[it[1]] for it in part])
                dc = np.array([it[2] for it in part])
                if np.any(dc != 0.0):
                    lo = np.array([ts.lo[it[3]] for it in part])
                    hi = np.array([ts.hi[it[3]] for it in part])
                    xi = (lo + hi)[:, None, :] / 2.0 + (hi - lo)[:, None, :] / 2.0 * offs[None]
                    ed = np.exp(1j * kappa * np.einsum("pkd,pd->pk", xi, dc))
                    u = u * ed.conj()
                np.add.at(acc, ps, u @ eref)
        for i, key in enumerate(parents):
            vt[key] = acc[i]

    def _s2m_vectorised(self, slots, v, vt, chunk=1 << 16):
        """S2M for many (leaf, direction) slots at once: tilde v = L_{s,c}^* v|_s."""
        ts, dirs, kappa = self.ts, self.dirs, self.kappa
        if not slots:
            return
        counts = np.array([ts.idx[s].size for (s, _) in slots], dtype=np.int64)
        pidx = np.concatenate([ts.idx[s] for (s, _) in slots])
        owner = np.repeat(np.arange(len(slots)), counts)
        lo = np.array([ts.lo[s] for (s, _) in slots])
        hi = np.array([ts.hi[s] for (s, _) in slots])
        cvec = np.array([dirs.vector(ts.level[s], c) for (s, c) in slots])
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        out = np.zeros((len(slots), self.n), dtype=np.complex128)
        # process whole slots per chunk so that reduceat segments stay intact
        slot_lo = 0
        while slot_lo < len(slots):
            slot_hi = slot_lo
            total = 0
            while slot_hi < len(slots) and (total + counts[slot_hi] <= chunk or slot_hi == slot_lo):
                total += counts[slot_hi]
                slot_hi += 1
            p0, p1 = starts[slot_lo], starts[slot_lo] + total
            own = owner[p0:p1]
            pts = ts.points[pidx[p0:p1]]
            lag = box_lagrange(lo[own], hi[own], self.order, pts)
            ph = np.exp(-1j * kappa * np.sum(pts * cvec[own], axis=1))
            w = lag * (ph * v[pidx[p0:p1]])[:, None]
            seg = starts[slot_lo:slot_hi] - p0
            out[slot_lo:slot_hi] = np.add.reduceat(w, seg, axis=0)
            slot_lo = slot_hi
        for i, key in enumerate(slots):
            vt[key] = out[i]
