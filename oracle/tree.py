"""Level-restricted quadtree and interaction lists (Section 3.1, Fig. 1).

Box geometry is integer only. The root (level 0) is the box of centre (cx, cy)
and width W; a box at level l has width h_l = W 2^-l and integer coordinates
(ix, iy) in [0, 2^l)^2; its centre is lo + (i + 1/2) h_l with lo = c - W/2.

Readings of the paper taken here:
* Level restriction (Section 3.1): adjacent leaves are at most one level apart,
  where "adjacent" includes contact at a single corner.
* Refinement (Section 3.1; the refinement tolerance of Section 6.1): a box at
  level l < max_depth is split when the largest trailing Chebyshev coefficient of
  its interpolant (last two rows and columns) exceeds tol * F, with F = max |f|
  over the nodes of the uniform tree of level min(5, max_depth). Boxes above
  min_depth are always split.
* The a-priori alternatives of Section 6.1 ("A note on adaptivity"): the same
  comparison with the interpolation error e (max |f - p| on the nodes of the four
  children, the "finer grid"), unweighted, times the relative area (h/W)^2, or times
  the area for boxes that meet the boundary and the relative side length h/W
  elsewhere. Readings: the weights are relative to the root width W so that tol
  stays dimensionless; a box meets the boundary when the kinked source's level set
  takes both signs on those nodes (the paper's boundary is where f_e is only C^0).
* Canonical order: boxes sorted by (level, Morton key); the Morton key puts
  bit b of ix at bit 2b and bit b of iy at bit 2b + 1. Lists are sorted by box
  index.
* Lists (the standard adaptive-FMM lists; Fig. 1 shows the near/far split):
    U(b), b leaf: b and every leaf adjacent to b.
    V(b): children of the colleagues of parent(b) that are not adjacent to b.
    W(b), b leaf: children of the colleagues of b that are not adjacent to b.
    X(b): leaves c with b in W(c).
"""
from __future__ import annotations

import numpy as np

from . import cheb
from . import source as srcmod


def morton(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    ix = np.asarray(ix, dtype=np.int64)
    iy = np.asarray(iy, dtype=np.int64)
    key = np.zeros(np.broadcast(ix, iy).shape, dtype=np.int64)
    for b in range(31):
        key |= ((ix >> b) & 1) << (2 * b)
        key |= ((iy >> b) & 1) << (2 * b + 1)
    return key


def node_coords(cx: float, cy: float, width: float, k: int, level, ix, iy):
    """Coordinates of the k*k nodes of boxes (level, ix, iy): arrays [n, k*k].

    x = lo_x + ((ix + 0.5) + xhat_i) * h with h = width * 2^-level, evaluated in
    exactly this order (no fused multiply-add).
    """
    xh = cheb.nodes(k)
    level = np.asarray(level, dtype=np.int64).reshape(-1)
    ix = np.asarray(ix, dtype=np.int64).reshape(-1)
    iy = np.asarray(iy, dtype=np.int64).reshape(-1)
    h = width * np.ldexp(1.0, -level)
    lox = cx - width / 2.0
    loy = cy - width / 2.0
    gi = np.tile(np.arange(k), k)      # x index of flat node j*k + i
    gj = np.repeat(np.arange(k), k)    # y index
    X = lox + ((ix[:, None] + 0.5) + xh[gi][None, :]) * h[:, None]
    Y = loy + ((iy[:, None] + 0.5) + xh[gj][None, :]) * h[:, None]
    return X, Y


class Tree:
    """Canonically ordered level-restricted quadtree."""

    def __init__(self, cx, cy, width, k, boxes):
        self.cx, self.cy, self.width, self.k = float(cx), float(cy), float(width), int(k)
        arr = np.array(sorted(boxes), dtype=np.int64).reshape(-1, 3)
        lev, ix, iy = arr[:, 0], arr[:, 1], arr[:, 2]
        order = np.lexsort((morton(ix, iy), lev))
        self.level = lev[order].astype(np.int32)
        self.ix = ix[order].astype(np.int32)
        self.iy = iy[order].astype(np.int32)
        n = self.level.shape[0]
        self.n_boxes = n
        self.depth = int(self.level.max())
        self.index = {(int(l), int(a), int(b)): i for i, (l, a, b) in
                      enumerate(zip(self.level, self.ix, self.iy))}
        self.parent = np.full(n, -1, dtype=np.int32)
        self.child = np.full((n, 4), -1, dtype=np.int32)
        for i in range(n):
            l, a, b = int(self.level[i]), int(self.ix[i]), int(self.iy[i])
            if l > 0:
                p = self.index[(l - 1, a >> 1, b >> 1)]
                self.parent[i] = p
                self.child[p, ((b & 1) << 1) | (a & 1)] = i
        has = self.child >= 0
        if np.any(has.any(axis=1) != has.all(axis=1)):
            raise ValueError("a split box lacks one of its four children")
        self.is_leaf = ~has.any(axis=1)
        self.leaves = np.nonzero(self.is_leaf)[0].astype(np.int32)
        self.leaf_index = np.full(n, -1, dtype=np.int32)
        self.leaf_index[self.leaves] = np.arange(self.leaves.shape[0], dtype=np.int32)
        self.n_leaves = int(self.leaves.shape[0])
        self.level_start = np.searchsorted(self.level, np.arange(self.depth + 2)).astype(np.int32)

    def h(self, b):
        return self.width * np.ldexp(1.0, -np.asarray(self.level[b], dtype=np.int64))

    def centre(self, b):
        h = self.h(b)
        return (self.cx - self.width / 2.0 + (self.ix[b] + 0.5) * h,
                self.cy - self.width / 2.0 + (self.iy[b] + 0.5) * h)

    def leaf_nodes(self):
        """Node coordinates of all leaves, [n_leaves, k*k] each (canonical leaf order)."""
        b = self.leaves
        return node_coords(self.cx, self.cy, self.width, self.k, self.level[b], self.ix[b], self.iy[b])

    def sample(self, src):
        X, Y = self.leaf_nodes()
        return srcmod.evaluate_source(src, X, Y)


# ----------------------------------------------------------------------------- geometry

def _span(level, i, top):
    """Closed interval of a box side in units of the level-`top` grid."""
    s = 1 << (top - level)
    return i * s, (i + 1) * s


def touching(la, ax, ay, lb, bx, by) -> bool:
    """Closed boxes share at least one point."""
    top = max(la, lb)
    a0, a1 = _span(la, ax, top)
    b0, b1 = _span(lb, bx, top)
    c0, c1 = _span(la, ay, top)
    d0, d1 = _span(lb, by, top)
    return a0 <= b1 and b0 <= a1 and c0 <= d1 and d0 <= c1


def overlapping(la, ax, ay, lb, bx, by) -> bool:
    """Open boxes share interior points."""
    top = max(la, lb)
    a0, a1 = _span(la, ax, top)
    b0, b1 = _span(lb, bx, top)
    c0, c1 = _span(la, ay, top)
    d0, d1 = _span(lb, by, top)
    return a0 < b1 and b0 < a1 and c0 < d1 and d0 < c1


def adjacent(la, ax, ay, lb, bx, by) -> bool:
    return touching(la, ax, ay, lb, bx, by) and not overlapping(la, ax, ay, lb, bx, by)


# ----------------------------------------------------------------------------- build

def _children(boxes):
    out = []
    for (l, a, b) in boxes:
        for c in range(4):
            out.append((l + 1, 2 * a + (c & 1), 2 * b + (c >> 1)))
    return out


def balance(boxes: set) -> set:
    """Smallest refinement satisfying the level restriction (ripple to a fixpoint).

    For every box B at level l >= 2, each level-(l-1) cell adjacent to B must be a
    box of the tree; when one is missing, the leaf covering it is split. Every
    split is forced, so the fixpoint is the minimal balanced refinement.
    """
    boxes = set(boxes)
    work = sorted(boxes, key=lambda t: t[0])  # pop() takes the finest first
    while work:
        l, a, b = work.pop()
        if l < 2:
            continue
        pa, pb = a >> 1, b >> 1
        n = 1 << (l - 1)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                qa, qb = pa + dx, pb + dy
                if (dx == 0 and dy == 0) or not (0 <= qa < n and 0 <= qb < n):
                    continue
                if not adjacent(l - 1, qa, qb, l, a, b):
                    continue
                if (l - 1, qa, qb) in boxes:
                    continue
                # walk up to the leaf that covers the missing cell and split it
                m, ca, cb = l - 1, qa, qb
                while (m, ca, cb) not in boxes:
                    m, ca, cb = m - 1, ca >> 1, cb >> 1
                kids = _children([(m, ca, cb)])
                for kid in kids:
                    if kid not in boxes:
                        boxes.add(kid)
                        work.append(kid)
                work.append((l, a, b))  # re-check B once the new boxes exist
    return boxes


def build_uniform(cx, cy, width, k, depth) -> Tree:
    boxes = [(0, 0, 0)]
    cur = [(0, 0, 0)]
    for _ in range(depth):
        cur = _children(cur)
        boxes += cur
    return Tree(cx, cy, width, k, boxes)


def f_scale(cx, cy, width, k, src, max_depth) -> float:
    """F = max |f| over the nodes of the uniform tree of level min(5, max_depth)."""
    m = min(5, max_depth)
    n = 1 << m
    ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    X, Y = node_coords(cx, cy, width, k, np.full(n * n, m), ix.reshape(-1), iy.reshape(-1))
    return float(np.max(np.abs(srcmod.evaluate_source(src, X, Y))))


RULES = ("tail", "interp", "interp_area", "interp_mixed")


def child_grid(cx, cy, width, k, level, ix, iy):
    """The 2k x 2k grid of the nodes of the four children of each box: X, Y [n, 2k, 2k] indexed
    [J, I], child column I // k and node I % k (rows likewise), i.e. the nodes of box
    (level + 1, 2 ix + I // k, 2 iy + J // k)."""
    level = np.asarray(level, dtype=np.int64).reshape(-1)
    ix = np.asarray(ix, dtype=np.int64).reshape(-1)
    iy = np.asarray(iy, dtype=np.int64).reshape(-1)
    n = level.shape[0]
    X = np.empty((n, 2 * k, 2 * k))
    Y = np.empty((n, 2 * k, 2 * k))
    for d in range(2):
        for c in range(2):
            Xc, Yc = node_coords(cx, cy, width, k, level + 1, 2 * ix + c, 2 * iy + d)
            X[:, d * k:(d + 1) * k, c * k:(c + 1) * k] = Xc.reshape(n, k, k)
            Y[:, d * k:(d + 1) * k, c * k:(c + 1) * k] = Yc.reshape(n, k, k)
    return X, Y


def interp_error(cx, cy, width, k, src, level, ix, iy):
    """The paper's a-priori test quantity (Section 6.1): the error of the box's interpolant of f,
    found by comparing f with it on a finer grid, here the nodes of the box's four children:
    e = max |f - p| over that grid, p interpolating f at the box's own k x k nodes (Lagrange
    basis of cheb.lagrange at the child nodes' positions in the box's unit coordinates).
    Also whether the box meets the boundary: for the kinked source, the level set phi (whose
    zero set is the curve where f is only continuous) takes both signs on the box's own and
    children's nodes; other sources have no boundary. Returns (e [n], meets_boundary [n])."""
    X, Y = node_coords(cx, cy, width, k, level, ix, iy)
    V = srcmod.evaluate_source(src, X, Y).reshape(-1, k, k)
    Xc, Yc = child_grid(cx, cy, width, k, level, ix, iy)
    Fc = srcmod.evaluate_source(src, Xc, Yc)
    u = np.concatenate([-0.25 + cheb.nodes(k) / 2.0, 0.25 + cheb.nodes(k) / 2.0])
    L = cheb.lagrange(k, u)  # [2k, k]
    P = np.einsum("Jj,nji,Ii->nJI", L, V, L)
    e = np.max(np.abs(Fc - P).reshape(V.shape[0], -1), axis=1)
    meets = np.zeros(V.shape[0], dtype=bool)
    if getattr(src, "kind", None) == srcmod.SRC_KINKED:
        ph = np.concatenate([srcmod.kinked_phi(np.asarray(src.params), X, Y).reshape(V.shape[0], -1),
                             srcmod.kinked_phi(np.asarray(src.params), Xc, Yc).reshape(V.shape[0], -1)], axis=1)
        meets = np.any(ph > 0.0, axis=1) & np.any(ph <= 0.0, axis=1)
    return e, meets


def rule_indicator(rule, cx, cy, width, k, src, level, ix, iy, C=None):
    """Quantity compared with tol * F for each box (split when larger), per refinement rule:
    "tail" the trailing Chebyshev coefficients (Section 3.1 reading), "interp" the interpolation
    error e, "interp_area" e (h / W)^2, "interp_mixed" e (h / W)^2 for boxes that meet the boundary
    and e (h / W) elsewhere (Section 6.1, the weightings by area and by side length)."""
    level = np.asarray(level, dtype=np.int64).reshape(-1)
    if rule == "tail":
        X, Y = node_coords(cx, cy, width, k, level, ix, iy)
        V = srcmod.evaluate_source(src, X, Y).reshape(-1, k, k)
        return cheb.tail(V, k, C)
    if rule not in RULES:
        raise ValueError("unknown refinement rule %r" % rule)
    e, meets = interp_error(cx, cy, width, k, src, level, ix, iy)
    side = np.ldexp(1.0, -level)
    if rule == "interp":
        return e
    if rule == "interp_area":
        return e * side * side
    return np.where(meets, e * side * side, e * side)


def build_adaptive(cx, cy, width, k, src, tol, max_depth, min_depth=0, return_info=False, rule="tail"):
    """Level-by-level refinement followed by balancing (Section 3.1); rule as rule_indicator."""
    C = cheb.values_to_coeffs_matrix(k)
    F = f_scale(cx, cy, width, k, src, max_depth)
    thresh = tol * F
    boxes = [(0, 0, 0)]
    cur = [(0, 0, 0)]
    margins = []
    for l in range(max_depth):
        if not cur:
            break
        arr = np.array(cur, dtype=np.int64)
        if l < min_depth:
            split = np.ones(len(cur), dtype=bool)
        else:
            tl = rule_indicator(rule, cx, cy, width, k, src, arr[:, 0], arr[:, 1], arr[:, 2], C)
            split = tl > thresh
            if thresh > 0:
                margins.append(np.abs(tl / thresh - 1.0))
        cur = _children([cur[i] for i in np.nonzero(split)[0]])
        boxes += cur
    # leaves the depth cap stopped: boxes created at level max_depth that the test would still split
    n_capped = 0
    if cur and (max_depth == 0 or cur[0][0] == max_depth):
        arr = np.array(cur, dtype=np.int64)
        n_capped = int(np.sum(rule_indicator(rule, cx, cy, width, k, src, arr[:, 0], arr[:, 1], arr[:, 2], C) > thresh))
    refined = set(boxes)
    boxes = balance(refined)
    tree = Tree(cx, cy, width, k, boxes)
    if return_info:
        mm = float(np.min(np.concatenate(margins))) if margins else float("inf")
        return tree, {"F": F, "min_margin": mm, "refined": refined, "n_capped": n_capped}
    return tree


def build_greedy(cx, cy, width, k, src, n_leaves, max_depth=16, return_info=False):
    """Leaf-count target for batches of uneven problems (the paper refines to a tolerance only).

    One split at a time: the leaf of highest priority is split until the tree has at least
    n_leaves leaves or no leaf below max_depth remains; then balance() as for the tolerance
    rule. Priority = binary exponent e of the leaf's tail (the tolerance rule's quantity, with
    tail in [2^(e-1), 2^e)), raised to at least e_F - 30 (F = f_scale = m 2^e_F, m in [0.5, 1)),
    so that tails near rounding level all tie; ties: coarser level first, then smaller Morton key.
    info["min_margin"]: smallest relative distance of a deciding tail to a power of two.
    """
    import heapq
    import math
    C = cheb.values_to_coeffs_matrix(k)
    F = f_scale(cx, cy, width, k, src, max_depth)
    e_floor = (math.frexp(F)[1] if F > 0 else 0) - 30
    margin = [float("inf")]

    def tails(boxes):
        arr = np.array(boxes, dtype=np.int64)
        X, Y = node_coords(cx, cy, width, k, arr[:, 0], arr[:, 1], arr[:, 2])
        return cheb.tail(srcmod.evaluate_source(src, X, Y).reshape(-1, k, k), k, C)

    def priority(t):
        e = e_floor
        if t > 0:
            e = math.frexp(t)[1]
            if e >= e_floor:
                lo, hi = math.ldexp(1.0, e - 1), math.ldexp(1.0, e)
                margin[0] = min(margin[0], t / lo - 1.0, 1.0 - t / hi)
        return max(e, e_floor)

    def entry(box, t):
        l, a, b = box
        return (-priority(float(t)), l, int(morton(np.array([a]), np.array([b]))[0]), box)

    root = (0, 0, 0)
    heap = [entry(root, tails([root])[0])] if max_depth > 0 else []
    boxes = {root}
    n = 1
    while n < n_leaves and heap:
        _, l, _, box = heapq.heappop(heap)
        kids = _children([box])
        tk = tails(kids)
        boxes.update(kids)
        n += 3
        for kid, t in zip(kids, tk):
            e = entry(kid, t)  # every child's tail decides a priority (also at max_depth)
            if l + 1 < max_depth:
                heapq.heappush(heap, e)
    refined = set(boxes)
    tree = Tree(cx, cy, width, k, balance(refined))
    if return_info:
        return tree, {"F": F, "min_margin": margin[0], "refined": refined}
    return tree


# ----------------------------------------------------------------------------- lists

NEAR_PATTERN = sorted([(sx * a, sy * b) for (a, b) in ((3, 1), (1, 3), (3, 3))
                       for sx in (-1, 1) for sy in (-1, 1)], key=lambda t: (t[1], t[0]))
FAR_PATTERN = sorted([(sx * a, sy * b) for (a, b) in ((5, 1), (1, 5), (5, 3), (3, 5), (5, 5))
                      for sx in (-1, 1) for sy in (-1, 1)], key=lambda t: (t[1], t[0]))
V_OFFSETS = [(dx, dy) for dy in range(-3, 4) for dx in range(-3, 4) if max(abs(dx), abs(dy)) >= 2]


def near_config(tree: Tree, t: int, s: int) -> int:
    """Index of the near-field configuration of source leaf s seen from target leaf t.

    0..8: same level, (dy+1)*3 + (dx+1). 9..20: source one level coarser, 21..32:
    one level finer; within a group, the position in NEAR_PATTERN of
    2D (coarser) or 4D (finer), D = (centre_s - centre_t) / h_t.
    """
    lt, ls = int(tree.level[t]), int(tree.level[s])
    dx4, dy4 = centre_offset(tree, t, s, lt)  # 4D
    if ls == lt:
        return (dy4 // 4 + 1) * 3 + (dx4 // 4 + 1)
    if ls == lt - 1:
        return 9 + NEAR_PATTERN.index((dx4 // 2, dy4 // 2))
    if ls == lt + 1:
        return 21 + NEAR_PATTERN.index((dx4, dy4))
    raise ValueError("leaves more than one level apart in a U list")


def centre_offset(tree: Tree, b: int, c: int, unit_level: int):
    """(centre_c - centre_b) in units of h_{unit_level} / 4, as exact integers."""
    def c4(x):
        l = int(tree.level[x])
        # centre in units of h_L/2 at L = max level, then rescale
        return (2 * int(tree.ix[x]) + 1) << (30 - l), (2 * int(tree.iy[x]) + 1) << (30 - l)
    bx, by = c4(b)
    cx, cy = c4(c)
    # one unit of h_L/2 at L=30 relative to h_unit/4: factor 2^(30-unit_level) / 2
    div = 1 << (30 - unit_level - 1)
    return (cx - bx) // div, (cy - by) // div


def build_lists(tree: Tree):
    """U, V, W, X lists by hashed neighbour lookup; CSR (ptr, idx, cfg), idx ascending.

    cfg is the configuration index of each entry: near_config for U, the position
    in V_OFFSETS for V, and the position in FAR_PATTERN of 4D (W, D in units of
    h_b) or 2D (X, D in units of h_b) with D = (centre_c - centre_b)/h_b.
    """
    n = tree.n_boxes
    idx = tree.index
    lv, ix, iy = tree.level, tree.ix, tree.iy
    U = [[] for _ in range(n)]
    V = [[] for _ in range(n)]
    W = [[] for _ in range(n)]
    X = [[] for _ in range(n)]
    for b in range(n):
        l, a, c = int(lv[b]), int(ix[b]), int(iy[b])
        side = 1 << l
        cols = []  # colleagues (same level, touching, not b)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == 0 and dy == 0:
                    continue
                q = idx.get((l, a + dx, c + dy)) if (0 <= a + dx < side and 0 <= c + dy < side) else None
                if q is not None:
                    cols.append(q)
        if tree.is_leaf[b]:
            U[b].append(b)
            for q in cols:
                if tree.is_leaf[q]:
                    U[b].append(q)
                else:
                    for ch in tree.child[q]:
                        if adjacent(l, a, c, int(lv[ch]), int(ix[ch]), int(iy[ch])):
                            U[b].append(int(ch))
                        else:
                            W[b].append(int(ch))
            if l >= 1:
                pa, pc = a >> 1, c >> 1
                ps = 1 << (l - 1)
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if dx == 0 and dy == 0:
                            continue
                        if not (0 <= pa + dx < ps and 0 <= pc + dy < ps):
                            continue
                        q = idx.get((l - 1, pa + dx, pc + dy))
                        if q is not None and tree.is_leaf[q] and adjacent(l, a, c, l - 1, pa + dx, pc + dy):
                            U[b].append(q)
        if l >= 2:
            pa, pc = a >> 1, c >> 1
            ps = 1 << (l - 1)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if not (0 <= pa + dx < ps and 0 <= pc + dy < ps):
                        continue
                    q = idx.get((l - 1, pa + dx, pc + dy))
                    if q is None:
                        continue
                    if tree.is_leaf[q]:
                        if (dx or dy) and not adjacent(l, a, c, l - 1, pa + dx, pc + dy):
                            X[b].append(q)
                        continue
                    for ch in tree.child[q]:
                        if not adjacent(l, a, c, int(lv[ch]), int(ix[ch]), int(iy[ch])) and ch != b:
                            V[b].append(int(ch))
    out = {}
    for name, L in (("U", U), ("V", V), ("W", W), ("X", X)):
        ptr = np.zeros(n + 1, dtype=np.int32)
        flat = []
        cfg = []
        for b in range(n):
            items = sorted(L[b])
            flat += items
            ptr[b + 1] = ptr[b] + len(items)
            for c in items:
                cfg.append(_cfg(tree, name, b, c))
        out[name] = (ptr, np.array(flat, dtype=np.int32), np.array(cfg, dtype=np.int32))
    return out


def _cfg(tree, name, b, c):
    if name == "U":
        return near_config(tree, b, c)
    lb = int(tree.level[b])
    dx4, dy4 = centre_offset(tree, b, c, lb)  # 4D, D in units of h_b
    if name == "V":
        return V_OFFSETS.index((dx4 // 4, dy4 // 4))
    if name == "W":
        return FAR_PATTERN.index((dx4, dy4))
    return FAR_PATTERN.index((dx4 // 2, dy4 // 2))  # X: 2D


def build_lists_bruteforce(tree: Tree):
    """The same lists from their definitions, by testing every pair of boxes."""
    n = tree.n_boxes
    lv, ix, iy = tree.level, tree.ix, tree.iy
    par = tree.parent
    res = {k: [[] for _ in range(n)] for k in "UVWX"}

    def adj(p, q):
        return adjacent(int(lv[p]), int(ix[p]), int(iy[p]), int(lv[q]), int(ix[q]), int(iy[q]))

    def colleague(p, q):
        return p != q and lv[p] == lv[q] and adj(p, q)

    for b in range(n):
        for c in range(n):
            if tree.is_leaf[b] and tree.is_leaf[c] and (b == c or adj(b, c)):
                res["U"][b].append(c)
            if b != c and lv[b] == lv[c] and lv[b] >= 2 and par[b] != par[c] and \
                    colleague(par[b], par[c]) and not adj(b, c):
                res["V"][b].append(c)
            if tree.is_leaf[b] and lv[c] == lv[b] + 1 and colleague(b, par[c]) and not adj(b, c):
                res["W"][b].append(c)
            if tree.is_leaf[c] and lv[c] == lv[b] - 1 and lv[b] >= 1 and colleague(par[b], c) and not adj(b, c):
                res["X"][b].append(c)
    out = {}
    for name in "UVWX":
        ptr = np.zeros(n + 1, dtype=np.int32)
        flat = []
        for b in range(n):
            flat += sorted(res[name][b])
            ptr[b + 1] = len(flat)
        out[name] = (ptr, np.array(flat, dtype=np.int32))
    return out


def is_balanced(tree: Tree) -> bool:
    lv, ix, iy = tree.level, tree.ix, tree.iy
    L = tree.leaves
    for p in range(len(L)):
        for q in range(p + 1, len(L)):
            a, b = L[p], L[q]
            if abs(int(lv[a]) - int(lv[b])) > 1 and adjacent(int(lv[a]), int(ix[a]), int(iy[a]),
                                                              int(lv[b]), int(ix[b]), int(iy[b])):
                return False
    return True
