"""Octree and dual-tree traversal, plain numpy/Python (oracle, test infra only).

Sec. 3.2 (Morton keys: interleaved coordinate bits, 63-bit keys, at most 21
levels) and Sec. 3.3 (Algorithm 1 Evaluate, Algorithm 2 Interact, the FMM MAC).

Readings taken where the paper is silent or ambiguous:
  * Keys: FP64 normalisation into the cube, 21 bits per axis: cell coordinate
    floor((x - x_min) f) with f = 2^21 / L rounded once (Sec. 3.2 fixes the
    interleaved bits of the normalised coordinates, not the rounding of the
    normalisation), clamped to [0, 2^21 - 1]; bit b of x, y, z at positions
    3b+2, 3b+1, 3b (x most significant).  Child digit = 4x+2y+z.
  * Free-space cube: centre of the bounding box, side = longest extent times
    (1 + 2^-10) (half-side 0.5 if all points coincide).  Periodic: given cube.
  * A cell splits while it holds more than ncrit particles and its level < 21.
    Children are the non-empty octants in digit order; cells are numbered level
    by level (breadth first), so every level is in Morton order.
  * Expansion centre = geometric cube centre; radius R = largest distance from
    the centre to one of the cell's particles (FP64).
  * MAC: M2L iff R_A + R_B < theta |X_A - X_B| and, because the far field uses
    the singular kernel, |X_A - X_B| - (R_A + R_B) >= k_sigma sigma_max.  The
    MAC is tested before the leaf test; two leaves that fail it do P2P; any
    other pair is pushed.  Option (the cost rule for cells of very few
    particles, Alg. 2): two leaves whose counts multiply to at most
    p2p_pair_max do P2P before the MAC is tested; p2p_pair_max >= ncrit^2
    gives Alg. 2's printed order (leaf test first).
  * Algorithm 1 splits A when its radius exceeds B's and B otherwise (the
    ELSE branch, so B on a tie).  "Radius" is read as the cube's size (the
    coarser level is the larger cell): comparing tight particle radii instead
    would let the rounding of the inputs decide between cells of equal
    cubes.  When the cell to split is a leaf, the other one is split (the
    pair was pushed because one of them has children).  Option
    split_tie="target" splits A instead on equal cubes (not the printed
    rule; kept to compare the two).
  * Periodic: the traversal starts from (root, root + o L) for the 27 shifts
    o in {-1,0,1}^3 (targets stay in the original cube).
All FP64 expressions are written in a fixed order with no fused operations so
the same decisions can be reproduced bit for bit elsewhere.
"""
import numpy as np

MAX_LEVEL = 21
KEY_SCALE = float(1 << MAX_LEVEL)


def free_space_box(pos):
    """(box_min[3], box_len) of the free-space cube (FP64)."""
    x = np.asarray(pos, np.float32).astype(np.float64)
    lo = x.min(0)
    hi = x.max(0)
    ext = float(np.max(hi - lo))
    half = (ext * 0.5) * (1.0 + 2.0 ** -10)
    if half == 0.0:
        half = 0.5
    center = (lo + hi) * 0.5
    return center - half, half * 2.0


def quantize(pos, box_min, box_len):
    """Integer cell coordinates at level 21, [n,3] int64."""
    x = np.asarray(pos, np.float32).astype(np.float64)
    f = KEY_SCALE / float(box_len)
    k = np.floor((x - np.asarray(box_min, np.float64)) * f)
    k = np.clip(k, 0.0, KEY_SCALE - 1.0)
    return k.astype(np.int64)


def interleave(k):
    """63-bit Morton keys from [n,3] integer coordinates (uint64)."""
    k = np.asarray(k, np.int64)
    key = np.zeros(k.shape[0], np.uint64)
    for b in range(MAX_LEVEL):
        for a, off in ((0, 2), (1, 1), (2, 0)):
            bit = ((k[:, a] >> b) & 1).astype(np.uint64)
            key |= bit << np.uint64(3 * b + off)
    return key


def deinterleave(key):
    """Inverse of interleave for [n] uint64 keys -> [n,3] int64."""
    key = np.asarray(key, np.uint64)
    k = np.zeros((key.shape[0], 3), np.int64)
    for b in range(MAX_LEVEL):
        for a, off in ((0, 2), (1, 1), (2, 0)):
            k[:, a] |= ((key >> np.uint64(3 * b + off)) & np.uint64(1)).astype(np.int64) << b
    return k


class Tree:
    """Cells numbered breadth first.  Arrays indexed by cell id."""

    def __init__(self):
        self.begin = self.end = self.level = self.parent = None
        self.child_begin = self.nchild = self.ijk = self.center = self.radius = None


def build(pos, ncrit, box_min=None, box_len=None):
    """Sort particles by Morton key and build the octree.

    Returns (order, keys_sorted, tree, box_min, box_len) where order is the
    stable permutation (sorted position -> input index).
    """
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    if box_min is None:
        box_min, box_len = free_space_box(pos) if n else (np.zeros(3), 1.0)
    box_min = np.asarray(box_min, np.float64)
    box_len = float(box_len)
    keys = interleave(quantize(pos, box_min, box_len))
    order = np.argsort(keys, kind="stable")
    skeys = keys[order]
    t = Tree()
    if n == 0:
        for f in ("begin", "end", "level", "parent", "child_begin", "nchild"):
            setattr(t, f, np.zeros(0, np.int64))
        t.ijk = np.zeros((0, 3), np.int64)
        t.center = np.zeros((0, 3))
        t.radius = np.zeros(0)
        return order, skeys, t, box_min, box_len
    begin, end, level, parent = [0], [n], [0], [-1]
    child_begin, nchild = [], []
    cur = [0]
    while cur:
        nxt = []
        for c in cur:
            lv = level[c]
            b, e = begin[c], end[c]
            if e - b > ncrit and lv < MAX_LEVEL:
                shift = np.uint64(3 * (MAX_LEVEL - 1 - lv))
                digits = ((skeys[b:e] >> shift) & np.uint64(7)).astype(np.int64)
                bounds = np.searchsorted(digits, np.arange(9), side="left") + b
                child_begin.append(len(begin))
                cnt = 0
                for d in range(8):
                    if bounds[d + 1] > bounds[d]:
                        begin.append(int(bounds[d]))
                        end.append(int(bounds[d + 1]))
                        level.append(lv + 1)
                        parent.append(c)
                        nxt.append(len(begin) - 1)
                        cnt += 1
                nchild.append(cnt)
            else:
                child_begin.append(-1)
                nchild.append(0)
        cur = nxt
    # child_begin/nchild were appended in cell-id order (BFS visits ids in order)
    t.begin = np.array(begin, np.int64)
    t.end = np.array(end, np.int64)
    t.level = np.array(level, np.int64)
    t.parent = np.array(parent, np.int64)
    t.child_begin = np.array(child_begin, np.int64)
    t.nchild = np.array(nchild, np.int64)
    kfirst = skeys[t.begin]
    shifts = (3 * (MAX_LEVEL - t.level)).astype(np.uint64)
    t.ijk = deinterleave(kfirst >> shifts)
    side = box_len * np.exp2(-t.level.astype(np.float64))
    t.center = box_min[None, :] + (t.ijk.astype(np.float64) + 0.5) * side[:, None]
    xs = pos[order].astype(np.float64)
    R = np.zeros(len(begin))
    for c in range(len(begin)):
        d = xs[t.begin[c]:t.end[c]] - t.center[c]
        R[c] = np.max(np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]))
    t.radius = R
    return order, skeys, t, box_min, box_len


def image_offsets(periodic):
    """Image shift multipliers: (0,0,0) only, or the 27 of {-1,0,1}^3 (o-major)."""
    if not periodic:
        return np.zeros((1, 3), np.int64)
    r = np.arange(-1, 2)
    ox, oy, oz = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([ox.ravel(), oy.ravel(), oz.ravel()], 1).astype(np.int64)


def traverse(tree, box_len, theta, ksig, sigma_max, periodic=False, p2p_pair_max=0, split_tie="source"):
    """Algorithms 1-2.  Returns (p2p, m2l) as int64 arrays of (A, B, image).

    split_tie: which cell Algorithm 1 splits when A and B are cubes of one
    size: "source" (B, the printed ELSE branch; default) or "target" (A).
    """
    if split_tie not in ("source", "target"):
        raise ValueError("split_tie must be 'source' or 'target'")
    tie_a = split_tie == "target"
    offs = image_offsets(periodic)
    shifts = offs.astype(np.float64) * float(box_len)
    theta = float(theta)
    ksig = float(ksig)
    sigma_max = float(sigma_max)
    C = tree.center
    R = tree.radius
    lev = tree.level
    leaf = tree.nchild == 0
    p2p, m2l, stack = [], [], []
    if len(tree.begin) == 0:
        return np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64)

    count = tree.end - tree.begin

    def interact(a, b, o):
        if p2p_pair_max > 0 and leaf[a] and leaf[b] and int(count[a]) * int(count[b]) <= p2p_pair_max:
            p2p.append((a, b, o))
            return
        cb = C[b] + shifts[o]
        dx = C[a] - cb
        dist = np.sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2])
        sr = R[a] + R[b]
        if sr < theta * dist and (dist - sr) >= ksig * sigma_max:
            m2l.append((a, b, o))
        elif leaf[a] and leaf[b]:
            p2p.append((a, b, o))
        else:
            stack.append((a, b, o))

    for o in range(offs.shape[0]):
        interact(0, 0, o)
    while stack:
        a, b, o = stack.pop()
        # A larger than B  <=>  A is on the coarser level (the cube size)
        split_a = lev[a] < lev[b] or (tie_a and lev[a] == lev[b])
        if split_a and leaf[a]:
            split_a = False
        elif (not split_a) and leaf[b]:
            split_a = True
        if split_a:
            for c in range(tree.child_begin[a], tree.child_begin[a] + tree.nchild[a]):
                interact(c, b, o)
        else:
            for c in range(tree.child_begin[b], tree.child_begin[b] + tree.nchild[b]):
                interact(a, c, o)
    return np.array(p2p, np.int64).reshape(-1, 3), np.array(m2l, np.int64).reshape(-1, 3)
