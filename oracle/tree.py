"""Adaptive quadtree, active DOF sets, near fields and proxy points.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

Sec. 2.1 and Remark (tree): the domain is split recursively into four
sub-squares until every leaf holds at most n_occ points (n_occ = 64, Sec. 5);
in practice the tree is adaptive (empty children are dropped).  Readings where
the paper is silent:

* root = the smallest axis-aligned square containing all points, centred on
  their bounding box;
* point coordinates are quantised to D-bit integers relative to the root
  square, q = floor((x - lo) * (2^D / side)) clamped to [0, 2^D - 1]; a box
  at level l holds the points whose top l bits agree, so a point on a split
  line goes to the upper quadrant;
* child slots are in Morton order SW, SE, NW, NE (slot = 2*ybit + xbit);
* tree order = points sorted by their Morton key, ties by original index;
* a box splits when it holds more than n_occ points and its level is below D.

Sec. 2.3.1 (modified proxy trick): the near field N of box B is the set of
active DOFs outside B within r_near * w of B's centre (w = side of B), and the
proxy set Gamma is n_prox points in the annulus [r_in * w, r_out * w]:
n_rings rings equispaced in radius, n_prox / n_rings equispaced angles each,
odd rings rotated by half an angular step.
"""
from __future__ import annotations

import numpy as np

DEPTH_BITS = 24

DEFAULT_OPTS = dict(n_occ=64, n_prox=256, r_near=1.0, r_in=1.0, r_out=2.0,
                    n_rings=8)


def morton_keys(q):
    """Interleave the bits of qy (high) and qx (low) of each point."""
    qx = q[:, 0].astype(np.uint64)
    qy = q[:, 1].astype(np.uint64)
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for b in range(DEPTH_BITS - 1, -1, -1):
        key = (key << np.uint64(2)) | (((qy >> np.uint64(b)) & np.uint64(1)) << np.uint64(1)) \
            | ((qx >> np.uint64(b)) & np.uint64(1))
    return key


class Tree:
    """Flattened quadtree.  Box arrays are indexed by box id; boxes of one
    level are contiguous and levels are stored root first."""

    def __init__(self, x, n_occ=64):
        x = np.asarray(x, dtype=np.float64)
        n = x.shape[0]
        self.n = n
        self.n_occ = n_occ
        xmin, ymin = x.min(axis=0)
        xmax, ymax = x.max(axis=0)
        side = max(xmax - xmin, ymax - ymin)
        if side <= 0.0:
            side = 1.0
        cx = (xmin + xmax) * 0.5
        cy = (ymin + ymax) * 0.5
        self.side = side
        self.lo = np.array([cx - side * 0.5, cy - side * 0.5])
        scale = float(2 ** DEPTH_BITS) / side
        qf = np.floor((x - self.lo[None, :]) * scale)
        qf = np.clip(qf, 0.0, float(2 ** DEPTH_BITS - 1))
        q = qf.astype(np.uint64)
        key = morton_keys(q)
        perm = np.lexsort((np.arange(n), key))  # key primary, index secondary
        self.perm = perm                      # tree position -> original index
        self.iperm = np.empty(n, dtype=np.int64)
        self.iperm[perm] = np.arange(n)
        self.key = key[perm]
        self.q = q[perm]
        self.xt = x[perm]                      # coordinates in tree order

        # Breadth-first construction.
        level = [0]; start = [0]; count = [n]; parent = [-1]; slot = [0]
        ix = [0]; iy = [0]
        children = [[-1, -1, -1, -1]]
        frontier = [0]
        lev = 0
        while frontier:
            nxt = []
            for b in frontier:
                if count[b] <= n_occ or lev >= DEPTH_BITS:
                    continue
                s0, c0 = start[b], count[b]
                shift = np.uint64(2 * (DEPTH_BITS - lev - 1))
                sub = (self.key[s0:s0 + c0] >> shift) & np.uint64(3)
                bounds = np.searchsorted(sub, np.arange(5, dtype=np.uint64))
                for sl in range(4):
                    a, e = int(bounds[sl]), int(bounds[sl + 1])
                    if e > a:
                        cid = len(level)
                        level.append(lev + 1); start.append(s0 + a); count.append(e - a)
                        parent.append(b); slot.append(sl)
                        ix.append(2 * ix[b] + (sl & 1)); iy.append(2 * iy[b] + (sl >> 1))
                        children.append([-1, -1, -1, -1])
                        children[b][sl] = cid
                        nxt.append(cid)
            frontier = nxt
            lev += 1
        self.level = np.array(level, dtype=np.int64)
        self.start = np.array(start, dtype=np.int64)
        self.count = np.array(count, dtype=np.int64)
        self.parent = np.array(parent, dtype=np.int64)
        self.slot = np.array(slot, dtype=np.int64)
        self.ix = np.array(ix, dtype=np.int64)
        self.iy = np.array(iy, dtype=np.int64)
        self.children = np.array(children, dtype=np.int64)
        self.is_leaf = np.all(self.children < 0, axis=1)
        self.nlevels = int(self.level.max()) + 1     # levels 0..L
        self.L = self.nlevels - 1
        w = side / (2.0 ** self.level)
        self.width = w
        self.centre = np.stack([self.lo[0] + (self.ix + 0.5) * w,
                                self.lo[1] + (self.iy + 0.5) * w], axis=1)

    def boxes_at(self, lev):
        return np.nonzero(self.level == lev)[0]

    def dofs(self, b):
        """All DOFs (tree positions) inside box b."""
        return np.arange(self.start[b], self.start[b] + self.count[b])

    def leaf_pos(self):
        """For each tree position, its index within its leaf box."""
        pos = np.empty(self.n, dtype=np.int64)
        for b in np.nonzero(self.is_leaf)[0]:
            pos[self.start[b]:self.start[b] + self.count[b]] = np.arange(self.count[b])
        return pos


def proxy_points(centre, w, n_prox=256, r_in=1.5, r_out=3.0, n_rings=8):
    """n_prox points in the annulus [r_in w, r_out w] around ``centre``."""
    n_ang = n_prox // n_rings
    out = []
    for i in range(n_rings):
        rad = (r_in + (r_out - r_in) * (i + 0.5) / n_rings) * w
        off = 0.5 if (i % 2) else 0.0
        ang = 2.0 * np.pi * (np.arange(n_ang) + off) / n_ang
        out.append(np.stack([centre[0] + rad * np.cos(ang),
                             centre[1] + rad * np.sin(ang)], axis=1))
    return np.vstack(out)
