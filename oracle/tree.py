"""Oracle grid hierarchy, near/far interaction lists and the static work map.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 5.1 (Definition): two grid blocks are near iff they share at least one
node, i.e. their integer box coordinates differ by at most one in each
direction.  Sec. 5.3 (eq. eq_rec01): each level splits every block in two
along each direction; a pair of blocks is compressed at the first level where
it is far (its parents were near).  Sec. 5.4: an atom is assigned whole to
the block holding its barycentre; the finest level holds at most one atom
per block, and every pair of distinct atoms not yet compressed is compressed
there, so the only near blocks left are the self blocks (Z_N = Z_D).

Reading (the paper's first grid is 3 x 3, Fig. fig_grid1): a power-of-two
quadtree.  With s the smallest centre separation in the infinity norm, the
root square has lower corner (min x - s/2, min y - s/2) and side s 2^L, with
2^L >= (largest extent)/s + 1; the finest level L has boxes of side s.
"""
import numpy as np


def atom_box_coords(centres):
    """(L, finest integer box coordinates (N, 2)) of the quadtree."""
    c = np.asarray(centres, float)[:, :2]
    N = len(c)
    if N == 1:
        return 0, np.zeros((1, 2), int)
    d = np.max(np.abs(c[:, None, :] - c[None, :, :]), axis=-1)
    d[np.arange(N), np.arange(N)] = np.inf
    s = d.min()
    lo = c.min(0) - 0.5 * s
    ext = (c.max(0) - c.min(0)).max()
    L = 0
    while 2 ** L < ext / s + 1.0 - 1e-9:
        L += 1
    idx = np.floor((c - lo) / s).astype(int)
    idx = np.clip(idx, 0, 2 ** L - 1)
    return L, idx


def build_tree(centres):
    """Far block pairs per level.

    Returns (L, blocks) where blocks is a list of (level, rows_atoms, cols_atoms),
    ordered by level, then target box (y, x), then source box (y, x); atoms
    inside a box are in ascending index order.
    """
    L, fine = atom_box_coords(centres)
    N = len(fine)
    blocks = []
    for lev in range(1, L + 1):
        shift = L - lev
        bc = fine >> shift                   # box coordinates at this level
        pc = fine >> (shift + 1)             # parent box coordinates
        boxes = {}
        for a in range(N):
            boxes.setdefault((int(bc[a, 1]), int(bc[a, 0])), []).append(a)
        keys = sorted(boxes)
        for tb in keys:
            for sb in keys:
                ta, sa = boxes[tb], boxes[sb]
                t_par = pc[ta[0]]
                s_par = pc[sa[0]]
                parents_near = np.max(np.abs(t_par - s_par)) <= 1
                if not parents_near:
                    continue
                dist = max(abs(tb[0] - sb[0]), abs(tb[1] - sb[1]))
                if lev == L:
                    far = tb != sb          # finest level: every distinct pair
                else:
                    far = dist > 1
                if far:
                    blocks.append((lev, list(ta), list(sa)))
    return L, blocks


def lpt_assign(weights, n_proc):
    """Greedy least-loaded assignment (App. C): sort descending, give each
    interaction to the currently least-loaded process (lowest index on ties).

    Returns (owner (len(weights),) in the original order, loads (n_proc,), order)."""
    w = np.asarray(weights, float)
    order = np.argsort(-w, kind="stable")
    loads = np.zeros(n_proc)
    owner = np.zeros(len(w), int)
    for i in order:
        k = int(np.argmin(loads))
        loads[k] += w[i]
        owner[i] = k
    return owner, loads, order
