"""Seeded synthetic workloads for STA-FEM assembly (superset meshes, masks, edit streams).

This module only generates inputs.  It holds none of the assembly arithmetic: no element
matrices, no sparsity pattern, no sums.  Both the CUDA path and the oracle read what it
returns, and nothing here imports either of them.

The paper evaluates on tetrahedral models that are not available here (Sec. 5.1: Bunny,
Gargoyle, Hand from Cutler et al. 2004), so these seeded generators stand in for them with
meshes and edit streams of the same shape: fracture, refinement and merge scenarios over a
preallocated superset (Sec. 5.1, Sec. 3.3), 10k-460k active tetrahedra (abstract, Table 2),
tens to thousands of edited tetrahedra per frame (Sec. 2.3).

Every random draw uses ``numpy.random.Generator(PCG64(seed))``.  Edits are int32 arrays of
shape (m, 3) with rows (op, tet, tet2): op 0 deactivates ``tet``, op 1 activates ``tet``,
op 2 swaps (deactivates ``tet``, activates ``tet2``); ``tet2`` is -1 unless op is 2.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

DEACTIVATE, ACTIVATE, SWAP = 0, 1, 2


@dataclass
class Workload:
    """One superset mesh with its initial active mask and per-frame edit lists."""
    name: str
    X: np.ndarray            # (n, 3) float64 node positions
    tets: np.ndarray         # (T, 4) int32 node ids, positively oriented
    E: np.ndarray            # (T,) float64 Young's modulus
    nu: np.ndarray           # (T,) float64 Poisson ratio
    mask0: np.ndarray        # (T,) uint8 initial active mask
    frames: list = field(default_factory=list)   # list of (m, 3) int32 edit arrays
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def masks(self):
        """Active mask after each frame (list of F+1 arrays, the first is mask0)."""
        out = [self.mask0.copy()]
        m = self.mask0.copy()
        for ed in self.frames:
            m = apply_edits_to_mask(m, ed)
            out.append(m.copy())
        return out


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    """Generator seeded as 1000 * config + instance."""
    return np.random.Generator(np.random.PCG64(1000 * config + instance))


def apply_edits_to_mask(mask: np.ndarray, edits: np.ndarray) -> np.ndarray:
    m = mask.copy()
    for op, t, t2 in np.asarray(edits).reshape(-1, 3):
        if op == DEACTIVATE:
            m[t] = 0
        elif op == ACTIVATE:
            m[t] = 1
        else:
            m[t] = 0
            m[t2] = 1
    return m


def make_edits(off=(), on=(), swaps=()) -> np.ndarray:
    rows = [(DEACTIVATE, int(t), -1) for t in off]
    rows += [(ACTIVATE, int(t), -1) for t in on]
    rows += [(SWAP, int(a), int(b)) for a, b in swaps]
    if not rows:
        return np.zeros((0, 3), np.int32)
    return np.asarray(rows, dtype=np.int32)


# ----------------------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------------------

def _orient_positive(X: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap the last two vertices of negatively oriented tetrahedra (sign via numpy det)."""
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    s = np.linalg.det(d)
    flip = s < 0
    tets = tets.copy()
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return tets


def _check_positive(X: np.ndarray, tets: np.ndarray) -> None:
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    s = np.linalg.det(d)
    if not np.all(s > 0):
        raise ValueError(f"{int(np.sum(s <= 0))} tetrahedra are not positively oriented")


def kuhn_cube(N: int, jitter: float = 0.0, rng: np.random.Generator | None = None,
              nx: int | None = None, ny: int | None = None):
    """Unit cube split into an nx x ny x N grid of hexes (nx = ny = N by default), each cut
    into the 6 Kuhn (Freudenthal) tetrahedra along its (0,0,0)-(1,1,1) diagonal, one per
    permutation of the axes.  The split is conforming.  Nodes are jittered uniformly by
    +-jitter*h per coordinate.  Tetrahedron id = 6 * hex + permutation index, hex = x + nx
    (y + ny z).  Returns (X, tets, grid_index) with grid_index the (n, 3) integer lattice
    coordinates of each node."""
    nx = N if nx is None else nx
    ny = N if ny is None else ny
    nz = N
    h = 1.0 / max(nx, ny, nz)
    gi = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1),
                              indexing="ij"), -1)
    gi = gi.transpose(2, 1, 0, 3).reshape(-1, 3)          # x fastest
    X = gi.astype(np.float64) * h
    if jitter > 0:
        X = X + rng.uniform(-jitter * h, jitter * h, size=X.shape)

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    hx, hy, hz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hx, hy, hz = (a.transpose(2, 1, 0).reshape(-1) for a in (hx, hy, hz))
    tets = []
    for perm in itertools.permutations(range(3)):
        steps = [np.zeros(3, int)]
        for ax in perm:
            s = steps[-1].copy()
            s[ax] += 1
            steps.append(s)
        vs = [nid(hx + s[0], hy + s[1], hz + s[2]) for s in steps]
        tets.append(np.stack(vs, -1))
    tets = np.stack(tets, 1).reshape(-1, 4).astype(np.int32)
    tets = _orient_positive(gi.astype(np.float64), tets)
    _check_positive(X, tets)
    return X, tets, gi


def lognormal_E(rng: np.random.Generator, T: int, median: float = 1e5, sigma: float = 0.3):
    return median * np.exp(sigma * rng.standard_normal(T))


# ----------------------------------------------------------------------------------------
# Edit streams
# ----------------------------------------------------------------------------------------

def deact_react_stream(rng, T: int, mask0: np.ndarray, frames: int, rate_off: float,
                       rate_on: float):
    """Each frame deactivates round(rate_off * |active|) tetrahedra drawn from those active at
    frame start and reactivates min(|inactive|, round(rate_on * T)) drawn from those inactive
    at frame start (fracture and merge of Sec. 5.1, randomised)."""
    m = mask0.copy()
    out = []
    for _ in range(frames):
        act = np.flatnonzero(m)
        ina = np.flatnonzero(m == 0)
        k_off = int(round(rate_off * act.size))
        k_on = min(ina.size, int(round(rate_on * T)))
        off = rng.choice(act, size=k_off, replace=False) if k_off else np.zeros(0, int)
        on = rng.choice(ina, size=k_on, replace=False) if k_on else np.zeros(0, int)
        ed = make_edits(off=off, on=on)
        out.append(ed)
        m = apply_edits_to_mask(m, ed)
    return out


def random_edit_stream(rng, mask0: np.ndarray, frames: int, most: int = 6):
    """Test input, not a paper workload: each frame draws up to `most` deactivations, `most`
    activations and `most` swaps (an active tet for an inactive one) over disjoint tetrahedra
    from the mask at frame start, rows shuffled; one frame in eight (on average) is empty."""
    m = mask0.copy()
    out = []
    for _ in range(frames):
        if rng.random() < 0.125:
            out.append(make_edits())
            continue
        act = rng.permutation(np.flatnonzero(m))
        ina = rng.permutation(np.flatnonzero(m == 0))
        k_off = int(rng.integers(0, min(act.size, most) + 1))
        k_on = int(rng.integers(0, min(ina.size, most) + 1))
        k_sw = int(rng.integers(0, min(act.size - k_off, ina.size - k_on, most) + 1))
        ed = make_edits(off=act[:k_off], on=ina[:k_on],
                        swaps=zip(act[k_off:k_off + k_sw], ina[k_on:k_on + k_sw]))
        ed = ed[rng.permutation(ed.shape[0])] if ed.shape[0] else ed
        out.append(ed)
        m = apply_edits_to_mask(m, ed)
    return out


def randomized(wl: Workload, seed: int, frames: int = 16, most: int = 6) -> Workload:
    """The superset of `wl` with a random initial mask (active fraction drawn in [0.2, 0.9])
    and a random_edit_stream: the randomized parity tests' input."""
    rng = rng_for(90, seed)
    mask0 = (rng.random(wl.n_tets) < rng.uniform(0.2, 0.9)).astype(np.uint8)
    return Workload(f"{wl.name}_random{seed}", wl.X, wl.tets, wl.E, wl.nu, mask0,
                    random_edit_stream(rng, mask0, frames, most), dict(wl.meta))


# ----------------------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------------------

def plain_small(seed: int = 0, N: int = 6, frames: int = 24) -> Workload:
    """Unit cube, 6x6x6 hexes x 6 = 1296 tets, 343 nodes, jitter +-0.15h, E = 1e5, nu = 0.3.
    Superset = all tets, all active at start.  Each frame deactivates 2% of the active tets
    and reactivates 0.5% of T."""
    rng = rng_for(1, seed)
    X, tets, gi = kuhn_cube(N, 0.15, rng)
    T = tets.shape[0]
    mask0 = np.ones(T, np.uint8)
    fr = deact_react_stream(rng, T, mask0, frames, 0.02, 0.005)
    return Workload(f"plain_small_N{N}", X, tets, np.full(T, 1e5), np.full(T, 0.3), mask0, fr,
                    {"N": N, "grid_index": gi})


def edge_fan(seed: int = 0, K: int = 300, frames: int = 12) -> Workload:
    """K tetrahedra around one edge: axis nodes 0 = (0,0,0) and 1 = (0,0,1), a ring of K
    jittered nodes at height 0.5, tets (0, 1, r_k, r_k+1).  The axis pair and both axis nodes
    are shared by all K tets -- the longest contributor lists a fold meets (edge cases of the
    fold's shared-memory staging).  70% active at start; each frame deactivates 10% of the
    active tets and reactivates 10% of T."""
    rng = rng_for(6, seed)
    th = 2 * np.pi * (np.arange(K) + rng.uniform(-0.2, 0.2, K)) / K
    ring = np.stack([np.cos(th), np.sin(th), 0.5 + rng.uniform(-0.1, 0.1, K)], axis=1)
    X = np.concatenate([[[0.0, 0.0, 0.0], [0.0, 0.0, 1.0]], ring])
    k = np.arange(K)
    tets = np.stack([np.zeros(K, int), np.ones(K, int), 2 + k, 2 + (k + 1) % K], axis=1)
    tets = _orient_positive(X, tets.astype(np.int32))
    _check_positive(X, tets)
    mask0 = (rng.uniform(size=K) < 0.7).astype(np.uint8)
    fr = deact_react_stream(rng, K, mask0, frames, 0.1, 0.1)
    return Workload(f"edge_fan_K{K}", X, tets, lognormal_E(rng, K), np.full(K, 0.3), mask0, fr,
                    {"K": K})


def prefractured_block(seed: int = 0, N: int = 40, sites: int = 64, frames: int = 24,
                       interfaces_per_frame: int = 3) -> Workload:
    """Pre-fractured block: N^3 hexes x 6 on [0,1]^3, jitter +-0.2h, E lognormal (median 1e5,
    sigma 0.3), nu = 0.3.  Seeded Voronoi sites partition the tets by centroid (nearest site,
    ties to the lower site id).  A node is on a cell boundary when its tets span two or more
    cells.  Every tet with a boundary node gets a preallocated split copy in which each
    boundary node is replaced by a duplicate node private to (node, cell of the tet).  The
    originals start active, the copies inactive.  Each frame picks `interfaces_per_frame`
    unused cell-cell interfaces and swaps every not-yet-swapped tet of either cell that has a
    node shared by both cells from its connected original to its split copy."""
    rng = rng_for(2, seed)
    X, tets, gi = kuhn_cube(N, 0.2, rng)
    T0 = tets.shape[0]
    n0 = X.shape[0]
    E = lognormal_E(rng, T0)
    S = rng.uniform(0.0, 1.0, size=(sites, 3))
    cen = X[tets].mean(axis=1)
    # nearest site per tet, chunked; argmin picks the lowest index among ties
    cell = np.empty(T0, np.int64)
    for s in range(0, T0, 65536):
        d2 = ((cen[s:s + 65536, None, :] - S[None, :, :]) ** 2).sum(-1)
        cell[s:s + 65536] = np.argmin(d2, axis=1)
    # cells incident to each node as a (node, cell) unique list
    nc = np.unique(np.stack([tets.reshape(-1).astype(np.int64),
                             np.repeat(cell, 4)], 1), axis=0)
    ncount = np.bincount(nc[:, 0], minlength=n0)
    boundary = ncount >= 2
    # duplicate node per (boundary node, cell) pair, ordered by (node, cell)
    bnc = nc[boundary[nc[:, 0]]]
    dup_id = {(int(v), int(c)): n0 + i for i, (v, c) in enumerate(bnc)}
    has_b = boundary[tets].any(axis=1)
    orig_ids = np.flatnonzero(has_b)
    copies = tets[orig_ids].copy()
    for r, t in enumerate(orig_ids):
        c = int(cell[t])
        for a in range(4):
            v = int(copies[r, a])
            if boundary[v]:
                copies[r, a] = dup_id[(v, c)]
    Xall = np.concatenate([X, X[bnc[:, 0]]], 0)
    tets_all = np.concatenate([tets, copies], 0).astype(np.int32)
    T = tets_all.shape[0]
    copy_of = np.full(T0, -1, np.int64)
    copy_of[orig_ids] = T0 + np.arange(orig_ids.size)
    E_all = np.concatenate([E, E[orig_ids]])
    mask0 = np.zeros(T, np.uint8)
    mask0[:T0] = 1
    # interfaces: cell pairs sharing a boundary node
    node_cells = {}
    for v, c in bnc:
        node_cells.setdefault(int(v), []).append(int(c))
    iface_nodes = {}
    for v, cs in node_cells.items():
        for a, b in itertools.combinations(sorted(cs), 2):
            iface_nodes.setdefault((a, b), []).append(v)
    iface_keys = sorted(iface_nodes)
    order = rng.permutation(len(iface_keys))
    # node -> tets incidence for interface membership
    inc_ptr = np.zeros(n0 + 1, np.int64)
    np.add.at(inc_ptr, tets.reshape(-1) + 1, 1)
    inc_ptr = np.cumsum(inc_ptr)
    inc = np.argsort(tets.reshape(-1), kind="stable") // 4
    swapped = np.zeros(T0, bool)
    fr = []
    pos = 0
    for _ in range(frames):
        chosen = []
        while len(chosen) < interfaces_per_frame and pos < len(order):
            chosen.append(iface_keys[order[pos]])
            pos += 1
        sel = set()
        for (a, b) in chosen:
            for v in iface_nodes[(a, b)]:
                for t in inc[inc_ptr[v]:inc_ptr[v + 1]]:
                    if cell[t] in (a, b) and not swapped[t]:
                        sel.add(int(t))
        sel = np.array(sorted(sel), np.int64)
        rng.shuffle(sel)
        swapped[sel] = True
        fr.append(make_edits(swaps=[(t, copy_of[t]) for t in sel]))
    return Workload(f"prefractured_block_N{N}", Xall, tets_all, E_all, np.full(T, 0.3), mask0,
                    fr, {"N": N, "sites": sites, "n_base_tets": T0, "n_copies": orig_ids.size,
                         "cell": cell})


def _red_children(tets: np.ndarray, mid) -> np.ndarray:
    """Eight red-refinement children per tet (v0..v3) given mid(a, b) -> midpoint node ids
    (vectorised): four corner tets and four octahedron tets split along the m02-m13
    diagonal.  Returns (T, 8, 4)."""
    v0, v1, v2, v3 = (tets[:, k].astype(np.int64) for k in range(4))
    m01, m02, m03 = mid(v0, v1), mid(v0, v2), mid(v0, v3)
    m12, m13, m23 = mid(v1, v2), mid(v1, v3), mid(v2, v3)
    kids = [(v0, m01, m02, m03), (m01, v1, m12, m13), (m02, m12, v2, m23), (m03, m13, m23, v3),
            (m01, m02, m03, m13), (m01, m02, m12, m13), (m02, m03, m13, m23),
            (m02, m12, m13, m23)]
    return np.stack([np.stack(k, -1) for k in kids], 1)


def slab_cycles(seed: int = 0, N: int = 12, half_width: float = 0.04, frames: int = 8) -> Workload:
    """Spatiotemporal edit locality (Sec. 6.4 locality sweep, Sec. 6.5 repeated edits): the
    unit cube, N^3 hexes x 6 (N = 12: 10,368 tets, the size of the paper's smallest model),
    jitter +-0.15h, E lognormal (median 1e5, sigma 0.3), nu = 0.3, all active at start.  The
    slab: the tets whose centroid lies within half_width of a plane through a seeded point of
    [0.35, 0.65]^3 with a seeded unit normal (the paper's "adaptively chosen" slab placement
    is not specified).  Even frames delete the slab's tets, odd frames reinsert them, so the
    same region is edited frame after frame and the mask returns to mask0 every 2 frames."""
    rng = rng_for(7, seed)
    X, tets, gi = kuhn_cube(N, 0.15, rng)
    T = tets.shape[0]
    p0 = rng.uniform(0.35, 0.65, 3)
    nrm = rng.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    cen = X[tets].mean(axis=1)
    slab = np.flatnonzero(np.abs((cen - p0) @ nrm) <= half_width)
    mask0 = np.ones(T, np.uint8)
    fr = [make_edits(off=slab) if f % 2 == 0 else make_edits(on=slab) for f in range(frames)]
    return Workload(f"slab_cycles_N{N}_hw{half_width}", X, tets, lognormal_E(rng, T),
                    np.full(T, 0.3), mask0, fr,
                    {"N": N, "half_width": half_width, "slab_tets": int(slab.size),
                     "grid_index": gi})


def slab_sequence(seed: int = 0, N: int = 20, half_width: float = 0.01, frames: int = 8,
                  merge: bool = False) -> Workload:
    """Fracture and merge scenarios of the paper's multi-model comparison (Sec. 5.1, Table 2):
    the unit cube, N^3 hexes x 6 (N = 20: 48,000 tets; 26: 105,456; 43: 477,042), jitter
    +-0.15h, E lognormal, nu = 0.3.  A seeded unit normal and `frames` parallel slabs of
    half-width `half_width` (centroid distance to the plane), spaced 4 half-widths apart around
    the cube's centre.  Fracture: all tets active at start, frame f deletes slab f.  Merge:
    every slab deleted at start, frame f reinserts slab f."""
    rng = rng_for(8, seed)
    X, tets, gi = kuhn_cube(N, 0.15, rng)
    T = tets.shape[0]
    nrm = rng.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    d = (X[tets].mean(axis=1) - 0.5) @ nrm
    offs = (np.arange(frames) - (frames - 1) / 2.0) * 4.0 * half_width
    slabs = [np.flatnonzero(np.abs(d - o) <= half_width) for o in offs]
    mask0 = np.ones(T, np.uint8)
    if merge:
        for sl in slabs:
            mask0[sl] = 0
    fr = [make_edits(on=sl) if merge else make_edits(off=sl) for sl in slabs]
    return Workload(f"slab_{'merge' if merge else 'fracture'}_N{N}", X, tets, lognormal_E(rng, T),
                    np.full(T, 0.3), mask0, fr,
                    {"N": N, "half_width": half_width, "slab_tets": [int(x.size) for x in slabs],
                     "grid_index": gi})


def refinement_hierarchy(seed: int = 0, N: int = 30, radius: float = 0.15, frames: int = 24
                         ) -> Workload:
    """Refinement hierarchy: N^3 hexes x 6 coarse tets (no jitter), each with its 8
    preallocated red-refinement children (ids T0 + 8p + k), midpoint nodes shared between
    neighbours.  A sphere of the given radius moves along a piecewise-linear path through 4
    seeded waypoints in [0.15, 0.85]^3, sampled uniformly by arc length at frames + 1 points.
    A coarse tet whose centroid lies inside the sphere is replaced by its children; one that
    leaves is coarsened back.  The mask of point 0 is the initial mask; each of the `frames`
    frames moves to the next point (refinement: 1 deactivation + 8 activations)."""
    rng = rng_for(3, seed)
    X, tets, gi = kuhn_cube(N, 0.0)
    T0 = tets.shape[0]
    n0 = X.shape[0]
    e = np.concatenate([tets[:, [a, b]] for a, b in itertools.combinations(range(4), 2)], 0)
    e = np.sort(e, axis=1).astype(np.int64)
    keys = np.unique(e[:, 0] * n0 + e[:, 1])
    Xm = 0.5 * (X[keys // n0] + X[keys % n0])
    Xall = np.concatenate([X, Xm], 0)

    def mid(a, b):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        return n0 + np.searchsorted(keys, lo * n0 + hi)

    ch = _red_children(tets, mid).reshape(-1, 4).astype(np.int32)
    ch = _orient_positive(Xall, ch)
    tets_all = np.concatenate([tets, ch], 0).astype(np.int32)
    _check_positive(Xall, tets_all)
    T = tets_all.shape[0]
    W = rng.uniform(0.15, 0.85, size=(4, 3))
    seg = np.linalg.norm(np.diff(W, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    centers = []
    for s in np.linspace(0.0, cum[-1], frames + 1):
        k = min(int(np.searchsorted(cum, s, side="right")) - 1, 2)
        u = (s - cum[k]) / seg[k] if seg[k] > 0 else 0.0
        centers.append(W[k] + u * (W[k + 1] - W[k]))
    cen = X[tets].mean(axis=1)

    def refined_at(c):
        return ((cen - c) ** 2).sum(1) < radius * radius

    def mask_of(ref):
        m = np.zeros(T, np.uint8)
        m[:T0] = ~ref
        m[T0:] = np.repeat(ref, 8)
        return m

    ref = refined_at(centers[0])
    mask0 = mask_of(ref)
    fr = []
    for t in range(1, frames + 1):
        nref = refined_at(centers[t])
        up = np.flatnonzero(nref & ~ref)
        down = np.flatnonzero(~nref & ref)
        off = list(up) + [T0 + 8 * p + k for p in down for k in range(8)]
        on = [T0 + 8 * p + k for p in up for k in range(8)] + list(down)
        fr.append(make_edits(off=off, on=on))
        ref = nref
    return Workload(f"refinement_N{N}_r{radius}", Xall, tets_all, np.full(T, 1e5),
                    np.full(T, 0.3), mask0, fr,
                    {"N": N, "radius": radius, "n_coarse": T0, "centers": np.array(centers)})


def batched_instances(seed: int = 0, count: int = 64, tmin: float = 2e3, tmax: float = 5e4,
                      frames: int = 24) -> list:
    """Batch of independent jittered cube meshes: tet counts drawn log-uniformly in
    [tmin, tmax], realised as N = max(1, round(cbrt(T/6))) hexes per side; each instance has
    its own deactivate/reactivate stream at a rate r drawn uniformly from [0.1%, 5%]
    (deactivate r of the active tets, reactivate r/4 of T per frame)."""
    rng = rng_for(4, seed)
    Ts = np.exp(rng.uniform(np.log(tmin), np.log(tmax), size=count))
    rates = rng.uniform(0.001, 0.05, size=count)
    out = []
    for i in range(count):
        N = max(1, int(round((Ts[i] / 6.0) ** (1.0 / 3.0))))
        r = rng_for(4, 1 + seed * count + i)
        X, tets, gi = kuhn_cube(N, 0.15, r)
        T = tets.shape[0]
        mask0 = np.ones(T, np.uint8)
        fr = deact_react_stream(r, T, mask0, frames, float(rates[i]), float(rates[i]) / 4)
        out.append(Workload(f"batch{i}_N{N}", X, tets, np.full(T, 1e5), np.full(T, 0.3),
                            mask0, fr, {"N": N, "rate": float(rates[i])}))
    return out


def adjoint_block(seed: int = 0, N: int = 20, frames: int = 24, traction: float = 1e3
                  ) -> Workload:
    """Adjoint workload: N^3 hexes x 6 (jitter +-0.1h), E lognormal (median 1e5, sigma 0.3),
    nu = 0.3, 2%-per-frame deactivation stream.  meta holds the load: nodes of the bottom
    lattice layer are clamped; a uniform downward traction acts on the top face, lumped as
    area/3 per node of each top-surface triangle of the superset (fixed over frames)."""
    rng = rng_for(5, seed)
    X, tets, gi = kuhn_cube(N, 0.1, rng)
    T = tets.shape[0]
    E = lognormal_E(rng, T)
    mask0 = np.ones(T, np.uint8)
    fr = deact_react_stream(rng, T, mask0, frames, 0.02, 0.0)
    top = gi[:, 2] == N
    f = np.zeros_like(X)
    for a, b, c in itertools.combinations(range(4), 3):
        tri = tets[:, [a, b, c]]
        on = top[tri].all(axis=1)
        tri = tri[on]
        area = 0.5 * np.linalg.norm(np.cross(X[tri[:, 1]] - X[tri[:, 0]],
                                             X[tri[:, 2]] - X[tri[:, 0]]), axis=1)
        for k in range(3):
            np.add.at(f[:, 2], tri[:, k], -traction * area / 3.0)
    clamped = gi[:, 2] == 0
    return Workload(f"adjoint_block_N{N}", X, tets, E, np.full(T, 0.3), mask0, fr,
                    {"N": N, "load": f.reshape(-1), "clamped_nodes": clamped, "grid_index": gi})


def free_dofs(tets: np.ndarray, mask: np.ndarray, clamped_nodes: np.ndarray) -> np.ndarray:
    """Host connectivity (Sec. 3.6's union-find role, via scipy connected components):
    active tets are linked when they share a face; a face-connected component is anchored
    when one of its tets has three or more clamped nodes.  Returns a (3n,) bool array: True
    for DOFs of nodes of anchored components that are not clamped.  All other DOFs are
    pinned, which keeps the reduced stiffness positive definite."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = clamped_nodes.shape[0]
    act = np.flatnonzero(mask)
    free = np.zeros(3 * n, bool)
    if act.size == 0:
        return free
    at = tets[act].astype(np.int64)
    faces = np.concatenate([np.sort(at[:, list(c)], axis=1)
                            for c in itertools.combinations(range(4), 3)], 0)
    owner = np.tile(np.arange(act.size), 4)
    key = (faces[:, 0] * n + faces[:, 1]) * n + faces[:, 2]
    o = np.argsort(key, kind="stable")
    ks, ow = key[o], owner[o]
    same = np.flatnonzero(ks[1:] == ks[:-1])
    A = coo_matrix((np.ones(same.size), (ow[same], ow[same + 1])), shape=(act.size, act.size))
    ncomp, lab = connected_components(A, directed=False)
    anchored_tet = clamped_nodes[at].sum(axis=1) >= 3
    good = np.zeros(ncomp, bool)
    good[lab[anchored_tet]] = True
    nodes = np.unique(at[good[lab]].reshape(-1))
    nodes = nodes[~clamped_nodes[nodes]]
    for i in range(3):
        free[3 * nodes + i] = True
    return free
