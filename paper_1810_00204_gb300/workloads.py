"""Seeded synthetic inputs shaped like the paper's 2-D navigation scenarios.

This module only *draws inputs*: occupancy maps, beacon cells, start and goal
cells, the initial belief b0 and the per-cell cost map.  It holds none of the
planning arithmetic (no transition model, no observation labels, no value
iteration, no Bayes update): both the CUDA path and the FP64 oracle consume
the same `Workload` objects and derive everything else themselves.

Layout: every array here is unpadded row-major [H][W]; cell index x = r*W + c.
The paper's maps exist only as figure images (Sec. V, Fig. 3-4), so the five
generators below stand in for them; their recipes are written out in the
design notes.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    """One planning problem: the tuple (X, A, Z, T, O, R, b0, gamma) of Sec. II
    in its generated form, plus the tree-search parameters."""

    name: str
    H: int
    W: int
    occ: np.ndarray            # uint8 [H][W]; m(x) = 1 for an occupied cell
    beacons: np.ndarray        # int32 [B]; distinct free cells (flat index)
    sense_range: int           # Manhattan sensing range of a beacon
    goal: int                  # flat index of the goal cell
    start: int                 # flat index of the true start cell
    slip: float                # epsilon: probability of each perpendicular slip
    accuracy: float            # alpha: probability of observing the true label
    discount: float            # gamma
    b0: np.ndarray             # float32 [H][W]; zero on occupied cells, sums to 1
    depth: int = 2             # tree depth d
    K: int = 4                 # forward samples per (V-node, action)
    seed: int = 0              # Philox key for the observation samples
    episode: int = 0           # Philox counter word 1
    vi_tol: float = 1e-6
    vi_dtype: str = "f64"
    vi_max_sweeps: int = 100000
    vi_truncated: int = 0      # >0: run exactly this many sweeps
    cost: Optional[np.ndarray] = None  # float32 [H][W] per-cell cost, or None
    p_sensor: float = 0.95     # the nine-action model's occupancy sensors: P(reading right)

    def __setattr__(self, name, value):
        # The model parameters are float32 numbers (the C ABI carries them as
        # float); storing them rounded lets every consumer see the same value.
        if name in ("slip", "accuracy", "discount", "p_sensor"):
            value = float(np.float32(value))
        object.__setattr__(self, name, value)

    @property
    def B(self) -> int:
        return int(len(self.beacons))

    @property
    def n_cells(self) -> int:
        return self.H * self.W


# ----------------------------------------------------------------------------
# map drawing helpers (input preparation only)
# ----------------------------------------------------------------------------

def _iid_occupancy(rng, H, W, p):
    return (rng.random((H, W)) < p).astype(np.uint8)


def _rect_occupancy(rng, H, W, target, side_lo=1, side_hi=4):
    occ = np.zeros((H, W), np.uint8)
    while occ.mean() < target:
        h = int(rng.integers(side_lo, side_hi + 1))
        w = int(rng.integers(side_lo, side_hi + 1))
        r = int(rng.integers(0, H))
        c = int(rng.integers(0, W))
        occ[r:r + h, c:c + w] = 1
    return occ


def _rooms_occupancy(rng, H, W, room=32, door=3, target=0.25):
    occ = np.zeros((H, W), np.uint8)
    # 1-cell walls on every room boundary
    for r in range(room - 1, H, room):
        occ[r, :] = 1
    for c in range(room - 1, W, room):
        occ[:, c] = 1
    # a door of width `door` in every wall segment between two rooms
    for r in range(room - 1, H, room):
        for c0 in range(0, W, room):
            seg = min(room - 1, W - c0)
            if seg > door:
                d = int(rng.integers(0, seg - door + 1))
                occ[r, c0 + d:c0 + d + door] = 0
    for c in range(room - 1, W, room):
        for r0 in range(0, H, room):
            seg = min(room - 1, H - r0)
            if seg > door:
                d = int(rng.integers(0, seg - door + 1))
                occ[r0 + d:r0 + d + door, c] = 0
    # random straight wall segments inside rooms until the target density
    while occ.mean() < target:
        length = int(rng.integers(4, 17))
        r = int(rng.integers(0, H))
        c = int(rng.integers(0, W))
        if rng.random() < 0.5:
            occ[r, c:c + length] = 1
        else:
            occ[r:r + length, c] = 1
    return occ


def _components(occ):
    """Label the 4-connected components of free cells."""
    from scipy import ndimage
    comp, n = ndimage.label(occ == 0, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    sizes = np.bincount(comp.ravel(), minlength=n + 1)
    sizes[0] = 0                      # label 0 = occupied cells
    return comp, sizes


def _start_goal(rng, occ):
    comp, sizes = _components(occ)
    big = int(np.argmax(sizes))        # largest free component
    cells = np.flatnonzero(comp.ravel() == big)
    goal, start = rng.choice(cells, size=2, replace=False)
    return int(goal), int(start)


def _beacons(rng, occ, B, exclude=()):
    free = np.flatnonzero(occ.ravel() == 0)
    free = np.setdiff1d(free, np.asarray(exclude, np.int64))
    return np.sort(rng.choice(free, size=B, replace=False)).astype(np.int32)


def _b0_block(occ, start, half=1):
    """Uniform over the free cells of the (2*half+1)^2 block centred on start."""
    H, W = occ.shape
    r0, c0 = divmod(start, W)
    b = np.zeros((H, W), np.float64)
    for r in range(max(0, r0 - half), min(H, r0 + half + 1)):
        for c in range(max(0, c0 - half), min(W, c0 + half + 1)):
            if not occ[r, c]:
                b[r, c] = 1.0
    b /= b.sum()
    return b.astype(np.float32)


def _b0_gauss(occ, start, sigma=4.0):
    """exp(-|x-s|^2 / (2 sigma^2)) over every free cell, normalised."""
    H, W = occ.shape
    r0, c0 = divmod(start, W)
    rr, cc = np.mgrid[0:H, 0:W]
    b = np.exp(-((rr - r0) ** 2 + (cc - c0) ** 2) / (2.0 * sigma * sigma))
    b[occ.astype(bool)] = 0.0
    b /= b.sum()
    return b.astype(np.float32)


# ----------------------------------------------------------------------------
# the five workload families
# ----------------------------------------------------------------------------

def tiny(seed: int = 0, H: int = 20, W: int = 20, depth: int = 2, K: int = 4) -> Workload:
    """20x20, iid 15 % obstacles, 4 beacons (range 3, alpha 0.9), eps 0.1,
    gamma 0.95, FP64 VI to 1e-6, b0 uniform over the 3x3 block at start,
    depth 2, K = 4."""
    rng = np.random.default_rng([1, seed])
    occ = _iid_occupancy(rng, H, W, 0.15)
    goal, start = _start_goal(rng, occ)
    return Workload(
        name=f"tiny{H}x{W}", H=H, W=W, occ=occ,
        beacons=_beacons(rng, occ, 4), sense_range=3, goal=goal, start=start,
        slip=0.1, accuracy=0.9, discount=0.95, b0=_b0_block(occ, start),
        depth=depth, K=K, seed=seed, episode=0, vi_tol=1e-6, vi_dtype="f64")


def mid(seed: int = 0, H: int = 128, W: int = 128, depth: int = 3, K: int = 8) -> Workload:
    """128x128, >= 20 % obstacles as 1-4 cell rectangles, 16 beacons (range 5,
    alpha 0.85), eps 0.1, gamma 0.97, FP32 VI to 1e-5, Gaussian b0 (sigma 4),
    depth 3, K = 8."""
    rng = np.random.default_rng([2, seed])
    occ = _rect_occupancy(rng, H, W, 0.20)
    goal, start = _start_goal(rng, occ)
    return Workload(
        name=f"mid{H}x{W}", H=H, W=W, occ=occ,
        beacons=_beacons(rng, occ, 16), sense_range=5, goal=goal, start=start,
        slip=0.1, accuracy=0.85, discount=0.97, b0=_b0_gauss(occ, start),
        depth=depth, K=K, seed=seed, episode=0, vi_tol=1e-5, vi_dtype="f32")


def batched(seed: int = 0, E: int = 256, lo: int = 32, hi: int = 256,
            depth: int = 3, K: int = 8) -> List[Workload]:
    """E episodes on maps of uneven size: H, W ~ U{lo..hi}, density
    U[0.10, 0.25] (rectangles), B ~ U{4..32} (range 5, alpha 0.85),
    eps ~ U[0.05, 0.15], gamma 0.97, Gaussian b0, depth 3, K = 8."""
    rng = np.random.default_rng([3, seed])
    out = []
    for e in range(E):
        H = int(rng.integers(lo, hi + 1))
        W = int(rng.integers(lo, hi + 1))
        occ = _rect_occupancy(rng, H, W, float(rng.uniform(0.10, 0.25)))
        goal, start = _start_goal(rng, occ)
        B = int(rng.integers(4, 33))
        out.append(Workload(
            name=f"batch{e}:{H}x{W}", H=H, W=W, occ=occ,
            beacons=_beacons(rng, occ, B), sense_range=5, goal=goal, start=start,
            slip=float(rng.uniform(0.05, 0.15)), accuracy=0.85, discount=0.97,
            b0=_b0_gauss(occ, start), depth=depth, K=K, seed=seed, episode=e,
            vi_tol=1e-5, vi_dtype="f32"))
    return out


def large(seed: int = 0, H: int = 512, W: int = 512, depth: int = 3, K: int = 4) -> Workload:
    """512x512 rooms-and-walls map at 25 % occupancy, 64 beacons (range 8,
    alpha 0.8), eps 0.1, gamma 0.97, FP32 VI to 1e-5, Gaussian b0,
    depth 3, K = 4."""
    rng = np.random.default_rng([4, seed])
    occ = _rooms_occupancy(rng, H, W)
    goal, start = _start_goal(rng, occ)
    return Workload(
        name=f"large{H}x{W}", H=H, W=W, occ=occ,
        beacons=_beacons(rng, occ, 64), sense_range=8, goal=goal, start=start,
        slip=0.1, accuracy=0.8, discount=0.97, b0=_b0_gauss(occ, start),
        depth=depth, K=K, seed=seed, episode=0, vi_tol=1e-5, vi_dtype="f32")


def diff(seed: int = 0, H: int = 128, W: int = 128, depth: int = 3, K: int = 8,
         sweeps: int = 200) -> Workload:
    """The tiny model's parameters on a 128x128 grid, a per-cell cost map
    c ~ U[0, 0.5] with c(goal) = 0, 200 truncated VI sweeps, depth 3, K = 8."""
    rng = np.random.default_rng([5, seed])
    occ = _iid_occupancy(rng, H, W, 0.15)
    goal, start = _start_goal(rng, occ)
    cost = rng.uniform(0.0, 0.5, size=(H, W)).astype(np.float32)
    cost.ravel()[goal] = 0.0
    return Workload(
        name=f"diff{H}x{W}", H=H, W=W, occ=occ,
        beacons=_beacons(rng, occ, 4), sense_range=3, goal=goal, start=start,
        slip=0.1, accuracy=0.9, discount=0.95, b0=_b0_block(occ, start),
        depth=depth, K=K, seed=seed, episode=0, vi_tol=0.0, vi_dtype="f32",
        vi_truncated=sweeps, cost=cost)


def episodes(w: Workload, R: int, seed: int = 0, first_episode: int = 0) -> List[Workload]:
    """R planning requests on the map of `w`: the same grid, beacons, goal and
    model, each with its own start cell (drawn from the goal's free
    component), its own b0 of the same family as `w`, and its own Philox
    episode word."""
    rng = np.random.default_rng([6, seed, first_episode])
    comp, _ = _components(w.occ)
    cells = np.flatnonzero(comp.ravel() == comp.ravel()[w.goal])
    cells = cells[cells != w.goal]
    gaussian = np.count_nonzero(w.b0) > 9
    out = []
    for r in range(R):
        start = int(rng.choice(cells))
        b0 = _b0_gauss(w.occ, start) if gaussian else _b0_block(w.occ, start)
        out.append(dataclasses.replace(w, name=f"{w.name}/ep{first_episode + r}", start=start, b0=b0,
                                       episode=first_episode + r))
    return out


def custom(H, W, occ, beacons, sense_range, goal, start, slip, accuracy, discount,
           b0, depth=1, K=4, seed=0, episode=0, cost=None, name="custom"):
    """Wrap hand-made arrays (test fixtures) as a Workload."""
    occ = np.asarray(occ, np.uint8).reshape(H, W)
    b0 = np.asarray(b0, np.float32).reshape(H, W)
    return Workload(
        name=name, H=H, W=W, occ=occ, beacons=np.asarray(beacons, np.int32),
        sense_range=int(sense_range), goal=int(goal), start=int(start),
        slip=float(slip), accuracy=float(accuracy), discount=float(discount),
        b0=b0, depth=depth, K=K, seed=seed, episode=episode,
        cost=None if cost is None else np.asarray(cost, np.float32).reshape(H, W))


CONFIGS = {"tiny": tiny, "mid": mid, "batched": batched, "large": large, "diff": diff}
