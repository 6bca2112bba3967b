"""Seeded synthetic occupancy grids.

The paper trains on binary-image maps (Map0..Map31, Sec. 4.3.2 "Task2Task
generalization") that are not available here.  These generators stand in for
them with the shapes the workloads name: a square uint8 grid, border walls one
cell thick, random axis-aligned rectangles and discs, and two cleared discs
around the start and goal areas (the paper's episodes run from the lower-left
to the upper-right corner, Sec. 4.3.1 "Problem formulation of LLP").

Grid convention: ``grid[cy, cx]`` (row = y, column = x), nonzero = occupied.
Cell (cx, cy) covers the square [cx, cx+1) x [cy, cy+1) in cell units.
"""

from __future__ import annotations

import numpy as np

# Start point S and goal point G sit START_OFFSET cells in from the lower-left
# and upper-right corners; both are cleared with radius CLEAR_RADIUS.
START_OFFSET = 30
CLEAR_RADIUS = 25


def map_start_goal(w: int, h: int, offset: int = START_OFFSET):
    """Nominal start S and goal G (cell units) of a w x h map."""
    return (float(offset), float(offset)), (float(w - offset), float(h - offset))


def _disc_fill(g: np.ndarray, ox2: int, oy2: int, r: int, value: int) -> None:
    """Set to ``value`` every cell whose centre lies within r of (ox2/2, oy2/2).

    Exact integer test: (2cx+1-ox2)^2 + (2cy+1-oy2)^2 <= (2r)^2, evaluated on
    the disc's bounding box only.
    """
    h, w = g.shape
    x0 = max(0, (ox2 - 2 * r - 1) // 2)
    x1 = min(w, (ox2 + 2 * r) // 2 + 1)
    y0 = max(0, (oy2 - 2 * r - 1) // 2)
    y1 = min(h, (oy2 + 2 * r) // 2 + 1)
    if x0 >= x1 or y0 >= y1:
        return
    cy, cx = np.mgrid[y0:y1, x0:x1]
    dx = 2 * cx + 1 - ox2
    dy = 2 * cy + 1 - oy2
    m = dx * dx + dy * dy <= 4 * r * r
    g[y0:y1, x0:x1][m] = value


def make_map(
    seed: int,
    side: int = 366,
    height: int | None = None,
    n_rects: int = 20,
    rect_min: int = 5,
    rect_max: int = 40,
    n_circles: int = 10,
    circ_min: int = 3,
    circ_max: int = 15,
    border: bool = True,
    clear_start_goal: bool = True,
) -> np.ndarray:
    """A seeded uint8 occupancy grid of shape (height, side).

    Recipe: border walls 1 cell thick; ``n_rects`` rectangles with sides drawn
    uniformly from {rect_min..rect_max}, placed fully inside the border;
    ``n_circles`` discs with radius uniform in {circ_min..circ_max} and an
    integer centre; then the discs of radius CLEAR_RADIUS around S and G are
    cleared so that every episode starts and ends in free space.
    """
    w = int(side)
    h = int(height if height is not None else side)
    rng = np.random.default_rng(int(seed))
    g = np.zeros((h, w), dtype=np.uint8)
    if border:
        g[0, :] = 1
        g[-1, :] = 1
        g[:, 0] = 1
        g[:, -1] = 1
    for _ in range(n_rects):
        rw = int(rng.integers(rect_min, rect_max + 1))
        rh = int(rng.integers(rect_min, rect_max + 1))
        rw = min(rw, w - 2)
        rh = min(rh, h - 2)
        x0 = int(rng.integers(1, w - 1 - rw + 1))
        y0 = int(rng.integers(1, h - 1 - rh + 1))
        g[y0:y0 + rh, x0:x0 + rw] = 1
    for _ in range(n_circles):
        r = int(rng.integers(circ_min, circ_max + 1))
        lo = 1 + r
        ox = int(rng.integers(lo, max(lo + 1, w - 1 - r)))
        oy = int(rng.integers(lo, max(lo + 1, h - 1 - r)))
        _disc_fill(g, 2 * ox, 2 * oy, r, 1)
    if clear_start_goal:
        (sx, sy), (gx, gy) = map_start_goal(w, h)
        for px, py in ((sx, sy), (gx, gy)):
            _disc_fill(g, int(2 * px), int(2 * py), CLEAR_RADIUS, 0)
        if border:
            g[0, :] = 1
            g[-1, :] = 1
            g[:, 0] = 1
            g[:, -1] = 1
    return g


def empty_map(w: int, h: int | None = None, border: bool = False) -> np.ndarray:
    """An all-free grid (optionally with border walls), for closed-form tests."""
    h = w if h is None else h
    g = np.zeros((h, w), dtype=np.uint8)
    if border:
        g[0, :] = 1
        g[-1, :] = 1
        g[:, 0] = 1
        g[:, -1] = 1
    return g


def random_tiny_map(seed: int, w: int, h: int | None = None, density: float = 0.2) -> np.ndarray:
    """A tiny grid with i.i.d. occupied cells, for brute-force ray tests."""
    h = w if h is None else h
    rng = np.random.default_rng(int(seed))
    return (rng.random((h, w)) < density).astype(np.uint8)
