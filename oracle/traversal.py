"""Grid traversal orders of the recycling path -- TEST INFRASTRUCTURE ONLY
(see the package docstring for who may import it).

The grid holds nx x ny points, point (ix, iy) at linear index iy * nx + ix.

Batch zigzag (Sec. 2.3, eq. (batch)).  Eq. (batch) groups vertically adjacent
points into column batches of b points, {x + i y, x + i (y + dy), ..., x + i
(y + (b - 1) dy)}; the batches with the same starting height form a batch
row.  The traversal is two nested loops: the outer one a row-wise zigzag over
the batches (batch rows from the bottom; the first swept left to right, the
next right to left, alternating), the inner one the points of the batch,
visited vertically in the order eq. (batch) lists them (increasing y).
Reading where the text leaves a choice: when b does not divide ny, the top
batch row holds the ny mod b remaining points of each column.  Written as the
definition: list every batch with its sort key (batch row, then position
along the row's sweep direction), sort, and expand each batch.

Hilbert and Morton orders (Sec. 5 names both as locality-preserving
alternatives).  Both are defined on a square of side N = 2^q, the smallest
holding the grid; points outside the grid are skipped, the rest keep the
curve's order.  Written as their recursive definitions on quadrants:
* Hilbert: the curve of side N runs from (0, 0) to (N - 1, 0) (side 2:
  (0, 0), (0, 1), (1, 1), (1, 0)).  It is four curves of side N/2: the lower-left one with x
  and y exchanged, the upper-left and upper-right ones as they are, and the
  lower-right one reflected in its anti-diagonal, so that each ends next to
  where the following one starts.
* Morton (Z-order): the quadrants in the order lower-left, lower-right,
  upper-left, upper-right, each traversed the same way.

Pinned in tests/test_oracle_traversal.py by hand-worked small grids, the
special cases b = 1 (the plain row-wise zigzag) and b >= ny (a left-to-right
sweep of whole columns), the step geometry of the zigzag sequence, the unit
steps and end points of the Hilbert curve and the contiguous aligned blocks
of the Morton order.
"""
from __future__ import annotations


def batch_zigzag(nx: int, ny: int, b: int) -> list[int]:
    if b < 1:
        raise ValueError("batch size b must be >= 1")
    if nx <= 0 or ny <= 0:
        return []
    batches = []  # (batch row, sweep position, x, first y)
    for y0 in range(0, ny, b):
        row = y0 // b
        for ix in range(nx):
            sweep = ix if row % 2 == 0 else -ix
            batches.append((row, sweep, ix, y0))
    batches.sort()
    order = []
    for _, _, ix, y0 in batches:
        for iy in range(y0, min(y0 + b, ny)):
            order.append(iy * nx + ix)
    return order


def _side(nx: int, ny: int) -> int:
    N = 1
    while N < max(nx, ny):
        N *= 2
    return N


def _hilbert_points(N: int) -> list[tuple[int, int]]:
    if N == 1:
        return [(0, 0)]
    h = N // 2
    sub = _hilbert_points(h)
    pts = [(y, x) for x, y in sub]                      # lower left, transposed
    pts += [(x, y + h) for x, y in sub]                 # upper left
    pts += [(x + h, y + h) for x, y in sub]             # upper right
    pts += [(2 * h - 1 - y, h - 1 - x) for x, y in sub]  # lower right, anti-transposed
    return pts


def _morton_points(N: int) -> list[tuple[int, int]]:
    if N == 1:
        return [(0, 0)]
    h = N // 2
    sub = _morton_points(h)
    return [(x + dx, y + dy) for dx, dy in ((0, 0), (h, 0), (0, h), (h, h)) for x, y in sub]


def _cropped(points, nx: int, ny: int) -> list[int]:
    return [y * nx + x for x, y in points if x < nx and y < ny]


def hilbert(nx: int, ny: int) -> list[int]:
    if nx <= 0 or ny <= 0:
        return []
    return _cropped(_hilbert_points(_side(nx, ny)), nx, ny)


def morton(nx: int, ny: int) -> list[int]:
    if nx <= 0 or ny <= 0:
        return []
    return _cropped(_morton_points(_side(nx, ny)), nx, ny)
