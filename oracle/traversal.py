"""Batch-zigzag visiting order of a Cartesian grid (Sec. 2.3, eq. (batch)) --
TEST INFRASTRUCTURE ONLY (see the package docstring for who may import it).

The grid holds nx x ny points, point (ix, iy) at linear index iy * nx + ix.
Eq. (batch) groups vertically adjacent points into column batches of b
points, {x + i y, x + i (y + dy), ..., x + i (y + (b - 1) dy)}; the batches
with the same starting height form a batch row.  The traversal is two nested
loops: the outer one a row-wise zigzag over the batches (batch rows from the
bottom; the first swept left to right, the next right to left, alternating),
the inner one the points of the batch, visited vertically in the order eq.
(batch) lists them (increasing y).

Reading where the text leaves a choice: when b does not divide ny, the top
batch row holds the ny mod b remaining points of each column.

Written as the definition: list every batch with its sort key (batch row,
then position along the row's sweep direction), sort, and expand each batch.
Pinned in tests/test_oracle_traversal.py by hand-worked small grids, the
special cases b = 1 (the plain row-wise zigzag) and b >= ny (a left-to-right
sweep of whole columns), and the step geometry of the sequence.
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
