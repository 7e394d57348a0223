"""The batch-zigzag traversal (Sec. 2.3, eq. (batch)): the oracle pinned by
hand-worked grids, the special cases the definition reduces to and the
geometry of its steps; the library's host-side order (pseudo_traversal_order,
the one the recycling path walks) compared with it index for index."""
import numpy as np
import pytest

from oracle.traversal import batch_zigzag, hilbert, morton

# (nx, ny, b) -> visiting order worked out by hand on the grid
# z[iy * nx + ix]; first batch row left to right, second right to left
HAND = {
    # 3 x 4 grid, b = 2: batches (x, rows 0-1) for x = 0, 1, 2, then
    # (x, rows 2-3) for x = 2, 1, 0
    (3, 4, 2): [0, 3, 1, 4, 2, 5, 8, 11, 7, 10, 6, 9],
    # 2 x 5 grid, b = 2: the top batch row holds one point per column
    (2, 5, 2): [0, 2, 1, 3, 5, 7, 4, 6, 8, 9],
    # 4 x 3 grid, b = 3: one batch row, whole columns left to right
    (4, 3, 3): [0, 4, 8, 1, 5, 9, 2, 6, 10, 3, 7, 11],
}


@pytest.mark.parametrize("key", sorted(HAND))
def test_hand_worked_grids(key):
    assert batch_zigzag(*key) == HAND[key]


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 3), (5, 2), (4, 7)])
def test_b1_is_the_row_wise_zigzag(nx, ny):
    # b = 1: the textbook boustrophedon, even rows left to right, odd rows right to left
    want = []
    for iy in range(ny):
        xs = range(nx) if iy % 2 == 0 else range(nx - 1, -1, -1)
        want += [iy * nx + ix for ix in xs]
    assert batch_zigzag(nx, ny, 1) == want


@pytest.mark.parametrize("nx,ny,b", [(3, 4, 4), (5, 3, 9)])
def test_b_at_least_ny_sweeps_whole_columns(nx, ny, b):
    assert batch_zigzag(nx, ny, b) == [iy * nx + ix for ix in range(nx) for iy in range(ny)]


@pytest.mark.parametrize("nx,ny,b", [(9, 9, 3), (7, 10, 3), (12, 5, 4), (1, 6, 4), (6, 1, 2)])
def test_permutation_and_step_geometry(nx, ny, b):
    order = batch_zigzag(nx, ny, b)
    assert sorted(order) == list(range(nx * ny))
    pts = [(i % nx, i // nx) for i in order]
    for (x0, y0), (x1, y1) in zip(pts, pts[1:]):
        if y0 // b == y1 // b and x0 == x1:  # inside a batch: one step up
            assert y1 == y0 + 1
        elif y0 // b == y1 // b:  # next batch of the same batch row: one column over, back to its bottom
            assert abs(x1 - x0) == 1 and y1 == (y1 // b) * b
            assert (x1 - x0) == (1 if (y0 // b) % 2 == 0 else -1)
        else:  # next batch row: same column (the zigzag turn), one point up
            assert x1 == x0 and y1 == y0 + 1 and y1 % b == 0


def test_degenerate_grids():
    assert batch_zigzag(0, 5, 2) == []
    assert batch_zigzag(3, 0, 2) == []
    with pytest.raises(ValueError):
        batch_zigzag(3, 2, 0)


@pytest.mark.parametrize("nx,ny,b", [(3, 4, 2), (2, 5, 2), (9, 9, 3), (200, 200, 20), (37, 53, 7), (8, 3, 1),
                                     (5, 4, 100), (1, 1, 1), (64, 64, 64)])
def test_library_order_matches_oracle(nx, ny, b):
    import paper_2606_26785_b300 as p

    got = p.traversal_order(nx, ny, b)
    assert got.dtype == np.int32
    assert got.tolist() == batch_zigzag(nx, ny, b)


def test_library_order_unordered_points_and_errors():
    import paper_2606_26785_b300 as p

    assert p.traversal_order(0, 0, 4, npts=6).tolist() == list(range(6))
    assert p.traversal_order(0, 0, 4, npts=0).tolist() == []
    with pytest.raises(p.PseudoError):
        p.traversal_order(3, 4, 2, npts=11)
    with pytest.raises(p.PseudoError):
        p.traversal_order(-1, 4, 2, npts=4)
    with pytest.raises(p.PseudoError):
        p.traversal_order(3, 4, 0)


def test_library_order_matches_oracle_on_random_grids():
    from hypothesis import given, settings
    from hypothesis import strategies as st

    import paper_2606_26785_b300 as p

    @settings(max_examples=300, deadline=None, derandomize=True)
    @given(st.integers(1, 90), st.integers(1, 90), st.integers(1, 100))
    def check(nx, ny, b):
        assert p.traversal_order(nx, ny, b).tolist() == batch_zigzag(nx, ny, b)
        assert p.traversal_order(nx, ny, b, p.TRAVERSE_HILBERT).tolist() == hilbert(nx, ny)
        assert p.traversal_order(nx, ny, b, p.TRAVERSE_MORTON).tolist() == morton(nx, ny)

    check()


# ------------------------------------------------ Hilbert and Morton (Sec. 5)


def _xy(order, nx):
    return [(i % nx, i // nx) for i in order]


def test_hilbert_side_2_and_4_by_hand():
    assert _xy(hilbert(2, 2), 2) == [(0, 0), (0, 1), (1, 1), (1, 0)]
    # the order-2 curve: the side-2 curve transposed, twice shifted, then anti-transposed
    assert _xy(hilbert(4, 4), 4) == [(0, 0), (1, 0), (1, 1), (0, 1), (0, 2), (0, 3), (1, 3), (1, 2),
                                     (2, 2), (2, 3), (3, 3), (3, 2), (3, 1), (2, 1), (2, 0), (3, 0)]


@pytest.mark.parametrize("N", [1, 2, 8, 16, 32])
def test_hilbert_unit_steps_and_end_points(N):
    pts = _xy(hilbert(N, N), N)
    assert sorted(pts) == [(x, y) for x in range(N) for y in range(N)]
    assert pts[0] == (0, 0) and pts[-1] == (N - 1, 0)
    for (x0, y0), (x1, y1) in zip(pts, pts[1:]):
        assert abs(x1 - x0) + abs(y1 - y0) == 1
    # every aligned quadrant of side N/2 is visited in one piece
    if N >= 2:
        h = N // 2
        quads = [(x // h, y // h) for x, y in pts]
        assert sum(a != b for a, b in zip(quads, quads[1:])) == 3


def test_morton_side_4_by_hand_and_aligned_blocks():
    assert _xy(morton(4, 4), 4) == [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (3, 0), (2, 1), (3, 1),
                                    (0, 2), (1, 2), (0, 3), (1, 3), (2, 2), (3, 2), (2, 3), (3, 3)]
    N = 16
    pts = _xy(morton(N, N), N)
    for s in (2, 4, 8):
        blocks = [(x // s, y // s) for x, y in pts]
        runs = 1 + sum(a != b for a, b in zip(blocks, blocks[1:]))
        assert runs == (N // s) ** 2  # each aligned s x s block in one contiguous run


@pytest.mark.parametrize("nx,ny", [(3, 2), (5, 9), (17, 4), (1, 7)])
def test_curves_on_rectangles_are_the_square_curve_cropped(nx, ny):
    side = 1
    while side < max(nx, ny):
        side *= 2
    for f in (hilbert, morton):
        full = _xy(f(side, side), side)
        assert _xy(f(nx, ny), nx) == [(x, y) for x, y in full if x < nx and y < ny]


@pytest.mark.parametrize("nx,ny", [(3, 4), (9, 9), (40, 40), (37, 53), (1, 1), (200, 200), (64, 3)])
def test_library_hilbert_and_morton_match_oracle(nx, ny):
    import paper_2606_26785_b300 as p

    assert p.traversal_order(nx, ny, 20, p.TRAVERSE_HILBERT).tolist() == hilbert(nx, ny)
    assert p.traversal_order(nx, ny, 20, p.TRAVERSE_MORTON).tolist() == morton(nx, ny)


def test_library_traversal_errors_and_unordered_points():
    import paper_2606_26785_b300 as p

    with pytest.raises(p.PseudoError):
        p.traversal_order(4, 4, 2, 3)
    assert p.traversal_order(0, 0, 2, p.TRAVERSE_HILBERT, npts=5).tolist() == list(range(5))
