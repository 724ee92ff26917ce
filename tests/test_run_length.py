"""Host-side choice of the paired kernel's run length (no GPU needed).

The choice never changes results (the GPU tests check that bit for bit); these
tests pin the cost model's qualitative behaviour: runs that fit the rows of a
dense block, no runs where items are not x-neighbours, and no runs when there
are fewer items than CTAs.
"""
import numpy as np
import pytest

from paper_2107_14790_b300 import tgv

OFFSETS = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
           (-1, 1, 0), (-1, 0, 1), (1, -1, 0), (0, -1, 1), (1, 0, -1), (0, 1, -1)]


def nbr_rows(coords):
    """Neighbour rows of active bricks (faces, then mixed-sign edges; -1 none)."""
    index = {tuple(c): i for i, c in enumerate(coords.tolist())}
    rows = np.full((len(coords), 12), -1, np.int32)
    for i, c in enumerate(coords.tolist()):
        for k, o in enumerate(OFFSETS):
            rows[i, k] = index.get((c[0] + o[0], c[1] + o[1], c[2] + o[2]), -1)
    return rows


def dense(nx, ny, nz):
    return np.array([(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)], np.int32)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()


@pytest.mark.parametrize("edge", [32, 24, 20])
def test_dense_block_runs_divide_the_row(edge):
    rows = nbr_rows(dense(edge, edge, edge))
    R = tgv.tgv_pair_run_length(rows, slots=296)
    assert R > 1 and edge % R == 0, R


def test_no_runs_without_x_neighbours_in_sequence():
    rows = nbr_rows(dense(24, 24, 24))
    rev = np.arange(len(rows), dtype=np.int32)[::-1]
    assert tgv.tgv_pair_run_length(rows, rev, slots=296) == 1
    # a column-major order: consecutive items are y-neighbours
    c = dense(24, 24, 24)
    col = np.lexsort((c[:, 1], c[:, 0], c[:, 2])).astype(np.int32)
    assert tgv.tgv_pair_run_length(rows, col, slots=296) == 1


def test_fewer_items_than_ctas_take_no_runs():
    rows = nbr_rows(dense(8, 4, 4))
    assert tgv.tgv_pair_run_length(rows, slots=296) == 1


def test_sixteen_bit_storage_takes_no_runs():
    rows = nbr_rows(dense(32, 32, 32))
    assert tgv.tgv_pair_run_length(rows, slots=296, storage="fp32") > 1
    for st in ("fp16", "bf16"):
        assert tgv.tgv_pair_run_length(rows, slots=296, storage=st) == 1


def test_work_list_is_checked():
    rows = nbr_rows(dense(16, 16, 16))
    with pytest.raises(tgv.TgvError):
        tgv.tgv_pair_run_length(rows, np.array([0, 0], np.int32))
    with pytest.raises(tgv.TgvError):
        tgv.tgv_pair_run_length(rows, np.array([len(rows)], np.int32))
    with pytest.raises(tgv.TgvError):
        tgv.tgv_pair_run_length(rows, slots=0)
