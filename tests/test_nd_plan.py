"""Host logic of the nested-dissection coarse LU (no GPU needed): the plan msfv_setup
builds for a coarse grid -- separator tree, index lists, child maps -- checked on many grid
shapes, and its size on the 16^3 coarse grid of the 128^3, c = 8 workload."""
import pytest

from paper_1707_07598_gb300 import build as B
from paper_1707_07598_gb300 import msfv as M


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


SHAPES = [(2, 1), (3, 3), (9, 7), (64, 64), (320 // 4, 256 // 4), (2, 2, 2), (4, 4, 4),
          (5, 3, 2), (8, 6, 4), (16, 16, 16), (17, 17, 17), (24, 16, 16), (12, 10, 6),
          (1, 1, 9), (24, 24, 24)]


@pytest.mark.parametrize("nc", SHAPES)
def test_plan_is_structurally_sound(lib, nc):
    """Every coarse node is the pivot of exactly one front and every child's update nodes
    are in its parent's index list (the two facts the multifrontal gathers rely on)."""
    p = M.nd_analyse(nc)
    assert p["ok"] == 1
    n = 1
    for v in nc:
        n *= v
    assert 1 <= p["fronts"] <= n and p["max_front"] >= 1


def test_single_front_is_a_dense_lu(lib):
    """A grid small enough to be one leaf is one dense front: 2/3 n^3 flops."""
    p = M.nd_analyse((2, 2, 2))
    assert p["fronts"] == 1 and p["levels"] == 1 and p["max_front"] == 8
    assert p["update_rows"] == 0
    assert abs(p["factor_flops"] - 2.0 / 3.0 * 8 ** 3) <= 1


def test_separators_cut_the_work_below_the_band(lib):
    """On the 16^3 coarse grid the plan has 531 fronts on 10 levels, the root front is the
    16 x 16 separator plane with its largest child front 384 wide, and the factorisation
    costs far less than a banded LU of the same matrix (half bandwidth 16^2 + 16 + 1)."""
    p = M.nd_analyse((16, 16, 16))
    assert p["fronts"] == 531 and p["levels"] == 10 and p["max_front"] == 384
    n, b = 16 ** 3, 16 * 16 + 16 + 1
    banded = 2.0 * n * b * b          # LU of a band of half width b (both triangles)
    assert p["factor_flops"] < 0.35 * banded


def test_rejects_bad_shapes(lib):
    with pytest.raises(M.MSFVError):
        M.nd_analyse((0, 4))
    with pytest.raises(M.MSFVError):
        M.nd_analyse((4, 4, 4, 4)[:1])
