"""The host plan of a batch (``vt_batch_plan``), which needs no GPU: one grid
per set, laid end to end in one global cell array, and the checks that keep
every set's grid and the whole array within the kernels' index range."""
import pytest

import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import _lib as L


def test_each_set_gets_its_own_grid_end_to_end():
    off = [0, 1000, 1000, 9000, 9001]
    p = vt.Params()
    plan, cells = vt.batch_plan(off, p, grid_res=[0, 0, 5, 0])
    G = [plan[i].G for i in range(4)]
    assert G == [vt.grid_resolution(p, 1000), 1, 5, vt.grid_resolution(p, 1)]
    base = 0
    for i in range(4):
        assert plan[i].cell_base == base
        assert plan[i].pt_begin == off[i] and plan[i].npts == off[i + 1] - off[i]
        assert plan[i].periodic == 0
        base += G[i] ** 3
    assert cells == base


def test_the_box_and_periodicity_reach_every_set():
    p = vt.Params(box_lo=(-2.0, 0.5, 3.0), box_hi=(-1.0, 2.0, 4.0))
    plan, _ = vt.batch_plan([0, 5000, 6000], p)
    for i in range(2):
        assert tuple(plan[i].lo) == (-2.0, 0.5, 3.0) and tuple(plan[i].hi) == (-1.0, 2.0, 4.0)
        G = plan[i].G
        assert plan[i].cw[1] == pytest.approx(1.5 / G)
    plan, _ = vt.batch_plan([0, 5000, 6000], vt.Params(periodic=True))
    assert [plan[i].periodic for i in range(2)] == [1, 1]


@pytest.mark.parametrize("off, grid_res", [
    ([1, 10], None),                 # offsets must start at 0
    ([0, 10, 5], None),              # and never decrease
    ([0, 10], [1025]),               # a set's grid above 1024 per axis
    ([0, 10, 20], [1024, 1024]),     # 2 x 1024^3 cells: beyond the int32 index range
])
def test_bad_plans_are_refused(off, grid_res):
    with pytest.raises(L.VtError) as e:
        vt.batch_plan(off, vt.Params(), grid_res=grid_res)
    assert e.value.code == L.VT_ERR_INVALID_ARG


def test_a_batch_needs_a_set():
    with pytest.raises(ValueError):
        vt.batch_plan([0], vt.Params())
