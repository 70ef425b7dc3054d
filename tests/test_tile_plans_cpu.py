"""The tile-plan table (ot_set_tile_plan / ot_get_tile_plan): host logic only, no GPU needed."""
import pytest

P = pytest.importorskip("paper_2609_33814_b300")


def test_plan_table_set_get_reset_and_validation():
    base = P.get_tile_plan(2, "mufu")
    assert base == (4, 16)                       # built-in: the measured choice on B300
    assert P.get_tile_plan(3, "mufu") == (4, 8)
    assert P.get_tile_plan(2, "comp") == (1, 8)
    P.set_tile_plan(2, "mufu", 2, 8)
    assert P.get_tile_plan(2, "mufu") == (2, 8)
    assert P.get_tile_plan(3, "mufu") == (4, 8)  # other entries untouched
    P.set_tile_plan(2, "mufu", 0, 0)
    assert P.get_tile_plan(2, "mufu") == base
    for bad in ((2, "mufu", 3, 16), (2, "mufu", 8, 16), (2, "comp", 2, 16), (4, "mufu", 2, 16), (2, "fp64", 4, 8), (2, "comp", 1, 16)):
        with pytest.raises(P.OTError) as e:
            P.set_tile_plan(*bad)
        assert e.value.status == P.OT_EINVAL


def test_builtin_plans_match_the_shipped_autotuner_table():
    """The built-in table is the autotuner's measured choice (tile_plans.txt in the package)."""
    import os
    path = os.path.join(os.path.dirname(P.__file__), "tile_plans.txt")
    names = {v: k for k, v in P.PRECISIONS.items()}
    for line in open(path):
        line = line.split("#")[0].split()
        if len(line) == 4:
            d, prec, R, ch = map(int, line)
            assert P.get_tile_plan(d, names[prec]) == (R, ch), line
