"""The balanced phase-B plan of the loop's default launch shape
(mvct_phase_b_plan, host arithmetic in the library, CPU only): every tile's
subset views are dealt to its view groups exactly once, every non-owner group
has its own partial-tile slot inside the plan's buffers, one block is left
without an item (the Phi_n reducer), and with block b on SM b mod num_sms the
busiest SM holds fewer tile-views than with two groups per tile."""
import numpy as np
import pytest

SMS = 152


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


def group_views(vs, h, ht):
    return list(range(h, vs, ht))


def check_plan(items, idle, n_tiles, vs, cap, grid, sms):
    assert items.shape == (grid, 4)
    assert 0 <= idle < grid and items[idle, 0] == -1
    used = items[items[:, 0] >= 0]
    assert len(used) == grid - 1                      # exactly one block without an item
    slots = set()
    for t in range(n_tiles):
        mine = used[used[:, 0] == t]
        assert len(mine) >= 1
        ht = int(mine[0, 2])
        assert 1 <= ht <= min(cap, vs)
        assert np.all(mine[:, 2] == ht) and np.all(mine[:, 3] == mine[0, 3])
        assert sorted(mine[:, 1].tolist()) == list(range(ht))   # each group once
        views = sorted(v for h in range(ht) for v in group_views(vs, h, ht))
        assert views == list(range(vs))                         # each view once
        for h in range(ht - 1):                                  # non-owners publish
            s = int(mine[0, 3]) + h
            assert s not in slots
            slots.add(s)
    assert all(0 <= s < n_tiles * cap for s in slots)
    # tile-views per SM (block b on SM b mod sms)
    load = np.zeros(sms)
    for b in range(grid):
        if items[b, 0] >= 0:
            load[b % sms] += len(group_views(vs, int(items[b, 1]), int(items[b, 2])))
    return load


def test_plan_of_the_512_workload(mvct):
    """512^2 (256 tiles), 40 views per subset, 4 blocks on each of 152 SMs."""
    n_tiles, vs, cap, grid = 256, 40, 8, 4 * SMS
    out = mvct.phase_b_plan(n_tiles, vs, cap, grid, SMS)
    assert out is not None
    items, idle = out
    load = check_plan(items, idle, n_tiles, vs, cap, grid, SMS)
    assert load.sum() == n_tiles * vs
    # every SM: three half-tile items (20 views) and at most one small item
    assert load.max() <= 3 * 20 + 8 and load.min() >= 3 * 20
    # two groups per tile on the same blocks: 512 items of 20 views, items
    # lb, lb + grid, ... -> some SM holds four of them
    uniform = np.zeros(SMS)
    for item in range(2 * n_tiles):
        uniform[item % grid % SMS] += 20
    assert uniform.max() == 80 and load.max() < uniform.max()


@pytest.mark.parametrize("n_tiles,vs,cap,grid,sms", [
    (256, 20, 8, 4 * SMS, SMS),     # 20 views per subset
    (256, 40, 8, 3 * SMS, SMS + 8),  # not a whole number of blocks per SM -> check below
    (300, 40, 8, 4 * SMS, SMS),
    (250, 40, 8, 4 * SMS, SMS),
])
def test_plan_invariants_when_it_exists(mvct, n_tiles, vs, cap, grid, sms):
    out = mvct.phase_b_plan(n_tiles, vs, cap, grid, sms)
    if grid % sms:
        assert out is None
        return
    assert out is not None
    items, idle = out
    load = check_plan(items, idle, n_tiles, vs, cap, grid, sms)
    assert load.sum() == n_tiles * vs


@pytest.mark.parametrize("n_tiles,vs,cap,grid,sms", [
    (64, 20, 8, 4 * SMS, SMS),      # 256^2: too few tiles for three half-tile items per SM
    (1024, 40, 8, 4 * SMS, SMS),    # 1024^2: too many tiles for one small item per SM
    (240, 40, 8, 4 * SMS, SMS),     # 12 tiles left: too few for 151 items of <= 8 groups
    (384, 40, 8, 4 * SMS, SMS),     # 156 tiles left: more than the 151 small items
    (256, 40, 8, SMS, SMS),         # one block per SM
    (256, 40, 8, 4 * SMS - 1, SMS), # not a whole number of blocks per SM
    (256, 1, 1, 4 * SMS, SMS),      # one view per subset: a tile cannot be split
])
def test_no_plan_outside_its_sizes(mvct, n_tiles, vs, cap, grid, sms):
    assert mvct.phase_b_plan(n_tiles, vs, cap, grid, sms) is None


def test_bad_arguments_rejected(mvct):
    with pytest.raises(mvct.MvctError):
        mvct.phase_b_plan(0, 40, 8, 608, 152)
    with pytest.raises(mvct.MvctError):
        mvct.phase_b_plan(256, 40, 8, 608, 0)
