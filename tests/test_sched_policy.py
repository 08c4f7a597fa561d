"""Host-only scheduling policy of the map server (no GPU needed):
admission under the device-memory budget and slice planning."""
import pytest


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def test_admission_first_fit_under_budget(rs):
    # 100 fits, 500 never fits the budget (caller fails it), 50 fits
    assert rs.sched_admit([(100, 0), (500, 0), (50, 0)], 0, 400, 0, 8) == [1, 0, 1]
    # bytes already in use count against the budget
    assert rs.sched_admit([(100, 0), (50, 0)], 320, 400, 0, 8) == [0, 1]
    # the slot limit stops admission
    assert rs.sched_admit([(1, 0)] * 5, 0, 400, 6, 8) == [1, 1, 0, 0, 0]


def test_admission_old_request_blocks_passing(rs):
    # a request passed max_skips times keeps later ones from overtaking it
    assert rs.sched_admit([(300, 4), (50, 0)], 200, 400, 0, 8, max_skips=4) == [0, 0]
    assert rs.sched_admit([(300, 3), (50, 0)], 200, 400, 0, 8, max_skips=4) == [0, 1]


def test_plan_shortest_remaining_first_and_budget(rs):
    items = [(1, 100, 10.0), (2, 5, 10.0), (3, 50, 100.0)]
    # remaining work 1000, 50, 5000: item 2 finishes, item 1 gets the rest
    assert rs.sched_plan(items, budget=500.0) == [45, 5, 0]
    # FIFO: arrival order
    assert rs.sched_plan(items, budget=500.0, policy=rs.SCHED_FIFO) == [50, 0, 0]
    # unlimited budget: everything in one slice
    assert rs.sched_plan(items, budget=float("inf")) == [100, 5, 50]


def test_plan_always_progresses_and_respects_map_limit(rs):
    # a tile larger than the whole budget still gets one tile
    assert rs.sched_plan([(1, 10, 1e9)], budget=1.0) == [1]
    items = [(k, 3, 1.0) for k in range(10)]
    got = rs.sched_plan(items, budget=1e9, max_maps=4)
    assert sum(1 for v in got if v) == 4 and all(v in (0, 3) for v in got)
    # finished requests get nothing
    assert rs.sched_plan([(1, 0, 1.0), (2, 2, 1.0)], budget=10.0) == [0, 2]


def test_plan_starvation_free_under_srpt_with_budget(rs):
    # a long request keeps progressing while short ones come and go
    long = [1, 1000, 10.0]
    done = 0
    for step in range(50):
        short = [(100 + step, 2, 10.0)]
        take = rs.sched_plan([tuple(long)] + short, budget=100.0)
        long[1] -= take[0]
        done += take[0]
    assert done > 0 and long[1] < 1000
