"""The batched kernel's work list (host logic, no GPU): every (request, step) range appears
once, the ranges tile [0, total) in list order, each request's prep, element and gather
ranges come in that order (an item only ever depends on earlier items, which is what makes
the kernel's waits end), and the list is the wave pipeline P(s), E(s-1), G(s-2)."""
import numpy as np
import pytest

from paper_2109_01158_gb300 import fem


def _waves(prep, elem, resident):
    wb, acc = [0], 0
    for k in range(len(prep)):
        acc += 2 * prep[k] + elem[k]
        if acc >= 4 * resident or k == len(prep) - 1:
            wb.append(k + 1)
            acc = 0
    return wb


@pytest.mark.parametrize("seed", range(6))
def test_plan_tiles_the_items_and_orders_the_steps(seed):
    fem.load_library()
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    prep = [int(x) for x in rng.integers(1, 400, n)]
    elem = [int(x) for x in rng.integers(1, 3000, n)]
    resident = int(rng.choice([1, 7, 152, 304]))
    ranges, total = fem.batch_plan(prep, elem, resident)
    assert len(ranges) == 3 * n and total == sum(2 * p + e for p, e in zip(prep, elem))
    # each (request, step) once; the ranges are contiguous in list order and cover [0, total)
    assert sorted((k, s) for _, k, s in ranges) == [(k, s) for k in range(n) for s in range(3)]
    pos = 0
    start = {}
    for st, k, s in ranges:
        assert st == pos
        start[(k, s)] = st
        pos += elem[k] if s == 1 else prep[k]
    assert pos == total
    # a request's element tiles follow all its prep tiles, its gather tiles all its element tiles
    for k in range(n):
        assert start[(k, 0)] + prep[k] <= start[(k, 1)]
        assert start[(k, 1)] + elem[k] <= start[(k, 2)]
    # the wave pipeline
    wb = _waves(prep, elem, resident)
    nw = len(wb) - 1
    expect = []
    for s in range(nw + 2):
        for wave, step in ((s, 0), (s - 1, 1), (s - 2, 2)):
            if 0 <= wave < nw:
                expect += [(k, step) for k in range(wb[wave], wb[wave + 1])]
    assert [(k, s) for _, k, s in ranges] == expect


def test_plan_single_request_is_prep_element_gather():
    fem.load_library()
    ranges, total = fem.batch_plan([3], [10], 152)
    assert ranges == [(0, 0, 0), (3, 0, 1), (13, 0, 2)] and total == 16


def test_plan_rejects_bad_arguments():
    fem.load_library()
    with pytest.raises(fem.FEError):
        fem.batch_plan([0], [5], 152)
    with pytest.raises(fem.FEError):
        fem.batch_plan([2], [5], 0)
    assert fem.batch_plan([], [], 152) == ([], 0)
