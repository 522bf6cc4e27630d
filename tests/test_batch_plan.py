"""The batch schedule (host logic behind mlgmres_solve_batch), through the C
ABI with no GPU: CTA groups in proportion to the systems' cost."""
import math

import pytest

from paper_2103_10975_gb300 import batch_plan, MLGMRESError
from synthetic import batched_sides


def cost(dim, n):
    return float(n ** dim) * n * n


def makespan(dim, sides, gc, go):
    load = [0.0] * len(gc)
    for n, g in zip(sides, go):
        load[g] += cost(dim, n) / gc[g]
    return max(load)


def check_valid(sides, ctas, gc, go):
    assert 1 <= len(gc) <= ctas and sum(gc) <= ctas and min(gc) >= 1
    assert len(go) == len(sides) and all(0 <= g < len(gc) for g in go)


def test_batch_workload_512_instances_on_152_ctas():
    sides = batched_sides(512)
    gc, go = batch_plan(2, sides, 152)
    check_valid(sides, 152, gc, go)
    total = sum(cost(2, n) for n in sides)
    ideal = total / 152
    biggest = max(cost(2, n) for n in sides)
    # with one CTA per system the launch could not end before the largest
    # system's cost, a third above the ideal share
    assert biggest > 1.3 * ideal
    ms = makespan(2, sides, gc, go)
    assert ms <= 1.05 * ideal, (ms / ideal)
    # the largest systems have groups of several CTAs
    big = max(range(len(sides)), key=lambda i: sides[i])
    assert gc[go[big]] == math.ceil(cost(2, sides[big]) / ideal) == 2


def test_single_system_takes_ctas_by_size():
    gc, go = batch_plan(2, [256], 152)
    assert gc == [128] and go == [0]       # 65536 points / 512 per CTA
    gc, go = batch_plan(2, [1024], 152)
    assert gc == [152] and go == [0]
    gc, go = batch_plan(3, [8], 152)
    assert gc == [1] and go == [0]         # 512 points: one CTA


def test_equal_systems_get_one_cta_each():
    gc, go = batch_plan(2, [100] * 40, 40)
    assert gc == [1] * 40 and sorted(go) == list(range(40))
    gc, go = batch_plan(2, [100] * 80, 40)
    assert gc == [1] * 40 and all(go.count(g) == 2 for g in range(40))


def test_few_large_systems_share_all_ctas():
    gc, go = batch_plan(2, [512, 512, 512], 152)
    check_valid([512] * 3, 152, gc, go)
    assert sorted(go) == [0, 1, 2] and sum(gc) >= 150


def test_3d_and_deterministic():
    sides = [12, 40, 64, 96, 20, 20, 33]
    a = batch_plan(3, sides, 16)
    b = batch_plan(3, sides, 16)
    assert a == b
    check_valid(sides, 16, *a)


@pytest.mark.parametrize("args", [(4, [10], 8), (2, [], 8), (2, [10], 0), (2, [0], 8)])
def test_bad_arguments(args):
    with pytest.raises((MLGMRESError, ValueError)):
        batch_plan(*args)
