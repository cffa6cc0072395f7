"""CPU checks of the strip operator's launch plan (libhmc's hmc_strip_plan, host only): every block
of the fused A = D D^dagger launch is accounted for, the right-hand sides with the longer time chunks
go first, and the chosen chunk counts are the best uniform-or-adjacent split under the documented
cost model (a block costs its chunk length + 1.5 slice steps, blocks are dealt greedily to the
resident slots in launch order)."""

import heapq
import os

import pytest

from paper_2204_14241_gb300 import hmc


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(hmc.LIB_PATH):
        from paper_2204_14241_gb300 import build
        build.build()


def makespan(Nt, nch, order, nstrip, slots):
    free = [0.0] * slots
    heapq.heapify(free)
    end = 0.0
    for k in order:
        nc = nch[k]
        for c in range(nc):
            length = (c + 1) * Nt // nc - c * Nt // nc + 1.5
            for _ in range(nstrip):
                t = heapq.heappop(free) + length
                heapq.heappush(free, t)
                end = max(end, t)
    return end


def test_plan_of_the_benchmark_launch():
    # 80x80x160 with 8 RHS on 152 SMs, one block per SM: four right-hand sides in 7 time chunks, four
    # in 8, five strips each: the 300-block grid the ncu capture of the operator shows
    nch, order, nblk = hmc.strip_plan(80, 160, 8, 152)
    assert sorted(nch) == [7] * 4 + [8] * 4
    assert nblk == 300


@pytest.mark.parametrize("L", [16, 48, 80])
@pytest.mark.parametrize("Nt", [1, 2, 7, 48, 160])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 64])
@pytest.mark.parametrize("slots", [1, 152, 456])
def test_plan_invariants(L, Nt, nrhs, slots):
    nstrip = L // 16
    nch, order, nblk = hmc.strip_plan(L, Nt, nrhs, slots)
    assert sorted(order) == list(range(nrhs))
    assert nblk == sum(nch) * nstrip
    assert all(1 <= c <= Nt for c in nch)
    assert max(nch) - min(nch) <= 1
    # longer chunks (fewer of them) are launched first
    along = [nch[k] for k in order]
    assert along == sorted(along)
    # no uniform split n (or n, n + 1 mixed the same way) that the plan considers ends earlier
    best = makespan(Nt, nch, order, nstrip, slots)
    nmax = max(1, min(Nt, 8 * slots // (nrhs * nstrip)))
    for n in range(1, nmax + 1):
        for m in range(nrhs + 1):
            if m > 0 and n + 1 > Nt:
                break
            cand = [n if i < nrhs - m else n + 1 for i in range(nrhs)]
            assert best <= makespan(Nt, cand, list(range(nrhs)), nstrip, slots) + 1e-9


@pytest.mark.parametrize("args", [(20, 48, 8, 152), (96, 48, 8, 152), (16, 0, 8, 152), (16, 48, 0, 152),
                                  (16, 48, 65, 152), (16, 48, 8, 0)])
def test_plan_rejects_bad_arguments(args):
    with pytest.raises(hmc.HmcError):
        hmc.strip_plan(*args)
