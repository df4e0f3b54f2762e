"""Host logic of the dataflow solve (runs on CPU): the task list that the
launch's CTAs claim in order. Forward progress of the launch rests on two
properties checked here for many orders: every task comes after the tasks it
reads (tiles of higher block subdiagonals, and the tile's earlier helpers),
and the owner and helpers of a tile together multiply each of its
subdiagonals exactly once (the block form of Alg. 3's update products)."""
import numpy as np
import pytest

from paper_2203_10879_gb300 import _binding as B


@pytest.fixture(scope="module")
def lib():
    return B.lib()


def _decode(t):
    t = int(t)
    J, I = t & 0xFFFF, (t >> 16) & 0xFFFF
    if t >> 63:
        return ("H", I, J, (t >> 32) & 0xFFF, (t >> 44) & 0xFFF, (t >> 56) & 0x7F)
    return ("S", I, J, (t >> 32) & 0xFFFF, (t >> 48) & 0xFFF)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 64, 100, 257, 700, 1000, 2048, 4096])
def test_plan_orders_inputs_first_and_covers_each_product_once(lib, n):
    tasks = [_decode(t) for t in B.schur_refine_solve_plan(n)]
    NB = (n + 31) // 32
    solve_at, helper_at = {}, {}
    for k, t in enumerate(tasks):
        if t[0] == "S":
            assert (t[1], t[2]) not in solve_at
            solve_at[(t[1], t[2])] = k
        else:
            helper_at[(t[1], t[2], t[5])] = k
    assert len(solve_at) == NB * (NB + 1) // 2

    def inputs(I, J, d):
        out = []
        if J + d < NB:
            out.append(solve_at[(J + d, J)])   # L(J+d, J)
        if I - d >= 0:
            out.append(solve_at[(I, I - d)])   # L(I, I-d)
        return out

    for k, t in enumerate(tasks):
        I, J = t[1], t[2]
        D = I - J
        assert 0 <= J <= I < NB
        if t[0] == "H":
            lo, hi, h = t[3], t[4], t[5]
            assert D < lo <= hi < NB
            assert all(x < k for d in range(lo, hi + 1) for x in inputs(I, J, d))
            if h:
                assert helper_at[(I, J, h - 1)] < k
        else:
            nhelp, own_hi = t[3], t[4]
            top = max(NB - 1 - J, I)
            done = list(range(D + 1, own_hi + 1))
            assert all(x < k for d in done for x in inputs(I, J, d))
            for h in range(nhelp):
                hk = helper_at[(I, J, h)]
                assert hk < k
                done += list(range(tasks[hk][3], tasks[hk][4] + 1))
            assert sorted(done) == list(range(D + 1, top + 1)), (I, J)


def test_plan_rejects_bad_arguments(lib):
    import ctypes
    cnt = ctypes.c_longlong(0)
    assert lib.schur_refine_solve_plan(0, None, 0, ctypes.byref(cnt)) == B.SR_ERR_INVALID_ARG
    assert lib.schur_refine_solve_plan(64, None, 0, None) == B.SR_ERR_INVALID_ARG
