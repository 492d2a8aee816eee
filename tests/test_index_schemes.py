"""CPU emulation of the index arithmetic of the fused MTTKRP partial sums of the
tensor-core replica CP-ALS (no GPU).

The GEMM epilogue reduces every block of 32 consecutive output rows m of one
replica (m = outer * Q + inner, Q^2 rows) against the weights of the inner
index.  When 32 divides Q a block lies inside one outer index and writes one
partial; otherwise a block may cross from one outer index to the next and
writes two segment sums (segment 0: the rows of the outer index the block
starts in; segment 1: the rows of the next one).  The solve then forms each
outer index's MTTKRP row from the partials of the blocks that hold its rows.
These tests model both sides with the same integer arithmetic as the kernels
and check, for every Q the tensor-core path takes, that every row of every
outer index is counted exactly once and with the weight of its own inner
index (a block spans at most two outer indices once Q >= 32).
"""
import pytest


def epilogue_partials(Q):
    """{(block, segment): [(row, weight index), ...]} as the epilogue writes them."""
    M = Q * Q
    part = {}
    if Q % 32 == 0:
        for j in range(M // 32):
            mb = 32 * j
            b0 = mb % Q
            part[(j, 0)] = [(mb + i, b0 + i) for i in range(32)]
        return part
    nblk = -(-M // 32)
    for j in range(nblk):
        mb = 32 * j
        b0 = mb % Q
        nv = min(32, M - mb)
        cut = Q - b0
        if cut >= 32 and nv == 32:           # the one-segment fast path
            seg0, seg1 = [(mb + i, b0 + i) for i in range(32)], []
        else:
            n0 = min(cut, nv)
            seg0 = [(mb + i, b0 + i) for i in range(n0)]
            seg1 = [(mb + i, b0 + i - Q) for i in range(n0, nv)]
        part[(j, 0)], part[(j, 1)] = seg0, seg1
    return part


def solve_rows(Q, part):
    """{outer: [(row, weight index), ...]} as the solve sums the partials."""
    out = {}
    for q in range(Q):
        terms = []
        if Q % 32 == 0:
            for s in range(Q // 32):        # Q / 32 partials per outer index
                terms += part[(q * (Q // 32) + s, 0)]
        else:
            first, last = q * Q, q * Q + Q - 1
            for j in range(first // 32, last // 32 + 1):
                sgm = 0 if (32 * j) // Q == q else 1
                terms += part[(j, sgm)]
        out[q] = terms
    return out


@pytest.mark.parametrize("Q", list(range(32, 257)))
def test_every_row_summed_once_with_its_own_weight(Q):
    part = epilogue_partials(Q)
    rows = solve_rows(Q, part)
    for q in range(Q):
        assert sorted(rows[q]) == [(q * Q + b, b) for b in range(Q)], q
    # nothing written is left unread, nothing is read twice
    used = sorted(t for q in range(Q) for t in rows[q])
    written = sorted(t for v in part.values() for t in v)
    assert used == written == [(m, m % Q) for m in range(Q * Q)]


@pytest.mark.parametrize("Q", [33, 40, 100, 200, 255])
def test_a_block_spans_at_most_two_outer_indices(Q):
    for j in range(-(-Q * Q // 32)):
        outers = {m // Q for m in range(32 * j, min(32 * j + 32, Q * Q))}
        assert len(outers) <= 2
        assert max(outers) - min(outers) <= 1
