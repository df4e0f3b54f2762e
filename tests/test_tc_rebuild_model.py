"""Host model of the lane exchanges that turn a warp's tensor-core product into
the residue rebuild's column sums (crt_sums_tc in the CUDA library).

The rebuild of the residue form needs, for each entry, the limb column sums
acc[k] = sum_l R_l w_l[k] (R_l its residue bytes, w_l[k] the 32-bit limbs of
the rebuild weights). Taken byte by byte this is a product of the entries'
residues with the weights' bytes, which the library forms with mma.sync
m16n8k16 (two m16 groups of 16 entries per warp, tiles of 8 byte positions).
Its accumulator fragments follow the PTX ISA's layout for m16n8k16 with FP32
accumulators: lane (g, tig) = (lane / 4, lane % 4) holds rows g and g + 8,
columns 2 tig and 2 tig + 1 of each 16 x 8 tile. The lanes then combine pairs
of byte positions into limbs with their xor-1 partner and swap limbs of the
other parity with their xor-2 partner.

This test restates those steps on the host with exact integers and checks
that every lane ends with the exact column sums of its own entry (row
16 (tig & 1) + g + 8 (tig >> 1) of the warp's 32). It pins the index algebra;
the GPU tests pin the device results bit for bit against the scalar sums.
"""
import numpy as np
import pytest


def _entry(lane):
    tig = lane & 3
    return 16 * (tig & 1) + (lane >> 2) + 8 * (tig >> 1)


def _warp_sums(R, w):
    """R: 32 x NM residue bytes; w: NM x L 32-bit limbs. Returns acc[lane][k]."""
    NM, L = w.shape
    NJ = L // 2
    # the weights' bytes: byte position p of weight l is byte p % 4 of limb p // 4
    Wb = np.zeros((NM, 4 * L), dtype=np.int64)
    for p in range(4 * L):
        Wb[:, p] = (w[:, p // 4] >> (8 * (p % 4))) & 255
    # D[G][j]: the 16 x 8 accumulator of group G, tile j (exact integers)
    D = [[R[16 * G:16 * G + 16, :].astype(np.int64) @ Wb[:, 8 * j:8 * j + 8] for j in range(NJ)] for G in range(2)]
    for G in range(2):
        for j in range(NJ):
            assert D[G][j].max() < 2 ** 22          # exact in the FP32 accumulation
    # fragments: c[lane][G][j] = (D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1])
    frag = {}
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        frag[lane] = [[(D[G][j][g, 2 * t], D[G][j][g, 2 * t + 1], D[G][j][g + 8, 2 * t], D[G][j][g + 8, 2 * t + 1])
                       for j in range(NJ)] for G in range(2)]
    acc = np.zeros((32, L), dtype=object)
    for j in range(NJ):
        # two byte positions in 32 bits, then the partner's two above them
        own = {lane: [[frag[lane][G][j][2 * hr] + (frag[lane][G][j][2 * hr + 1] << 8) for hr in range(2)]
                      for G in range(2)] for lane in range(32)}
        v = {}
        for lane in range(32):
            bh = lane & 1
            v[lane] = [[None, None], [None, None]]
            for G in range(2):
                for hr in range(2):
                    a, b = own[lane][G][hr], own[lane ^ 1][G][hr]
                    assert a < 2 ** 32 and b < 2 ** 32
                    lo, hi = (b, a) if bh else (a, b)
                    v[lane][G][hr] = lo + (hi << 16)
        send = {}
        mine = {}
        for lane in range(32):
            t = lane & 3
            gm, hm = t & 1, t >> 1
            mine[lane] = v[lane][gm][hm]
            send[lane] = v[lane][gm][1 - hm]
        for lane in range(32):
            got = send[lane ^ 2]
            odd = (lane & 3) >> 1
            acc[lane, 2 * j] = got if odd else mine[lane]
            acc[lane, 2 * j + 1] = mine[lane] if odd else got
    return acc


@pytest.mark.parametrize("NM,L", [(16, 4), (32, 8), (48, 12)])
def test_lane_exchange_gives_each_lane_its_entry_sums(NM, L):
    rng = np.random.default_rng(NM + L)
    R = rng.integers(0, 256, (32, NM))
    w = rng.integers(0, 2 ** 32, (NM, L), dtype=np.int64)
    acc = _warp_sums(R, w)
    for lane in range(32):
        e = _entry(lane)
        for k in range(L):
            want = sum(int(R[e, l]) * int(w[l, k]) for l in range(NM))
            assert acc[lane, k] == want, (lane, k)


def test_every_entry_has_one_lane():
    assert sorted(_entry(lane) for lane in range(32)) == list(range(32))


def test_extreme_bytes_stay_exact():
    # all residues and weight bytes at 255: the largest column sums
    NM, L = 48, 12
    R = np.full((32, NM), 255)
    w = np.full((NM, L), 2 ** 32 - 1, dtype=np.int64)
    acc = _warp_sums(R, w)
    want = NM * 255 * (2 ** 32 - 1)
    assert all(acc[lane, k] == want for lane in range(32) for k in range(L))
