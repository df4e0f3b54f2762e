"""Host logic of the residue form of the emulated products (CPU only): the
table the library builds for the Chinese remainder rebuild, checked against
the definition with exact Python integers. The moduli are the N largest
pairwise coprime integers <= 256 taken greedily; M is their product; weight l
is M_l (M_l^-1 mod m_l) with M_l = M / m_l, so that it is 1 modulo m_l and 0
modulo every other modulus; the library stores M and the weights times
2^sigma with M 2^sigma's top bit at 32 limbs - 1; t is the largest integer
with K 2^(2t) < M / 2, the condition under which every rebuilt integer
product of t-bit operands over K terms is exact."""
from math import gcd, prod

import pytest

from paper_2203_10879_gb300 import _binding as B


def _moduli(N):
    ms, m = [], 256
    while len(ms) < N:
        if all(gcd(m, x) == 1 for x in ms):
            ms.append(m)
        m -= 1
    return ms


@pytest.mark.parametrize("N,limbs", [(1, 4), (8, 4), (15, 4), (16, 4), (20, 8), (31, 8), (32, 8), (34, 8),
                                     (40, 12), (48, 12), (49, 12)])
def test_table_matches_definition(N, limbs):
    for K in (1, 64, 1000, 4096, 16384):
        s, mods, w, Ms, sigma, t = B.schur_refine_crt_info(N, limbs, K)
        assert s == B.SR_OK
        assert mods == _moduli(N)
        M = prod(mods)
        assert Ms == M << sigma and Ms.bit_length() == 32 * limbs
        for l, m in enumerate(mods):
            assert w[l] % (1 << sigma) == 0
            wl = w[l] >> sigma
            assert 0 < wl < M
            for k, mk in enumerate(mods):
                assert wl % mk == (1 if k == l else 0)
        assert K * 2 ** (2 * t) * 2 < M <= K * 2 ** (2 * t + 2) * 2


def test_table_rejects_what_does_not_fit():
    assert B.schur_refine_crt_info(17, 4, 64)[0] == B.SR_ERR_INVALID_ARG   # M >= 2^128
    assert B.schur_refine_crt_info(0, 4, 64)[0] == B.SR_ERR_INVALID_ARG
    assert B.schur_refine_crt_info(35, 8, 64)[0] == B.SR_ERR_INVALID_ARG   # M >= 2^256
    assert B.schur_refine_crt_info(50, 12, 64)[0] == B.SR_ERR_INVALID_ARG  # no 50th coprime modulus <= 256
    assert B.schur_refine_crt_info(8, 5, 64)[0] == B.SR_ERR_INVALID_ARG
    assert B.schur_refine_crt_info(8, 4, 0)[0] == B.SR_ERR_INVALID_ARG


def test_sixteen_moduli_give_56_bits_at_4096():
    # the default of the FP64 form: 56-bit operands where 7 digits hold 55
    assert B.schur_refine_crt_info(16, 4, 4096)[5] == 56
    assert B.schur_refine_crt_info(32, 8, 2048)[5] == 114


def test_greedy_list_has_49_moduli():
    # the greedy rule finds no 50th integer <= 256 coprime to all before it
    assert len(_moduli(49)) == 49 and min(_moduli(49)) == 29
    taken = _moduli(49)
    assert all(any(gcd(m, x) > 1 for x in taken) for m in range(2, 257) if m not in taken)


def test_forty_eight_moduli_give_triple_double_operands():
    # the triple-double form: 48 moduli, M < 2^338, operands of t >= 159 bits
    # (three doubles) up to K = 8192
    s, mods, w, Ms, sigma, t = B.schur_refine_crt_info(48, 12, 4096)
    assert s == B.SR_OK and t == 162 and prod(mods).bit_length() == 338
    assert B.schur_refine_crt_info(48, 12, 8192)[5] >= 159


def test_six_double_halves_sit_at_fixed_word_offsets():
    # the six-double rebuild places HH at 2t and HL + LH at t bits: 5 and 2 whole
    # words plus a bit shift for t in [160, 174], the range the split and the
    # rebuild accept; every inner length up to the workspace's limit lands there,
    # and each half-product still rebuilds exactly (K 2^(2t) < M / 2)
    for K in (1, 2, 64, 1000, 1024, 4096, 8192):
        s, mods, w, Ms, sigma, t = B.schur_refine_crt_info(48, 12, K)
        assert s == B.SR_OK
        assert 160 <= t <= 174, (K, t)
        assert (2 * t) >> 6 == 5 and t >> 6 == 2
        M = 1
        for m in mods:
            M *= m
        assert K * 2 ** (2 * t) < M // 2
