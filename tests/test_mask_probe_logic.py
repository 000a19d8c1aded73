"""CPU checks of the refinement's mask-probe addressing (no GPU needed).

From padded dimension 12 each 32-point sub-tile of the refinement carries a
table of 16 x 8 words: word k * 8 + l holds bit j set iff point j's 3-bit
code (the top three bits of its 7-bit code) in dimension k is <= l. A lane
holding point p keeps one byte per dimension, (k mod 8) * 32 + 4 * l_k(p),
and forms the address of word (k, l_k(p)) by replacing the low byte of the
table half's 256-byte-aligned address (dimensions 0-7 in the first 256 bytes,
8-15 in the second) with that byte (a byte permute, selector 0x3214 + k mod
4). ANDing the d words gives the q's that pass the 3-bit test against p.
This file restates that layout and addressing and checks the result against
the definition on random codes, with padding points (code 127 everywhere)
and the dimensions past d (code 0)."""
import numpy as np
import pytest


def byte_perm(x, y, s):
    """The byte permute as documented: result byte i is byte (s >> 4i) & 7
    of the 8 bytes x0..x3, y0..y3."""
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(b[(s >> (4 * i)) & 7] << (8 * i) for i in range(4))


def table(codes):
    """codes: 32 x 16 array of 7-bit codes of one sub-tile -> 128 words."""
    c3 = codes >> 4
    t = np.zeros(128, dtype=np.uint64)
    for k in range(16):
        for lvl in range(8):
            bits = 0
            for j in range(32):
                if lvl == 7 or c3[j, k] <= lvl:
                    bits |= 1 << j
            t[k * 8 + lvl] = bits
    return t


def offsets(pcode):
    """p's four offset words: byte k % 4 of word k // 4."""
    words = [0, 0, 0, 0]
    for k in range(16):
        words[k // 4] |= ((k % 8) * 32 + 4 * int(pcode[k] >> 4)) << (8 * (k % 4))
    return words


def probe(tab, base, pcode, dp):
    """The AND of the d words the lane loads, addresses formed as the kernel does."""
    ow = offsets(pcode)
    m = (1 << 32) - 1
    for k in range(dp):
        half = base + (0 if k < 8 else 256)
        addr = byte_perm(half, ow[k >> 2], 0x3214 + (k & 3))
        idx = (addr - base) // 4
        assert 0 <= idx < 128 and (idx < 64) == (k < 8)
        m &= int(tab[idx])
    return m


@pytest.mark.parametrize("dp", [12, 16])
def test_mask_probe_selects_the_three_bit_dominance_set(dp):
    rng = np.random.default_rng(dp)
    for trial in range(300):
        d = int(rng.integers(dp - 3, dp + 1))
        codes = np.zeros((32, 16), dtype=np.int64)
        codes[:, :d] = rng.integers(0, 128, size=(32, d))
        npad = int(rng.integers(0, 4)) if trial % 3 == 0 else 0
        if npad:
            codes[32 - npad:, :dp] = 127           # padding points of the last tile
        p = np.zeros(16, dtype=np.int64)
        p[:d] = rng.integers(0, 128, size=d)
        if trial % 5 == 0:
            p[:d] = codes[int(rng.integers(0, 32)), :d]   # equal codes
        tab = table(codes)
        base = 0x4000 + 512 * int(rng.integers(0, 40))   # a 256-byte-aligned sub-tile table
        got = probe(tab, base, p, dp)
        want = 0
        for j in range(32):
            if all((codes[j, k] >> 4) <= (p[k] >> 4) for k in range(dp)):
                want |= 1 << j
        assert got == want, (trial, d)


def test_three_bit_test_is_necessary_for_seven_bit_order():
    """q <= p in every 7-bit code implies the 3-bit test passes (the mask
    probe never drops a pair the 7-bit and exact tests would keep)."""
    rng = np.random.default_rng(1)
    for _ in range(2000):
        p = rng.integers(0, 128, size=16)
        q = np.minimum(p, rng.integers(0, 128, size=16))
        tab = table(np.vstack([q] + [np.full(16, 127)] * 31))
        assert probe(tab, 0x8000, p, 16) & 1
