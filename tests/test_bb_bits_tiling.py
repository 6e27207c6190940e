"""Host-side model of how the bit-sliced bounding-box row kernels
(bb_bits2_kernel, bb_bits3_kernel) split a row of n cells into writes: strips
992 cells apart, lane l (0..30) of a strip writing the two aligned 16-byte
chunks from F + xs + 32 l - k + 16 when they end inside the row, strip 0
writing the head bytes F .. F + xs - k + 15, and the chunk that holds the
row's end written byte by byte by the strip whose range has it.  For every
row length and every alignment of the row's start this checks that each byte
of the row is written exactly once and nothing outside it, and that every
written byte comes from a lane cell whose neighbours the warp holds (lane 0's
cell 0 only when the strip starts the row; lane 31's cells only up to 15 - k,
whose right neighbours are at most cell 16 - k of the same lane)."""
import numpy as np
import pytest

STRIP = 992


def strips_for(n):
    return 1 if n <= 993 else (n - 993 + 991) // 992 + 1


def writes(n, f0):
    """(byte, strip, lane, cell) for every byte the kernels write in a row of
    n cells starting at flat offset f0."""
    out = []
    e = f0 + n
    for sx in range(strips_for(n)):
        xs = sx * STRIP
        k = (f0 + xs) & 15
        a0 = f0 + xs - k
        for lane in range(31):
            for h in range(2):
                c = a0 + 32 * lane + 16 + 16 * h
                if c + 16 <= e:
                    for j in range(16):
                        # byte c + j is cell (c + j) - (a0 + k) of lane 0's numbering
                        cell = c + j - (a0 + k)
                        out.append((c + j, sx, cell // 32, cell % 32, k))
        if xs == 0:
            for j in range(16 - k):
                out.append((f0 + j, sx, 0, j, k))
        rem = e & 15
        if rem:
            q = (e - a0 - 16) >> 4
            if 0 <= q < 62:
                base = a0 + 16 + 16 * q
                for j in range(rem):
                    cell = base + j - (a0 + k)
                    out.append((base + j, sx, cell // 32, cell % 32, k))
    return out


@pytest.mark.parametrize("n", [32, 33, 48, 81, 128, 243, 496, 511, 729, 991, 992, 993, 994, 1024, 1985, 1986,
                               2187, 2976, 6561])
def test_every_byte_once_and_from_valid_cells(n):
    for f0 in range(0, 16 * 5, 5):   # every start alignment mod 16, several rows apart
        w = writes(n, f0)
        idx = np.array([b for b, *_ in w], dtype=np.int64)
        assert idx.min() >= f0 and idx.max() < f0 + n, (n, f0)
        counts = np.bincount(idx - f0, minlength=n)
        assert (counts == 1).all(), (n, f0, np.nonzero(counts != 1)[0][:5])
        for b, sx, lane, cell, k in w:
            x = b - f0
            assert x == sx * STRIP + 32 * lane + cell, (n, f0, b)   # the byte is that lane's cell
            assert lane <= 31
            if lane == 0 and cell == 0:
                assert sx == 0   # its left neighbour is known only at the row's start
            if lane == 31:
                assert cell <= 15 - k   # right neighbour cell <= 16 - k of lane 31, still loaded


def test_strip_count_is_minimal():
    for n in range(32, 5000, 7):
        s = strips_for(n)
        assert (s - 1) * STRIP + 993 >= n   # the last strip reaches the row's end
        if s > 1:
            assert (s - 2) * STRIP + 993 < n   # one strip fewer would not
