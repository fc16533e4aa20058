"""Integer arithmetic of the FP64 tensor-core kernels, restated on the host (CPU only).

The device code cuts each row-scaled value into balanced 7-bit digits (least significant
first, in two 28-bit halves) and stores every digit as bf16; after the MMAs it combines the
eight diagonal sums from their FP32 bit patterns with two folded constants.  These tests
check the stated identities of that arithmetic -- exact reconstruction, digit bounds, exact
bf16 storage, and the folded combination against the plain Horner form -- on random and
extreme integers, so that a change to either recipe that breaks them fails here."""
import struct

import numpy as np

MASK64 = (1 << 64) - 1


def f32_bits_of_int(v):
    """FP32 bits of (1.5 2^23 + v) - 1.5 2^23 for |v| < 2^22."""
    a = struct.unpack("<f", struct.pack("<I", (0x4B400000 + v) & 0xFFFFFFFF))[0]
    r = np.float32(a) - np.float32(12582912.0)
    return struct.unpack("<I", struct.pack("<f", float(r)))[0]


def digits(R):
    """Balanced base-2^7 digits of |R| < 2^56, least significant first, in two halves."""
    lo, hi = R & 0x0FFFFFFF, R >> 28
    d = [0] * 8
    for p in range(7, -1, -1):
        if p >= 4:
            dg = ((lo + 64) & 127) - 64
            lo = (lo - dg) >> 7
            if p == 4:
                assert lo in (0, 1)
                hi += lo
        elif p >= 1:
            dg = ((hi + 64) & 127) - 64
            hi = (hi - dg) >> 7
        else:
            dg = hi
        d[p] = dg
    return d


def test_digits_reconstruct_within_bounds_and_store_exactly_in_bf16():
    rng = np.random.default_rng(7)
    cases = [0, 1, -1, 2**56 - 1, -(2**56 - 1), 2**48 - 1, -(2**48), 2**55, 64, -64, 63, 127, 128]
    cases += [int(x) for x in rng.integers(-(2**56) + 1, 2**56, size=20000, dtype=np.int64)]
    cases += [int(s) * int(rng.integers(0, 2 ** int(b))) for s, b in
              zip(rng.choice([-1, 1], 5000), rng.integers(1, 57, 5000))]
    for R in cases:
        d = digits(R)
        assert sum(d[p] << (49 - 7 * p) for p in range(8)) == R
        assert abs(d[0]) <= 128 and all(-64 <= x <= 63 for x in d[1:])
        for x in d:
            b = f32_bits_of_int(x)
            assert b & 0xFFFF == 0  # the low half is zero: the high half is x in bf16
            assert struct.unpack("<f", struct.pack("<I", b))[0] == x


LO_BIAS = 0xFFF6850A14C00080
HI_BIAS = 0x50A14C00


def combine(D):
    """W from the eight diagonals' FP32 bit patterns f_d = 0x4B400000 + D_d, as the kernel
    forms it (64-bit wraparound, arithmetic shift, folded offsets)."""
    f = [(0x4B400000 + x) & 0xFFFFFFFF for x in D]
    v = (f[7] + LO_BIAS) & MASK64
    v = (f[6] * 128 + v) & MASK64
    v = (f[5] * 16384 + v) & MASK64
    v = (f[4] * 2097152 + v) & MASK64
    sv = v - (1 << 64) if v >> 63 else v
    lo = (sv >> 8) & MASK64
    w = (f[3] * 1048576 + lo) & MASK64
    w = (f[2] * 134217728 + w) & MASK64
    w = (w + ((((f[1] * 4 + f[0] * 512 + HI_BIAS) & 0xFFFFFFFF)) << 32)) & MASK64
    return w - (1 << 64) if w >> 63 else w


def horner(D):
    v_hi = sum(D[d] << (7 * (3 - d)) for d in range(4))
    v_lo = sum(D[d] << (7 * (7 - d)) for d in range(4, 8))
    return (v_hi << 20) + ((v_lo + 128) >> 8)  # round(V_lo / 2^8), half up


# Bounds of the diagonal sums for K <= 64 (|s_0| <= 2^7, |s_p| <= 2^6): diagonal d sums d + 1
# slice pairs over K, at most two of them with slice 0, so |D_0| <= K 2^14 and
# |D_d| <= K 2^12 (d + 3) for d >= 1 -- all below 2^22 (exact in FP32), and |W| < 2^62.
K = 64
BOUND = [K * 2**14] + [K * 2**12 * (d + 3) for d in range(1, 8)]


def test_diagonal_bounds_are_exact_in_fp32():
    assert max(BOUND) < 2**22
    # the largest |W| the bounds allow stays below 2^62
    assert abs(horner(BOUND)) < 2**62


def test_folded_combination_equals_horner_form():
    rng = np.random.default_rng(11)
    hi, lo = BOUND, [-b for b in BOUND]
    cases = [[0] * 8, hi, lo, [hi[d] if d % 2 else lo[d] for d in range(8)],
             [lo[d] if d % 2 else hi[d] for d in range(8)]]
    cases += [[int(rng.integers(-b, b + 1)) for b in BOUND] for _ in range(20000)]
    cases += [[int(rng.choice([-b, -1, 0, 1, b])) for b in BOUND] for _ in range(2000)]
    for D in cases:
        assert combine(D) == horner(D), D
