"""The float64-accurate tensor-core scheme of the Dyson products, restated on the host
with exact integers (CPU only).

The kernels (k_ozaki.cu, k_ozgemm.cu, oz_slice.cuh, oz_combine.cuh) cut each row of an
operand into integer digits after scaling it into (-1/2, 1/2), multiply digit planes on
the tensor cores into per-level fp32 accumulators, combine the levels into one 64-bit
integer and round it to float64 with integer instructions.  These tests check the
arithmetic facts the kernels rely on: the digit ranges (exact in bf16), the level sums
staying within 2^22 (exact in fp32 and readable by one fp32 add), the 64-bit
combination not overflowing, the integer rounding equalling IEEE round-to-nearest-even,
and the result staying within the error bound of a float64 dot product.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def row_scale(row):
    """e with every |x| < 2^(e-1): from the largest exponent field (frexp gives m = f 2^E, f in [0.5, 1))."""
    m = max(abs(x) for x in row)
    if m == 0.0:
        return -1020
    _, E = math.frexp(m)
    return E + 1


def fixed56(x, e):
    """round(x 2^(56 - e)), halves away from zero, exactly (x is a float64)."""
    num, den = float(x).as_integer_ratio()
    scaled_num = num * (2 ** (56 - e)) if 56 - e >= 0 else num
    scaled_den = den if 56 - e >= 0 else den * 2 ** (e - 56)
    q, r = divmod(abs(scaled_num), scaled_den)
    if 2 * r >= scaled_den:
        q += 1
    return q if scaled_num >= 0 else -q


def digits(N, base, count):
    """Balanced digits of N, least significant first removed: N = sum_t d_t base^(count-1-t)."""
    half = base // 2
    out = []
    for _ in range(count - 1):
        d = ((N + half) % base) - half
        out.append(d)
        N = (N - d) // base
    out.append(N)
    return out[::-1]


SCHEMES = {
    # name: (base, digits, kept levels t + u <= L, K of one exact segment, shifts of the 64-bit combination)
    "update": (256, 7, 6, 32, [40, 32, 24, 16, 8, 0, -8]),
    "gemm": (128, 8, 7, 128, [42, 35, 28, 21, 14, 7, 0, -7]),
}


def product_by_scheme(a_rows, b_rows, scheme):
    base, nd, maxlev, _, shifts = SCHEMES[scheme]
    ea = [row_scale(r) for r in a_rows]
    eb = [row_scale(r) for r in b_rows]
    da = [[digits(fixed56(x, ea[i]), base, nd) for x in r] for i, r in enumerate(a_rows)]
    db = [[digits(fixed56(x, eb[j]), base, nd) for x in r] for j, r in enumerate(b_rows)]
    out = np.zeros((len(a_rows), len(b_rows)))
    max_level = 0
    max_v = 0
    for i in range(len(a_rows)):
        for j in range(len(b_rows)):
            S = [0] * (maxlev + 1)
            for k in range(len(a_rows[i])):
                for t in range(nd):
                    for u in range(nd):
                        if t + u <= maxlev:
                            S[t + u] += da[i][k][t] * db[j][k][u]
            max_level = max(max_level, max(abs(s) for s in S))
            V = 0
            for L, s in enumerate(S):
                V += s << shifts[L] if shifts[L] >= 0 else s >> -shifts[L]   # floor, as the kernels
            max_v = max(max_v, abs(V))
            out[i, j] = math.ldexp(float(V), ea[i] + eb[j] - 56)   # int -> float rounds to nearest even
    return out, ea, eb, max_level, max_v


@pytest.mark.parametrize("scheme", ["update", "gemm"])
def test_digit_ranges_and_reconstruction(scheme):
    base, nd, *_ = SCHEMES[scheme]
    rng = np.random.default_rng(1)
    for _ in range(2000):
        row = rng.standard_normal(8) * 10.0 ** rng.uniform(-30, 30, 8)
        e = row_scale(row)
        for x in row:
            N = fixed56(x, e)
            assert abs(N) <= 2 ** 55
            d = digits(N, base, nd)
            assert all(abs(v) <= base // 2 for v in d)              # at most 8 significant bits
            assert sum(v * base ** (nd - 1 - t) for t, v in enumerate(d)) == N
            assert abs(N * 2.0 ** (e - 56) - x) <= 2.0 ** (e - 57) * (1 + 1e-12)


@pytest.mark.parametrize("scheme", ["update", "gemm"])
def test_level_sums_exact_and_combination_in_range_at_worst_case(scheme):
    """All digits at their extreme: the level sums reach at most 2^22 and V stays below 2^63."""
    base, nd, maxlev, K, shifts = SCHEMES[scheme]
    worst = [base // 2] * nd                                    # |digit| bound
    S = [sum(worst[t] * worst[L - t] for t in range(L + 1)) * K for L in range(maxlev + 1)]
    assert max(S) <= 2 ** 22
    V = sum((s << sh) if sh >= 0 else (s >> -sh) for s, sh in zip(S, shifts))
    assert V < 2 ** 63


def test_magic_number_reads_level_sums_exactly():
    """S + 1.5 2^23 in fp32, minus the bits of 1.5 2^23, is S for every |S| <= 2^22."""
    S = np.concatenate([np.arange(-2 ** 22, -2 ** 22 + 5000), np.arange(-3000, 3000),
                        np.arange(2 ** 22 - 5000, 2 ** 22 + 1),
                        np.random.default_rng(2).integers(-2 ** 22, 2 ** 22, 200000)]).astype(np.int64)
    f = S.astype(np.float32) + np.float32(12582912.0)
    back = f.view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(back, S)


def test_integer_rounding_equals_ieee_round_to_nearest_even():
    """The rounding of a 64-bit integer (leading one, 53 bits, ties to even on the 11 dropped bits,
    exponent added), written on whole 64-bit words, equals float(v) 2^k; the kernels compute the
    same steps on 32-bit halves without branches (pinned in the next test)."""
    rng = np.random.default_rng(3)

    def by_bits(v, k):
        if v == 0:
            return 0.0
        a = abs(v)
        lz = 64 - a.bit_length()
        m = a << lz
        mant = m >> 11
        rem = m & 0x7FF
        if rem > 0x400 or (rem == 0x400 and (mant & 1)):
            mant += 1
        e = 63 - lz + k
        return math.copysign(math.ldexp(mant, e - 52), v)

    for _ in range(100000):
        v = int(rng.integers(-2 ** 62, 2 ** 62)) >> int(rng.integers(0, 62))
        if rng.random() < 0.2:   # ties and near-ties
            v = (v >> 11 << 11) | (0x400 if rng.random() < 0.5 else 0x3FF)
        k = int(rng.integers(-300, 300))
        assert by_bits(v, k) == math.ldexp(float(v), k)


@pytest.mark.parametrize("scheme", ["update", "gemm"])
def test_products_within_a_float64_dot_product_bound(scheme):
    """Rows with a wide dynamic range: the scheme's product differs from the exact dot product
    by less than 2^-52 K |a|max |b|max (a float64 dot product's bound is about K 2^-53 of the
    same)."""
    K = 32 if scheme == "update" else 40
    rng = np.random.default_rng(4)
    a = rng.standard_normal((6, K)) * 10.0 ** rng.uniform(-3, 3, (6, K))
    b = rng.standard_normal((5, K)) * 10.0 ** rng.uniform(-3, 3, (5, K))
    got, *_ = product_by_scheme(a.tolist(), b.tolist(), scheme)
    for i in range(a.shape[0]):
        for j in range(b.shape[0]):
            exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a[i], b[j]))
            bound = 2.0 ** -52 * K * np.max(np.abs(a[i])) * np.max(np.abs(b[j]))
            assert abs(Fraction(got[i, j]) - exact) <= Fraction(bound)


def test_level_pairs_combine_in_int32():
    """The epilogues first add pairs of adjacent levels in int32, (S_a << s) + S_b, and assemble the
    64-bit integer from those; at the worst-case level magnitudes no int32 intermediate overflows and
    the result equals the level-by-level 64-bit combination."""
    rng = np.random.default_rng(5)
    i32 = (-(1 << 31), (1 << 31) - 1)
    # update kernel: 7 levels, base 2^8, |S| < 2^22; GEMM: 8 levels, base 2^7, |S| <= 2^22
    for nlev, sh, bound in ((7, 8, (1 << 22) - 1), (8, 7, 1 << 22)):
        cases = [np.full(nlev, bound), np.full(nlev, -bound)]
        cases += [rng.integers(-bound, bound + 1, nlev) for _ in range(2000)]
        for S in cases:
            S = [int(x) for x in S]
            if nlev == 7:
                ref = sum(S[L] << (40 - 8 * L) for L in range(6)) + (S[6] >> 8)
                t3 = (S[0] << 8) + S[1]
                t2 = (S[2] << 8) + S[3]
                t1 = (S[4] << 8) + S[5] + (S[6] >> 8)
                parts, got = (t3, t2, t1), (t3 << 32) + (t2 << 16) + t1
            else:
                ref = sum(S[L] << (42 - 7 * L) for L in range(7)) + (S[7] >> 7)
                ta = (S[1] << 7) + S[2]
                tb = (S[3] << 7) + S[4]
                tc = (S[5] << 7) + S[6] + (S[7] >> 7)
                parts, got = (ta, tb, tc), (S[0] << 42) + (ta << 28) + (tb << 14) + tc
            assert all(i32[0] <= p <= i32[1] for p in parts)
            assert got == ref


def test_level_pairs_from_biased_bit_patterns():
    """The epilogues read each level sum as the bit pattern b = S + 0x4B400000 of the fp32 value
    S + 1.5 2^23 and remove the bias once per pair: (b_a << w) + b_b - ((bias << w) + bias) in
    32-bit arithmetic that wraps modulo 2^32 equals (S_a << w) + S_b, and (b >> w) - (bias >> w)
    equals floor(S / 2^w), for |S| <= 2^22 and w = 7, 8 (the bias is a multiple of 2^22)."""
    bias = 0x4B400000
    rng = np.random.default_rng(6)
    m32 = (1 << 32) - 1

    def as_i32(x):
        x &= m32
        return x - (1 << 32) if x >> 31 else x

    for w in (7, 8):
        cases = [((1 << 22), (1 << 22)), (-(1 << 22), -(1 << 22)), ((1 << 22), -(1 << 22)), (0, 0)]
        cases += [tuple(int(v) for v in rng.integers(-(1 << 22), (1 << 22) + 1, 2)) for _ in range(5000)]
        for sa, sb in cases:
            # the fp32 value S + 1.5 2^23 has the bit pattern S + bias (consecutive integers)
            ba = int(np.float32(sa + 12582912.0).view(np.uint32))
            bb = int(np.float32(sb + 12582912.0).view(np.uint32))
            assert ba == sa + bias and bb == sb + bias
            pair = as_i32(((ba << w) & m32) + bb - (((bias << w) & m32) + bias))
            assert pair == (sa << w) + sb
            assert (ba >> w) - (bias >> w) == sa >> w


def test_branch_free_rounding_on_32_bit_halves_equals_ieee():
    """The update epilogue's branch-free rounding (oz_round_pow2): the leading one found on
    32-bit halves (clamped funnel shifts), 53 bits kept, the tie-to-even bit added after the
    exponent field is assembled, v = 0 giving +0, and results whose exponent leaves
    (-1020, 1022) flagged for the out-of-line path.  Restated with explicit 32-bit words."""
    m32 = (1 << 32) - 1

    def clz32(x):
        return 32 - x.bit_length()

    def funnel_lc(lo, hi, s):          # top word of (hi:lo) << min(s, 32)
        return ((((hi << 32) | lo) << min(s, 32)) >> 32) & m32

    def funnel_r(lo, hi, s):           # low word of (hi:lo) >> (s & 31)
        return ((((hi << 32) | lo) >> (s & 31))) & m32

    def branch_free(v, k):
        sm = m32 * 2 ** 32 + m32 if v < 0 else 0
        a = ((v & ((1 << 64) - 1)) ^ sm) - sm & ((1 << 64) - 1)
        ah, al = a >> 32, a & m32
        big = ah != 0
        xh, xl = (ah, al) if big else (al, 0)
        s = clz32(xh)
        mh, ml = funnel_lc(xl, xh, s), funnel_lc(0, xl, s)
        nh, nl = mh >> 11, funnel_r(ml, mh, 11)
        up = ((ml & 0x7FF) + (nl & 1) + 0x3FF) >> 11
        e = (63 if big else 31) - s + k
        in_range = 0 <= e + 1019 <= 2040
        ok = in_range or xh == 0
        hi = (((e + 1022) << 20) + nh) & m32
        bits = (((hi << 32) | nl) + up) & ((1 << 64) - 1)
        bits |= sm & (1 << 63)
        if not (xh != 0 and in_range):
            bits = 0
        return np.array([bits], dtype=np.uint64).view(np.float64)[0], ok

    rng = np.random.default_rng(7)
    cases = [(0, 5), (1, 0), (-1, 0), ((1 << 62) - 1, -40), (-(1 << 62) + 1, 7), ((1 << 53) + 1, 0),
             ((1 << 53) + 3, 0), ((1 << 32) - 1, 3), (1 << 32, -3), (0x7FF, 0), (0xFFF, 2)]
    for _ in range(60000):
        v = int(rng.integers(-2 ** 62, 2 ** 62)) >> int(rng.integers(0, 62))
        if rng.random() < 0.25:   # ties and near-ties
            v = (v >> 11 << 11) | int(rng.choice([0x400, 0x3FF, 0x401, 0xC00]))
        cases.append((v, int(rng.integers(-400, 400))))
    # exponents at the edges of the directly assembled range
    cases += [(3 << 40, -1020 - 41), (3 << 40, -1020 - 42), (3 << 40, 1021 - 41), (3 << 40, 1022 - 41)]
    for v, k in cases:
        got, ok = branch_free(v, k)
        if v == 0:
            assert ok and got == 0.0 and not math.copysign(1.0, got) < 0
        elif ok:
            assert got == math.ldexp(float(v), k), (v, k)
        else:
            e = v.bit_length() - 1 + k if v > 0 else (-v).bit_length() - 1 + k
            assert not (-1020 < e < 1022) and got == 0.0


def test_bias_product_starts_each_level_at_the_magic_number():
    """The update kernel starts every level accumulator with one K = 16 product of constant
    bf16 tiles, 1.0 (bits 0x3F80) times 1.5 2^19 (bits 0x4940): sixteen exact products sum to
    1.5 2^23, so each level then holds S + 1.5 2^23, whose fp32 bits are S + 0x4B400000."""
    one = np.array([0x3F80 << 16], dtype=np.uint32).view(np.float32)[0]
    c = np.array([0x4940 << 16], dtype=np.uint32).view(np.float32)[0]
    assert one == 1.0 and c == 1.5 * 2 ** 19
    acc = np.float32(0.0)
    for _ in range(16):
        acc = np.float32(acc + np.float32(one * c))
    assert acc == np.float32(12582912.0)
    assert int(np.array([acc], dtype=np.float32).view(np.uint32)[0]) == 0x4B400000


def _update_tile(L):
    """The update kernel's numbering of the tiles that reach the lower triangle (oz_tile)."""
    s = int(math.sqrt(L))
    while s * s > L:
        s -= 1
    while (s + 1) * (s + 1) <= L:
        s += 1
    return (2 * s - 1, L - s * s) if L < s * s + s else (2 * s, L - s * s - s)


def _update_tile_count(ti_tiles):
    m = ti_tiles >> 1
    return (m + 1) * (m + 1) if ti_tiles & 1 else m * (m + 1)


def test_update_tiles_numbered_directly_are_the_lower_triangle_tiles():
    """Tiles of 64 rows x 128 columns: the direct numbering lists, in row order, exactly the tiles
    with tj 128 <= ti 64 + 63, and no column tile beyond ceil(n / 128)."""
    for n in list(range(1, 700)) + [2592, 3889, 6768, 9312]:
        ti_tiles, tj_tiles = -(-n // 64), -(-n // 128)
        want = [(ti, tj) for ti in range(ti_tiles) for tj in range(tj_tiles) if tj * 128 <= ti * 64 + 63]
        got = [_update_tile(L) for L in range(_update_tile_count(ti_tiles))]
        assert got == want, n


@pytest.mark.parametrize("n,x0,x1,grid", [(100, 0, 64, 152), (130, 32, 96, 152), (257, 224, 257, 7),
                                          (700, 320, 384, 152), (1000, 0, 0, 3), (64, 0, 32, 152), (1, 0, 0, 152)])
def test_update_tile_walk_rewrites_each_lower_element_once(n, x0, x1, grid):
    """The update's epilogue walk (16 warps, each 32 columns of its TMEM lane quarter x 16 rows, the
    per-lane row masks): every element on or below the diagonal outside the rows and columns
    [x0, x1) is rewritten exactly once, nothing else is touched, and stage indices stay in range."""
    ti_tiles = -(-n // 64)
    tiles = _update_tile_count(ti_tiles)
    hits = np.zeros((n, n), np.int32)
    g = min(tiles, grid)
    for b in range(g):
        for L in range(b, tiles, g):
            ti, tj = _update_tile(L)
            for ew in range(16):
                quarter, cg = (ew + 2) & 3, ew >> 2
                i0 = ti * 64 + cg * 16
                rows_in = 0
                for lane in range(16):
                    i = i0 + lane
                    if i < n and not (x0 <= i < x1):
                        rows_in |= 1 << lane
                for lane in range(32):
                    j = tj * 128 + quarter * 32 + lane
                    rmin = j - i0
                    lower = 0xFFFF if rmin <= 0 else (0 if rmin >= 16 else (0xFFFF << rmin) & 0xFFFF)
                    take = (rows_in & lower) if (j < n and not (x0 <= j < x1)) else 0
                    for c in range(16):
                        if take >> c & 1:
                            assert ew * 16 * 32 + c * 32 + lane < 16 * 16 * 32
                            hits[i0 + c, j] += 1
    want = np.tril(np.ones((n, n), np.int32))
    want[x0:x1, :] = 0
    want[:, x0:x1] = 0
    assert np.array_equal(hits, want)
