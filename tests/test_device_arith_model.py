"""The exact-arithmetic steps of the fused BC-Back wave (evd_bcback.cu), checked on
the CPU against exact integer arithmetic.  Each check restates the step from its
mathematical definition and the instruction semantics it relies on (IEEE float32 and
float16 round-to-nearest, PTX byte permute, PTX 64-bit shifts whose amounts clamp at
64); it does not call the CUDA path.

* Digits: an operand with frexp exponent e is T = round_half_away(x 2^(8S - 1 - e)),
  |T| <= 2^(8S - 1); with the offset O = 128 (1 + 256 + ... + 256^(S-2)) the bytes of
  T + O minus 128 and the top part (T + O) >> 8(S - 1) are balanced base-256 digits
  in [-128, 127] and [-128, 128] that rebuild T.
* Float16 digit construction: the float16 with bits 0x6400 | f is 1024 + f, minus
  1152 gives f - 128; the bits 0x6480 + d are 1152 + d for a top digit d.
* Accumulator bounds: with every digit in [-128, 128], diagonal k (the pairs
  t + u = k) is bounded by (k + 1) K 2^14 < 2^24 for K <= 128 and S <= 7, so the
  FP32 accumulators hold exact integers.
* Add trick and its test: bits(v + 1.5 * 2^23) - 0x4B400000 is v exactly when the
  sum stays in [2^23, 2^24), which the exponent field shows; otherwise the hardware
  conversion's term replaces it.
* Rescale: T = floor(R 2^d + 1/2) from a signed 128-bit R by a half-unit add in
  two's complement and an arithmetic shift, with PTX's clamped shift amounts, matches
  exact rounding (to nearest, ties toward +infinity); so does the 64-bit form
  (Rh << (G - k)) + ((Rl + 2^(k-1)) >> k) of R = Rh 2^G + Rl for 0 < k < G, and the
  bit length of the split form equals that of the 128-bit value.
* Scale of W from the one's complement bit length: every scaled value stays within
  [-2^w, 2^w], the top digit within [-128, 128].
* Recombination and drain: R = Rh 2^(8 (L - H)) + Rl rebuilds sum_k acc_k 2^(8 (L - k)),
  also through the wide multiply-adds modulo 2^64 with the magic offsets cancelled.
* The whole wave on one small tile: X^T V, the W split, Y W and the fixed-point update
  with the kernel's scale exponents, against the exact rational products.
"""
import math
import random
from fractions import Fraction

import numpy as np

M64 = (1 << 64) - 1
MAGIC = 0x4B400000


def f32(x):
    return np.float32(x)


def _bits(v):
    s = f32(f32(v) + f32(12582912.0))
    return int(np.array([s], dtype=np.float32).view(np.uint32)[0])


def offset8(S):
    o = 0
    for _ in range(S - 1):
        o = (o << 8) + 128
    return o


def digits8(T, S):
    """Slices 0 .. S-1 (slice 0 the top digit) of T as the kernel forms them."""
    TO = T + offset8(S)
    d = []
    for t in range(S):
        j = S - 1 - t
        d.append(TO >> (8 * j) if t == 0 else ((TO >> (8 * j)) & 255) - 128)
    return d


def test_digits_rebuild_the_integer():
    rng = random.Random(7)
    for S in (6, 7):
        lim = 1 << (8 * S - 1)
        vals = [lim, -lim, 0, 1, -1, lim - 1, -lim + 1] + [rng.randint(-lim, lim) for _ in range(20000)]
        for T in vals:
            d = digits8(T, S)
            assert -128 <= d[0] <= 128
            assert all(-128 <= x <= 127 for x in d[1:])
            assert sum(d[t] << (8 * (S - 1 - t)) for t in range(S)) == T


def byte_perm(a, b, sel):
    """PTX prmt.b32 (default mode): output byte i is byte (sel >> 4i) & 7 of b:a."""
    pool = (b << 32) | a
    out = 0
    for i in range(4):
        k = (sel >> (4 * i)) & 7
        out |= ((pool >> (8 * k)) & 255) << (8 * i)
    return out


def f16_value(bits16):
    return float(np.array([bits16], dtype=np.uint16).view(np.float16)[0])


def test_float16_digit_pairs():
    assert f16_value(0x6480) == 1152.0
    for f in range(256):
        assert f16_value(0x6400 | f) == 1024.0 + f
        d = np.float16(f16_value(0x6400 | f)) - np.float16(1152.0)
        assert float(d) == f - 128
    for d in range(-128, 129):
        v = np.float16(f16_value(0x6480 + d)) - np.float16(1152.0)
        assert float(v) == d
    # the byte permute places byte j of two words at bytes 0 and 2; the mask and the
    # exponent bytes make the float16 pair (1024 + fa, 1024 + fb)
    rng = random.Random(8)
    for _ in range(2000):
        wa, wb, j = rng.getrandbits(32), rng.getrandbits(32), rng.randrange(4)
        w = (byte_perm(wa, wb, j | ((4 + j) << 8)) & 0x00FF00FF) | 0x64006400
        assert f16_value(w & 0xFFFF) == 1024 + ((wa >> (8 * j)) & 255)
        assert f16_value(w >> 16) == 1024 + ((wb >> (8 * j)) & 255)
    # the top pair: low halves of two words
    for _ in range(2000):
        a, b = rng.getrandbits(32), rng.getrandbits(32)
        assert byte_perm(a, b, 0x5410) == (a & 0xFFFF) | ((b & 0xFFFF) << 16)


def test_accumulator_bound():
    for S in (6, 7):
        for k in range(S):
            pairs = min(k, S - 1) + 1
            for K in (127, 64):  # phase 1 (h = 127 rows; the 128th is zero) and phase 2
                assert pairs * K * 128 * 128 < (1 << 24), (S, k, K)


def test_add_trick_and_its_exactness_test():
    rng = random.Random(1)
    vals = list(range(-3000, 3000)) + [-(1 << 22), (1 << 22) - 1, (1 << 22), -(1 << 22) - 1, (1 << 24) - 1,
                                       -(1 << 24) + 1]
    vals += [rng.randrange(-(1 << 24) + 1, 1 << 24) for _ in range(40000)]
    for v in vals:
        b = _bits(v)
        in_binade = ((b ^ 0x4B000000) >> 23) == 0
        assert in_binade == (-(1 << 22) <= v < (1 << 22)), v
        if in_binade:
            assert b - MAGIC == v


def shl64(x, k):
    k &= 0xFFFFFFFF
    return 0 if k >= 64 else (x << k) & M64


def shr64(x, k):
    k &= 0xFFFFFFFF
    return 0 if k >= 64 else (x & M64) >> k


def sar64(x, k):
    """shr.s64: an amount above 64 clamps to 64 (the sign fill)."""
    k &= 0xFFFFFFFF
    x = x - (1 << 64) if x >> 63 else x
    return x >> min(k, 64)


def round_shift(hi, lo, d):
    """The kernel's two's-complement form: add 2^(k-1), shift right arithmetically."""
    if d >= 0:
        v = shl64(lo, d)
        return v - (1 << 64) if v >> 63 else v
    k = (-d) & 0xFFFFFFFF
    nl = (lo + shl64(1, (k - 1) & 0xFFFFFFFF)) & M64
    nh = (hi + shl64(1, (k - 65) & 0xFFFFFFFF) + (1 if nl < lo else 0)) & M64
    low = shr64(nl, k) | shl64(nh, (64 - k) & 0xFFFFFFFF)
    high = sar64(nh, (k - 64) & 0xFFFFFFFF)
    r = 0 if k >= 127 else (low if k < 64 else high)
    r &= M64
    return r - (1 << 64) if r >> 63 else r


def bitlen128(hi, lo):
    sg = M64 if hi < 0 else 0
    h, l = (hi & M64) ^ sg, lo ^ sg
    return 64 + h.bit_length() if h else l.bit_length()


def _split128(R):
    Ru = R & ((1 << 128) - 1)
    hi = Ru >> 64
    return (hi - (1 << 64) if hi >> 63 else hi), Ru & M64


def test_round_shift_is_round_to_nearest_ties_up():
    rng = random.Random(2)
    for _ in range(100000):
        d = rng.randint(-140, 40)
        lim = min(62 - d, 125)
        if lim <= 0:
            continue
        R = rng.getrandbits(rng.randint(0, lim - 1))
        if d < 0 and -d - 1 < lim - 1 and rng.random() < 0.1:
            R = ((R >> -d) << -d) + (1 << (-d - 1))  # an exact tie
        if rng.random() < 0.5:
            R = -R
        hi, lo = _split128(R)
        exact = R << d if d >= 0 else (R + (1 << (-d - 1))) >> -d  # floor(R 2^d + 1/2)
        assert round_shift(hi, lo, d) == exact, (R, d)


def round_split(Rh, Rl, k, G):
    """The kernel's 64-bit rescale of R = Rh 2^G + Rl for 0 < k < G."""
    a = (Rh << (G - k)) & M64
    b = ((Rl + (1 << (k - 1))) & M64)
    b = (b - (1 << 64) if b >> 63 else b) >> k
    return _signed((a + b) & M64)


def bitlen64(x):
    x &= M64
    x ^= M64 if x >> 63 else 0
    return x.bit_length()


def bitlen_split(Rh, Rl, G):
    s = Rh + (Rl >> G)
    r = _signed(((s << G) + (Rl & ((1 << G) - 1))) & M64)
    return bitlen64(s) + G if s not in (0, -1) else bitlen64(r)


def test_split_rescale_and_bit_length():
    rng = random.Random(9)
    for S in (6, 7):
        L, H, w = _weights(S)
        G = 8 * (L - H)
        for _ in range(40000):
            acc = [rng.randint(-(1 << 24) + 1, (1 << 24) - 1) if rng.random() < 0.8 else rng.randint(-300, 300)
                   for _ in range(S)]
            if rng.random() < 0.05:
                acc = [0] * S
                acc[rng.randrange(S)] = rng.choice([1, -1, 2, -2, 1 << 20, -(1 << 20)])
            Rh = sum(acc[k] * w[k] for k in range(0, H + 1))
            Rl = sum(acc[k] * w[k] for k in range(H + 1, S))
            R = (Rh << G) + Rl
            hi, lo = _split128(R)
            assert bitlen_split(Rh, Rl, G) == bitlen128(hi, lo)
            kmin = max(1, abs(R).bit_length() - 61)  # the kernel's range: |R 2^-k| < 2^62
            if kmin > G - 1:
                continue
            k = rng.randint(kmin, G - 1)
            assert round_split(Rh, Rl, k, G) == (R + (1 << (k - 1))) >> k == round_shift(hi, lo, -k)


def test_one_complement_bit_length_keeps_the_top_digit_in_range():
    """With the scale from the one's complement bit length, every scaled value rounds
    into [-2^w, 2^w] (w = 8S - 1), and only a negative power of two reaches -2^w: a top
    digit of magnitude at most 128."""
    rng = random.Random(5)
    for S in (6, 7):
        w = 8 * S - 1
        for _ in range(30000):
            p = rng.randint(1, 120)
            R = rng.getrandbits(p) if rng.random() < 0.9 else (1 << (p - 1))
            if rng.random() < 0.5:
                R = -R
            if R == 0:
                continue
            hi, lo = _split128(R)
            bl = bitlen128(hi, lo)
            assert bl == (abs(R).bit_length() if R > 0 else (abs(R) - 1).bit_length())
            T = round_shift(hi, lo, w - bl)
            assert -(1 << w) <= T <= (1 << w)
            assert -128 <= digits8(T, S)[0] <= 128
            if T == -(1 << w):
                assert R < 0 and abs(R) & (abs(R) - 1) == 0


def _weights(S):
    L, H = S - 1, min(S - 1, 3)
    return L, H, [1 << (8 * (H - k)) if k <= H else 1 << (8 * (L - k)) for k in range(S)]


def test_recombination_is_exact():
    rng = random.Random(3)
    for S in (6, 7):
        L, H, w = _weights(S)
        for _ in range(2000):
            acc = [rng.randint(-(1 << 24) + 1, (1 << 24) - 1) for _ in range(S)]
            Rh = sum(acc[k] * w[k] for k in range(0, H + 1))
            Rl = sum(acc[k] * w[k] for k in range(H + 1, S))
            assert (Rh << (8 * (L - H))) + Rl == sum(acc[k] << (8 * (L - k)) for k in range(S))
            assert -(1 << 63) <= Rh < (1 << 63) and -(1 << 63) <= Rl < (1 << 63)


def _signed(x):
    return x - (1 << 64) if x >> 63 else x


def drain_model(acc, S):
    """Rh, Rl as the kernel forms them: wide multiply-adds of the add trick's bits from
    the magic starting values, then the conversion's correction where a sum left the
    binade (all modulo 2^64)."""
    L, H, w = _weights(S)
    uh = (-MAGIC * sum(w[k] for k in range(S) if k <= H)) & M64
    ul = (-MAGIC * sum(w[k] for k in range(S) if k > H)) & M64
    for k in range(S):
        b = _bits(acc[k])
        term = b * w[k]
        if ((b ^ 0x4B000000) >> 23) != 0:
            term += w[k] * (acc[k] - (b - MAGIC))
        if k <= H:
            uh = (uh + term) & M64
        else:
            ul = (ul + term) & M64
    return _signed(uh), _signed(ul)


def test_drain_by_wide_multiply_add_matches_direct_sums():
    rng = random.Random(4)
    for S in (6, 7):
        L, H, w = _weights(S)
        for _ in range(4000):
            acc = [rng.randint(-(1 << 22), (1 << 22) - 1) if rng.random() < 0.7 else
                   rng.choice([(1 << 24) - 1, -(1 << 24) + 1, rng.randint(-(1 << 24) + 1, (1 << 24) - 1)])
                   for _ in range(S)]
            Rh, Rl = drain_model(acc, S)
            assert Rh == sum(acc[k] * w[k] for k in range(0, H + 1))
            assert Rl == sum(acc[k] * w[k] for k in range(H + 1, S))


def scaled(x, p):
    """round_half_away(x 2^p) for a double x."""
    v = Fraction(x) * (Fraction(2) ** p)
    r = math.floor(abs(v) + Fraction(1, 2))
    return r if v >= 0 else -r


def frexp_e(vals):
    mx = max(abs(v) for v in vals)
    return math.frexp(mx)[1] if mx > 0 else -1022


def diag_product(dA, dB, S):
    """R = sum_k acc_k 256^(L - k), acc_k = sum over pairs t + u = k and over K of dA_t dB_u."""
    L = S - 1
    acc = [0] * S
    for t in range(S):
        for u in range(S - t):
            acc[t + u] += sum(a * b for a, b in zip(dA[t], dB[u]))
    for a in acc:
        assert abs(a) < (1 << 24)
    Rh, Rl = drain_model(acc, S)
    H = min(L, 3)
    R = (Rh << (8 * (L - H))) + Rl
    assert R == sum(acc[k] << (8 * (L - k)) for k in range(S))
    return R


def test_wave_tile_scales_match_exact_products():
    """One column of X (h rows), a 64-column V and a Y through the kernel's integer
    steps: W^T = R 2^(eV_i - 8S - 6), T_W = round(R 2^(eV_i - 7 - eW)), the update
    round(R2 2^(eW + eY_r - 7)) on the grid 2^(1 - 8S).  The result must match the
    exact rational Y (V^T x) to the digits' precision; a wrong exponent anywhere is off
    by a power of two."""
    rng = np.random.default_rng(11)
    for S in (6, 7):
        h, g = 127, 64
        x = rng.standard_normal(h)
        x /= np.linalg.norm(x) * 1.01
        V = rng.standard_normal((h, g)) * np.exp2(rng.integers(-3, 3, size=g))
        Y = rng.standard_normal((h, g)) * np.exp2(rng.integers(-3, 3, size=h))[:, None]
        # X in fixed point, its digits per row
        TX = [scaled(float(v), 8 * S - 1) for v in x]
        dX = list(zip(*[digits8(T, S) for T in TX]))
        # phase 1: W^T(i) for the one column of X
        eV = [frexp_e(V[:, i]) for i in range(g)]
        R1, bl = [], []
        for i in range(g):
            TV = [scaled(float(V[r, i]), 8 * S - 1 - eV[i]) for r in range(h)]
            dV = list(zip(*[digits8(T, S) for T in TV]))
            R = diag_product(dX, dV, S)
            R1.append(R)
            hi, lo = _split128(R)
            bl.append(bitlen128(hi, lo))
            exact = sum(Fraction(float(x[r])) * Fraction(float(V[r, i])) for r in range(h))
            approx = Fraction(R) * Fraction(2) ** (eV[i] - 8 * S - 6)
            assert abs(approx - exact) <= Fraction(2) ** (eV[i] - 8 * S + 10), (S, i)
        eW = max(b + e - 8 * S - 6 for b, e in zip(bl, eV) if b > 0)
        TW = [round_shift(*_split128(R), e - 7 - eW) for R, e in zip(R1, eV)]
        assert all(-(1 << (8 * S - 1)) <= T <= (1 << (8 * S - 1)) for T in TW)
        dW = list(zip(*[digits8(T, S) for T in TW]))
        w_exact = [sum(Fraction(float(x[r])) * Fraction(float(V[r, i])) for r in range(h)) for i in range(g)]
        # phase 2: the update of the column at every row r
        for r in range(0, h, 9):
            eY = frexp_e(Y[r, :])
            TY = [scaled(float(Y[r, i]), 8 * S - 1 - eY) for i in range(g)]
            dY = list(zip(*[digits8(T, S) for T in TY]))
            R2 = diag_product(dY, dW, S)
            dT = round_shift(*_split128(R2), eW + eY - 7)
            exact = sum(Fraction(float(Y[r, i])) * w_exact[i] for i in range(g))
            got = Fraction(dT) * Fraction(2) ** (1 - 8 * S)
            tol = Fraction(2) ** (eY + eW - 8 * S + 12)
            assert abs(got - exact) <= tol, (S, r, float(got), float(exact))
