"""The exact-arithmetic steps of the fused BC-Back wave (evd_bcback.cu), checked on
the CPU against exact integer arithmetic.  Each check restates the step from its
mathematical definition and the instruction semantics it relies on (IEEE float32
round-to-nearest, bfloat16 as the top half of a float32, PTX 64-bit shifts whose
amounts clamp at 64); it does not call the CUDA path.

* Add trick: an FP32 accumulator value v that is an integer with |v| < 2^22 is
  recovered exactly as bits(v + 1.5 * 2^23) - 0x4B400000.
* Accumulator bounds: with top digits in [-128, 128] and the others in [-64, 63],
  K * (128^2 for k = 0, 2 * 128 * 64 + (k - 1) * 64^2 for k >= 1) bounds the sum of
  the slice-pair products of diagonal k, so the add trick is used only where it is
  exact.
* Digit pairs: the bfloat16 with bits 0x4300 | f is 128 + f for f in [0, 127], and
  subtracting 192 gives the digit f - 64 exactly.
* Rescale: T = floor(R 2^d + 1/2) from a signed 128-bit R by a half-unit add in
  two's complement and an arithmetic shift, with PTX's clamped shift amounts, matches
  exact rounding (to nearest, ties toward +infinity).
* Scale of W from the one's complement bit length: every scaled value stays within
  [-2^w, 2^w], the top digit within [-128, 128].
* Recombination: R = Rh 2^(7 (L - H)) + Rl rebuilds the exact sum of the diagonal
  sums sum_k acc_k 2^(7 (L - k)).
* Drain by wide multiply-adds: starting Rh and Rl at -0x4B400000 times the summed
  weights of the add-trick diagonals, then adding bits(v + 1.5 * 2^23) times the
  weight (or the converted integer for the other diagonals), modulo 2^64, gives the
  same Rh and Rl as the direct sums.
"""
import random

import numpy as np

M64 = (1 << 64) - 1


def f32(x):
    return np.float32(x)


def test_add_trick_recovers_integers():
    magic = f32(12582912.0)  # 1.5 * 2^23
    vals = list(range(-2000, 2000)) + [-(1 << 22), (1 << 22) - 1, (1 << 21) + 12345, -(1 << 21) - 777]
    rng = random.Random(1)
    vals += [rng.randrange(-(1 << 22), 1 << 22) for _ in range(20000)]
    for v in vals:
        s = f32(f32(v) + magic)  # exact: the sum lies in [2^23, 2^24), where the ulp is 1
        bits = int(np.array([s], dtype=np.float32).view(np.int32)[0])
        assert bits - 0x4B400000 == v


def diag_bound(K, k):
    return K * (128 * 128 if k == 0 else 2 * 128 * 64 + (k - 1) * 64 * 64)


def test_accumulator_bound_covers_all_digit_products():
    # the largest |sum over pairs (t, u), t + u = k, of d_t d'_u| for digit ranges
    # top: [-128, 128], others: [-64, 63]
    def dmax(t):
        return 128 if t == 0 else 64
    for S in (6, 8):
        for k in range(S):
            per_K = sum(dmax(t) * dmax(k - t) for t in range(k + 1) if k - t < S)
            assert per_K <= diag_bound(1, k), (S, k)
    # the kernel applies the trick where the bound is below 2^22: phase 1 (K = 128): diagonals 0..4 qualify, 5..7 take the hardware conversion
    assert [diag_bound(128, k) < (1 << 22) for k in range(8)] == [True] * 5 + [False] * 3
    assert all(diag_bound(64, k) < (1 << 22) for k in range(8))


def bf16_value(bits16):
    return float(np.array([bits16 << 16], dtype=np.uint32).view(np.float32)[0])


def bf16_round(x):
    # round a float32 to bfloat16 (nearest even) and return the value
    b = int(np.array([np.float32(x)], dtype=np.float32).view(np.uint32)[0])
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return bf16_value(b)


def test_digit_pair_construction():
    c192 = bf16_value(0x4340)
    assert c192 == 192.0
    for f in range(128):
        v = bf16_value(0x4300 | f)
        assert v == 128.0 + f
        d = bf16_round(np.float32(v) - np.float32(c192))
        assert d == f - 64


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


def test_one_complement_bit_length_keeps_the_top_digit_in_range():
    """With the scale from the one's complement bit length, every scaled value rounds
    into [-2^w, 2^w] (w = the digits' total width), and only a negative power of two
    reaches -2^w: a top digit of magnitude at most 128."""
    rng = random.Random(5)
    w = 56
    for _ in range(50000):
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
        if T == -(1 << w):
            assert R < 0 and abs(R) & (abs(R) - 1) == 0


def test_recombination_is_exact():
    rng = random.Random(3)
    for S in (6, 8):
        L, H = S - 1, min(S - 1, 3)
        for _ in range(2000):
            acc = [rng.randint(-(1 << 23), 1 << 23) for _ in range(S)]
            Rh = sum(acc[k] << (7 * (H - k)) for k in range(0, H + 1))
            Rl = sum(acc[k] << (7 * (L - k)) for k in range(H + 1, S))
            assert (Rh << (7 * (L - H))) + Rl == sum(acc[k] << (7 * (L - k)) for k in range(S))
            assert -(1 << 63) <= Rh < (1 << 63) and -(1 << 63) <= Rl < (1 << 63)


def _small(K, k):
    return diag_bound(K, k) < (1 << 22)


def _bits(v):
    s = f32(f32(v) + f32(12582912.0))
    return int(np.array([s], dtype=np.float32).view(np.uint32)[0])


def test_drain_by_wide_multiply_add_matches_direct_sums():
    rng = random.Random(4)
    for S in (6, 8):
        L, H = S - 1, min(S - 1, 3)
        w = [1 << (7 * (H - k)) if k <= H else 1 << (7 * (L - k)) for k in range(S)]
        for K in (128, 64):
            start_h = -0x4B400000 * sum(w[k] for k in range(S) if _small(K, k) and k <= H)
            start_l = -0x4B400000 * sum(w[k] for k in range(S) if _small(K, k) and k > H)
            for _ in range(3000):
                acc = [rng.randint(-diag_bound(K, k), diag_bound(K, k)) if rng.random() < 0.9 else
                       (diag_bound(K, k) if rng.random() < 0.5 else -diag_bound(K, k)) for k in range(S)]
                uh, ul = start_h & M64, start_l & M64
                for k in range(S):
                    term = (_bits(acc[k]) if _small(K, k) else acc[k]) * w[k]
                    if k <= H:
                        uh = (uh + term) & M64
                    else:
                        ul = (ul + term) & M64
                signed = lambda x: x - (1 << 64) if x >> 63 else x
                assert signed(uh) == sum(acc[k] * w[k] for k in range(0, H + 1))
                assert signed(ul) == sum(acc[k] * w[k] for k in range(H + 1, S))
