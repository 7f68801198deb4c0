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
* Rescale: T = round_half_away(R 2^d) from a signed 128-bit R by magnitude, a
  half-unit add and shifts, matches exact rounding.
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


def scale_round(hi, lo, d):
    """The magnitude form: |R| as (uh, ul), add half a unit, shift, restore the sign."""
    sg = M64 if hi < 0 else 0
    ul = ((lo ^ sg) - sg) & M64
    uh = (((hi & M64) ^ sg) + (1 if (sg and ul == 0) else 0)) & M64
    k = (-d) & 0xFFFFFFFF
    nl = (ul + shl64(1, (k - 1) & 0xFFFFFFFF)) & M64
    nh = (uh + shl64(1, (k - 65) & 0xFFFFFFFF) + (1 if nl < ul else 0)) & M64
    mr = shr64(nl, k) | shl64(nh, (64 - k) & 0xFFFFFFFF) | shr64(nh, (k - 64) & 0xFFFFFFFF)
    m = shl64(ul, d) if d >= 0 else mr
    return -m if hi < 0 else m


def test_scale_round_matches_exact_rounding():
    rng = random.Random(2)
    for _ in range(100000):
        d = rng.randint(-135, 40)
        lim = min(62 - d, 126)
        if lim <= 0:
            continue
        R = rng.getrandbits(rng.randint(0, lim - 1))
        if d < 0 and -d - 1 < lim - 1 and rng.random() < 0.1:
            R = ((R >> -d) << -d) + (1 << (-d - 1))  # an exact tie (still below 2^126)
        if R >= (1 << 126):
            continue
        if rng.random() < 0.5:
            R = -R
        Ru = R & ((1 << 128) - 1)
        hi = Ru >> 64
        hi = hi - (1 << 64) if hi >> 63 else hi
        lo = Ru & M64
        if d >= 0:
            exact = R << d
        else:
            k = -d
            a = abs(R)
            q = (a + (1 << (k - 1))) >> k  # half away from zero on the magnitude
            exact = -q if R < 0 else q
        assert scale_round(hi, lo, d) == exact, (R, d)


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
