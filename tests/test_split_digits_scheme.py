"""The split-precision representation (emulated FP64 on BF16 tensor cores), checked as
arithmetic on the CPU: a value scaled by its row's power of two, rounded to an integer of 8S bits
and written as S balanced base-256 digits (top digit signed, the rest in [-128, 127]) is recovered
exactly; every digit scaled by 2^(-8t) is a BF16 number; and the products of two such expansions
kept for t + u <= S + 1 (1-based), the set the GEMM accumulates, reproduce the FP64 product to
about 2^(-8S) of its scale."""
import numpy as np
import pytest

S = 6


def digits(x, E):
    """Balanced base-256 digits of round(x 2^(8S-1-E)) via the biased-byte reading: adding 128 to
    every byte below the top turns the balanced digits into the plain bytes of the sum."""
    g = int(np.rint(np.ldexp(x, 8 * S - 1 - E)))
    bias = sum(128 << (8 * t) for t in range(S - 1))
    b = g + bias
    d = [b >> (8 * (S - 1))]                        # top digit (Python's >> is arithmetic)
    for t in range(1, S):
        d.append(((b >> (8 * (S - 1 - t))) & 0xFF) - 128)
    return g, d


def is_bf16(v):
    f = np.float32(v)
    return float(f) == v and (f.view(np.uint32) & 0xFFFF) == 0


@pytest.mark.parametrize("seed", range(5))
def test_digits_reconstruct_and_are_bf16(seed):
    rng = np.random.default_rng(seed)
    for _ in range(2000):
        x = rng.normal() * 10.0 ** rng.uniform(-3, 3)
        E = int(np.frexp(abs(x))[1]) if x != 0 else -1021     # |x| < 2^E
        g, d = digits(x, E)
        assert sum(dt * 256 ** (S - 1 - t) for t, dt in enumerate(d)) == g
        assert all(-128 <= dt <= 127 for dt in d[1:]) and -129 <= d[0] <= 128
        for t, dt in enumerate(d):
            assert is_bf16(np.ldexp(float(dt), -8 * t))


def test_truncated_product_set_is_accurate():
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(2000):
        x, y = rng.uniform(-1, 1, 2)
        _, dx = digits(x, 0)
        _, dy = digits(y, 0)
        # value of digit t: d_t 2^(-8t) 2^(E - 8S + 1 + 8(S-1)) with E = 0 -> d_t 2^(-8t - 7)
        p = sum(dx[t] * dy[u] * 2.0 ** (-8 * (t + u) - 14)
                for t in range(S) for u in range(S) if t + u <= S - 1)
        worst = max(worst, abs(p - x * y))
    assert worst < 2.0 ** (-8 * S + 2)
