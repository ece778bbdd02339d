"""A numpy model of the split-precision arithmetic (the scheme, not the kernel), checking the
claims the tensor-core GEMM rests on:

* rows scaled by 2^E (|x| < 2^E) and cut into S balanced base-256 digits reproduce x to 8S - 1
  bits, every digit exact in BF16 (8 significant bits);
* within a 256-element K chunk, the accumulator of scale t+u holds at most four products per K for
  the leading four scales, so each partial sum is an integer below 2^24 (times the scale) and
  exact in FP32, in any summation order;
* keeping the slice products with t+u <= S+1 and summing the chunks in float-float gives a
  product whose error falls by about 2^8 per slice (S = 4, 5, 6).
"""
import numpy as np
import pytest


def _digits(x, S):
    """Balanced base-256 digits of every row of x: x = 2^(E-7) sum_t d_t 2^(-8(t-1))."""
    E = np.ceil(np.log2(np.max(np.abs(x), axis=1) * (1 + 2.0 ** -52) + 1e-300)).astype(int)
    X = np.rint(x * np.ldexp(1.0, 8 * S - 1 - E)[:, None]).astype(np.int64)   # |X| < 2^(8S-1)
    d = np.zeros((S,) + x.shape, dtype=np.int64)
    r = X.copy()
    for t in range(S - 1, 0, -1):                 # low digits in [-128, 127]
        lo = ((r + 128) % 256) - 128
        d[t] = lo
        r = (r - lo) // 256
    d[0] = r                                      # leading digit in [-128, 128]
    return d, E


def _bf16_exact(v):
    f = v.astype(np.float32)
    return np.all((f.view(np.uint32) & 0xFFFF) == 0) and np.all(f.astype(np.float64) == v)


@pytest.mark.parametrize("S", [4, 5, 6])
def test_digits_reproduce_the_rows_and_are_bf16(S):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(16, 300)) * np.exp(rng.uniform(-20, 20, size=(16, 1)))
    d, E = _digits(x, S)
    assert d[0].min() >= -128 and d[0].max() <= 128
    assert d[1:].min() >= -128 and d[1:].max() <= 127
    back = sum(d[t].astype(np.float64) * 2.0 ** (-8 * t) for t in range(S)) * np.ldexp(1.0, E - 7)[:, None]
    assert np.max(np.abs(back - x) / np.ldexp(1.0, E)[:, None]) <= 2.0 ** (-8 * S + 1)
    for t in range(S):
        assert _bf16_exact(d[t].astype(np.float64) * 2.0 ** (-8 * t))


def test_leading_scales_are_exact_in_fp32_per_chunk():
    # worst case: every digit at its extreme, 256 stacked K per chunk
    S, K = 6, 256
    a = np.full((S, K), -128, dtype=np.int64)
    b = np.full((S, K), -128, dtype=np.int64)
    for s in range(S):                                    # scale s = t + u (0-based)
        pairs = [(t, s - t) for t in range(S) if 0 <= s - t < S]
        exact = sum(int(np.dot(a[t], b[u])) for t, u in pairs)
        f = np.float32(0.0)
        for k in range(K):                                # sequential FP32 accumulation
            for t, u in pairs:
                f = np.float32(f + np.float32(a[t, k] * b[u, k]))
        if len(pairs) <= 4:
            assert abs(exact) <= 2 ** 24 and int(f) == exact
        else:
            assert abs(exact) > 2 ** 24                   # the lower scales may round


@pytest.mark.parametrize("S,bound", [(4, 3e-8), (5, 1.5e-10), (6, 5e-13)])
def test_product_error_falls_with_each_slice(S, bound):
    rng = np.random.default_rng(5)
    M, N, K = 48, 40, 1024
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(K, N))
    da, ea = _digits(A, S)
    db, eb = _digits(B.T, S)
    C = np.zeros((M, N))
    for s in range(S):                                    # one accumulator per scale
        acc = np.zeros((M, N))
        for k0 in range(0, K, 256):                       # chunks read out in float-float (here FP64)
            part = np.zeros((M, N), dtype=np.float32)
            for t in range(S):
                u = s - t
                if 0 <= u < S:
                    part += (da[t][:, k0:k0 + 256].astype(np.float32) @ db[u][:, k0:k0 + 256].T.astype(np.float32))
            acc += part.astype(np.float64)
        C += acc * 2.0 ** (-8 * s)
    C *= np.ldexp(1.0, ea - 7)[:, None] * np.ldexp(1.0, eb - 7)[None, :]
    ref = A @ B
    err = np.max(np.abs(C - ref)) / np.max(np.abs(ref))
    assert err < bound
    if S < 6:
        assert err > bound / 2 ** 8                       # and not much better: the truncation is real
