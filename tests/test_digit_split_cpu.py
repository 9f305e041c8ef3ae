"""The error-free split behind the tensor-core contractions, emulated on the CPU in
IEEE single precision (numpy float32 rounds to nearest even, as the kernels'
`__fadd_rn`): the facts their exactness rests on, each checked on random values.

- Rounding to a fixed quantum q with the magic constant 1.5 * 2^23 * q gives a
  multiple of q, and the subtraction of the digit is exact.
- Six digits of a value below 1 in magnitude (a double-float hi + lo, the low word
  entering after the third digit) on the grid 2^(-7-8i) are exact bf16 numbers
  (at most 8 significant bits: the float32 pattern's low 16 bits are zero), each
  at most 128 of its quanta but the fourth, which takes the low word: at most 192
  (an integer below 256 still has 8 significant bits), and they rebuild the value
  to 2^-47 (the last digit's rounding, 2^-48, and the low word's entry, 2^-48).
- A sum of 256 products of such digits (the tile's K entries) stays below
  256 * 192^2 < 2^24 quanta, so float32 accumulation in any order is exact.
"""
import numpy as np

f32 = np.float32


def round_to(x, s):
    """(x + s) - s in float32, s = 1.5 * 2^23 * q."""
    return f32(f32(x + s) - s)


def split6(h, l, s0):
    """Six digits of the double-float h + l (float32 each) on the grid with magic s0."""
    d = []
    r = f32(h)
    for i in range(6):
        di = round_to(r, f32(s0 * 2.0 ** (-8 * i)))
        d.append(di)
        r = f32(r - di)
        if i == 2:
            r = f32(r + f32(l))
    return d


def is_bf16(x):
    return (np.asarray(x, dtype=np.float32).view(np.uint32) & 0xFFFF) == 0


def test_round_to_fixed_quantum_is_exact():
    rng = np.random.default_rng(0)
    for e in (-7, -15, -23, -31, -39, -47):
        q = 2.0**e
        s = f32(1.5 * 2**23 * q)
        x = (rng.uniform(-1, 1, 2000) * 2**22 * q).astype(np.float32)
        d = np.array([round_to(v, s) for v in x], dtype=np.float32)
        k = d.astype(np.float64) / q
        assert np.all(k == np.round(k))                      # multiples of q
        assert np.all(np.abs(x.astype(np.float64) - d) <= q / 2)  # nearest
        r = (x - d).astype(np.float64)                        # the subtraction is exact
        assert np.all(r == x.astype(np.float64) - d.astype(np.float64))


def test_six_digits_rebuild_a_double_float_value():
    rng = np.random.default_rng(1)
    s0 = f32(98304.0)  # 1.5 * 2^23 * 2^-7: the grid of values below 1 (Lambda / u_p)
    worst = 0.0
    for v in rng.uniform(-1, 1, 3000) * 2.0 ** rng.integers(-30, 1, 3000):
        h = f32(v)
        lo = f32(v - float(h))
        d = split6(h, lo, s0)
        for i, di in enumerate(d):
            q = 2.0 ** (-7 - 8 * i)
            assert is_bf16(di), (v, i, di)
            assert abs(float(di)) <= (192 if i == 3 else 128) * q
            assert float(di) / q == round(float(di) / q)
        rebuilt = sum(float(di) for di in d)
        worst = max(worst, abs(rebuilt - (float(h) + float(lo))))
    assert worst <= 2.0**-47, worst


def test_level_sums_of_256_digit_products_are_exact():
    rng = np.random.default_rng(2)
    for i, j in ((0, 0), (0, 1), (1, 1), (2, 3), (3, 3), (5, 0)):
        qa, qb = 2.0 ** (-7 - 8 * i), 2.0 ** (-7 - 8 * j)
        ba, bb = (192 if i == 3 else 128), (192 if j == 3 else 128)
        a = (rng.integers(-ba, ba + 1, 256) * qa).astype(np.float32)
        b = (rng.integers(-bb, bb + 1, 256) * qb).astype(np.float32)
        exact = sum(int(x) * int(y) for x, y in zip(np.round(a / qa), np.round(b / qb)))  # in quanta qa qb
        for order in (np.arange(256), rng.permutation(256), np.arange(256)[::-1]):
            acc = f32(0.0)
            for k in order:
                acc = f32(acc + f32(a[k] * b[k]))  # each product exact in float32
            assert float(acc) == exact * qa * qb
