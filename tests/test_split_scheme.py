"""The hi + lo split-precision arithmetic of the tensor-core paths, modelled
exactly on the host (no GPU): x = hi + lo + r with hi = round(x) and
lo = round(x - hi) to the significand of BF16 (8 bits) or TF32 (11 bits),
round to nearest even.

The product x y is approximated by hi hi' + hi lo' + lo hi' (three products,
the (T) contractions) or with lo lo' added (four products, RI-MP2).  For a
sum of squares -- the same-index elements g_aa = sum_gamma C_ai^2 of the
RI-MP2 pairs i = j -- the dropped lo lo' = lo^2 is one-signed, so the
three-product g_aa is biased low by the mean of lo^2 / x^2.  Rounding to s
significant bits leaves a relative error uniform within +-2^-s / m for the
significand m in [0.5, 1), so that mean lies between 4^-(s+1) / 3 and
4^-s / 3: 1.3e-6 to 5.1e-6 in BF16 (2.7e-6 for normal values), enough to
move E_MP2 by more than 1e-6 when the same-index terms carry much of it.
The fourth product removes the bias; what remains is the residual r, whose
sign is random."""
import numpy as np


def round_sig(x, bits):
    """x rounded to `bits` significant bits, round to nearest even (no
    overflow or subnormal handling: the test values are O(0.1))."""
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def split(x, bits):
    hi = round_sig(x, bits)
    lo = round_sig(x - hi, bits)
    return hi, lo


def gram(hi, lo, four):
    g = hi.T @ hi + hi.T @ lo + lo.T @ hi
    if four:
        g = g + lo.T @ lo
    return g


def test_round_sig_is_bf16_and_tf32_rounding():
    # 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1)
    assert round_sig(np.array([1.0 + 2.0 ** -8]), 8)[0] == 1.0
    assert round_sig(np.array([1.0 + 3 * 2.0 ** -9]), 8)[0] == 1.0 + 2.0 ** -7
    # 11 significant bits (TF32: 10 stored + the implicit one)
    assert round_sig(np.array([1.0 + 2.0 ** -11]), 11)[0] == 1.0
    assert round_sig(np.array([1.0 + 3 * 2.0 ** -12]), 11)[0] == 1.0 + 2.0 ** -10
    x = np.random.default_rng(0).normal(size=1000)
    hi, lo = split(x, 8)
    assert np.all(np.abs(x - hi) <= 2.0 ** -8 * np.abs(x))        # half an ulp of 8 bits
    assert np.all(np.abs(x - hi - lo) <= 2.0 ** -16 * np.abs(x))  # residual: two roundings


def test_three_products_bias_sums_of_squares_four_do_not():
    rng = np.random.default_rng(7)
    naux, v = 420, 300
    C = rng.normal(0.0, 0.1, size=(naux, v))       # C^gamma_a for one occupied index
    exact = C.T @ C
    d = np.diag(exact)
    for bits in (8, 11):
        lo_min, lo_max = 4.0 ** -(bits + 1) / 3, 4.0 ** -bits / 3
        hi, lo = split(C, bits)
        r3 = (np.diag(gram(hi, lo, False)) - d) / d
        r4 = (np.diag(gram(hi, lo, True)) - d) / d
        # three products: every g_aa low, by the mean of lo^2 / x^2
        assert np.all(r3 < 0)
        assert lo_min < -np.mean(r3) < lo_max
        # four products: no systematic part left (mean well below the spread)
        assert abs(np.mean(r4)) < 0.1 * lo_min
        assert abs(np.mean(r4)) < 3.0 * np.std(r4) / np.sqrt(v) + 1e-15
    # BF16: the bias is above 1e-6 (2.7e-6 here), TF32 below 1e-7
    hi, lo = split(C, 8)
    assert 1e-6 < -np.mean((np.diag(gram(hi, lo, False)) - d) / d) < 5e-6
    hi, lo = split(C, 11)
    assert -np.mean((np.diag(gram(hi, lo, False)) - d) / d) < 1e-7


def test_energy_of_an_i_eq_j_pair():
    """E_J-like sum -2 sum_ab g_ab^2 / eps of one i = j pair: with three BF16
    products its relative error is one-signed and above 1e-6 when the
    same-index terms dominate (few pairs, large naux); with four it is not."""
    rng = np.random.default_rng(3)
    naux, v = 420, 300
    C = rng.normal(0.0, 0.1, size=(naux, v))
    ev = np.sort(rng.uniform(0.1, 5.0, size=v))
    eps = ev[:, None] + ev[None, :] + 2 * 1.15       # e_a + e_b - 2 e_i, e_i ~ -1.15
    exact = -2.0 * np.sum((C.T @ C) ** 2 / eps)
    hi, lo = split(C, 8)
    e3 = -2.0 * np.sum(gram(hi, lo, False) ** 2 / eps)
    e4 = -2.0 * np.sum(gram(hi, lo, True) ** 2 / eps)
    rel3, rel4 = (e3 - exact) / exact, (e4 - exact) / exact
    assert rel3 < -1e-6                              # |E| too small, beyond the 1e-6 target
    assert abs(rel4) < 1e-7
