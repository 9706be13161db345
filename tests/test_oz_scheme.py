"""The arithmetic of the FP64 emulation (TCORR_FP64_OZ) modelled in numpy,
independently of the GPU: 5 signed 7-bit slices under a power-of-two scale,
the 15 slice pairs with i + j <= 6 grouped by weight, blocks of 8 K chunks of
32.  Checks the three facts the kernel relies on: every slice is an integer
exact in BF16, every block's weight sum stays below 2^24 (so FP32
accumulation is exact), and the recombined dot product is within the slice
truncation bound of the FP64 one."""
import numpy as np

S, BETA, KCH, KB = 5, 7, 32, 8


def slices(x, e):
    y = x * 2.0 ** (-e)
    out = []
    for _ in range(S):
        y = y * 2.0 ** BETA
        a = np.rint(y)
        y = y - a
        out.append(a)
    return np.array(out)          # [S][...]


def bf16_exact(a):
    # integers with |a| <= 256 have at most 8 significant bits
    return np.all(np.abs(a) <= 256) and np.all(a == np.rint(a))


def test_slices_exact_and_block_sums_below_2_24():
    rng = np.random.default_rng(0)
    K = 1056                                  # 2 v_pad + 2 o_pad at v = 450, o = 50
    x = rng.normal(size=(64, K)) * rng.choice([1.0, 1e-3, 1e-6], size=(64, K))
    y = rng.normal(size=(48, K))
    ex = int(np.frexp(np.abs(x).max())[1])
    ey = int(np.frexp(np.abs(y).max())[1])
    ax, ay = slices(x, ex), slices(y, ey)
    assert bf16_exact(ax) and bf16_exact(ay)
    assert np.abs(ax[0]).max() <= 128 and np.abs(ax[1:]).max() <= 64
    worst = 0.0
    for k0 in range(0, K, KCH * KB):
        sl = slice(k0, min(K, k0 + KCH * KB))
        for t in range(S):
            P = sum(ax[i][:, sl] @ ay[t - i][:, sl].T for i in range(t + 1))
            worst = max(worst, np.abs(P).max())
    assert worst < 2 ** 24


def test_recombination_error_bound():
    rng = np.random.default_rng(1)
    K = 512
    x = rng.normal(size=(32, K))
    y = rng.normal(size=(16, K))
    ex = int(np.frexp(np.abs(x).max())[1])
    ey = int(np.frexp(np.abs(y).max())[1])
    ax, ay = slices(x, ex), slices(y, ey)
    total = np.zeros((32, 16), dtype=np.int64)
    for k0 in range(0, K, KCH * KB):
        sl = slice(k0, k0 + KCH * KB)
        for t in range(S):
            P = sum(ax[i][:, sl] @ ay[t - i][:, sl].T for i in range(t + 1))
            total += P.astype(np.int64) * (1 << (BETA * (S - 1 - t)))
    u = total.astype(np.float64) * 2.0 ** (ex + ey - BETA * (S + 1))
    ref = x @ y.T
    # each operand is represented to 2^(e - beta S - 1); dropped pairs add < 2^(e_x + e_y - 7*7) per term
    bound = K * (2.0 ** (ex - BETA * S - 1) * np.abs(y).max() + 2.0 ** (ey - BETA * S - 1) * np.abs(x).max()
                 + 2.0 ** (ex + ey - BETA * (S + 2)) * S * S * 128 * 128)
    assert np.abs(u - ref).max() <= bound
    assert np.abs(u - ref).max() / np.abs(ref).max() < 1e-9
