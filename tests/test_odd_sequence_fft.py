"""The odd-sequence form of the sine transforms (the compiled line lengths of the spatial kernels):
the pass structure written out in numpy, with the kernels' radix schedule and index algebra, and
checked against the sine transform and the shifted solve computed directly. No GPU is involved;
the CUDA kernels themselves are compared with the oracle in the GPU parity tests.

Odd extension of a line x_1..x_n: length L = 2(n+1), x_0 = x_{L/2} = 0, x_{L-i} = -x_i. Its DFT is
odd (Y_{L-j} = -Y_j); the first pass (radix R, stride S = L/R) sends frequency j to block j mod R,
so only blocks q <= R/2 are formed and the inverse rebuilds the others from
z_{R-q}(n2) = -W_S^{n2} z_q(S - n2)."""
import numpy as np
import pytest


def npass(logL):
    return (logL + 3) // 4


def logradix(logL, i):
    n = npass(logL)
    return logL // n + (1 if i < logL % n else 0)


def fft_pos(j, logL):
    p, logLs = 0, logL
    for i in range(npass(logL)):
        lr = logradix(logL, i)
        q = j & ((1 << lr) - 1)
        j >>= lr
        logLs -= lr
        p += q << logLs
    return p


def dft(x, sign):
    R = len(x)
    r = np.arange(R)
    return np.array([np.sum(x * np.exp(sign * 2j * np.pi * r * q / R)) for q in range(R)])


def pass_ct(X, LR, forward, logL, logLs, rows):
    # one decimation-in-frequency pass (forward) or its conjugate transpose on the leading rows
    R, L = 1 << LR, 1 << logL
    logS = logLs - LR
    S = 1 << logS
    tw = np.exp(-2j * np.pi * np.arange(L) / L)
    for g in range(rows // R):
        n2 = g & (S - 1)
        base = ((g >> logS) << logLs) + n2
        idx = [base + r * S for r in range(R)]
        x = X[idx].copy()
        w = tw[((n2 * np.arange(R)) << (logL - logLs)) % L]
        X[idx] = dft(x, -1) * w if forward else dft(x * np.conj(w), 1)


def odd_forward_pass0(X, logL):
    L, R = 1 << logL, 1 << logradix(logL, 0)
    S, H = L // R, R // 2
    tw = np.exp(-2j * np.pi * np.arange(L) / L)
    out = {}
    for n2 in range(S):                      # inputs: rows 0..L/2 only
        a = np.array([X[n2 + S * r] if r < H else -X[S * (R - r) - n2] for r in range(R)])
        out[n2] = dft(a, -1) * tw[(n2 * np.arange(R)) % L]
    for n2, A in out.items():                # blocks 0..R/2 only
        for q in range(H + 1):
            X[n2 + S * q] = A[q]


def odd_inverse_pass0(X, logL):
    L, R = 1 << logL, 1 << logradix(logL, 0)
    S, H = L // R, R // 2
    tw = np.exp(-2j * np.pi * np.arange(L) / L)
    out = {}
    for n2 in range(S):
        m2 = (S - n2) % S
        y = np.zeros(R, complex)
        for q in range(H + 1):
            y[q] = X[S * q + n2] * np.conj(tw[(n2 * q) % L])
        for q in range(1, H):
            y[R - q] = -X[S * q + m2] * tw[(n2 * q) % L]
        out[n2] = dft(y, 1)
    for n2, x in out.items():
        for r in range(H):
            X[n2 + S * r] = x[r]


def odd_transform(x, logL, divisor=None):
    """op 0 (divisor None): -2i D x at frequencies 1..n; op 1: the shifted solve (2i D)(-2i D x)/d."""
    L = 1 << logL
    n = L // 2 - 1
    R0 = 1 << logradix(logL, 0)
    rows = L // 2 + L // R0
    X = np.full(rows, np.nan + 0j)           # rows beyond the extension start undefined
    X[0], X[1:n + 1], X[n + 1] = 0, x, 0
    odd_forward_pass0(X, logL)
    logLs = logL - logradix(logL, 0)
    for P in range(1, npass(logL)):
        lr = logradix(logL, P)
        pass_ct(X, lr, True, logL, logLs, rows)
        logLs -= lr
    if divisor is None:
        return np.array([X[fft_pos(p, logL)] if p % R0 <= R0 // 2 else -X[fft_pos(L - p, logL)]
                         for p in range(1, n + 1)])
    for pos in range(rows):                  # the divide, at each formed row's frequency
        j = int(np.where([fft_pos(f, logL) == pos for f in range(L)])[0][0])
        f = j if j <= n + 1 else L - j
        X[pos] = 0 if f in (0, n + 1) else X[pos] / divisor[f]
    logLs = 0
    for P in range(npass(logL) - 1, 0, -1):
        lr = logradix(logL, P)
        logLs += lr
        pass_ct(X, lr, False, logL, logLs, rows)
    odd_inverse_pass0(X, logL)
    return X[1:n + 1]


@pytest.mark.parametrize("logL", [7, 8, 9, 10])
def test_odd_sequence_passes_give_the_sine_transform_and_the_solve(logL):
    L = 1 << logL
    n = L // 2 - 1
    rng = np.random.default_rng(logL)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    D = np.sin(np.pi * np.outer(np.arange(1, n + 1), np.arange(1, n + 1)) / (n + 1))
    y = odd_transform(x, logL)
    assert np.abs(y - (-2j * D @ x)).max() <= 1e-12 * np.abs(D @ x).max() * n
    d = 3.0 + rng.standard_normal(n + 2) + 1j * rng.standard_normal(n + 2)
    q = odd_transform(x, logL, divisor=d)
    ref = (2j * D) @ ((-2j * D @ x) / d[1:n + 1])
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max() * n


@pytest.mark.parametrize("logL", [7, 8, 9, 10, 11, 12])
def test_first_pass_pairs_touch_disjoint_rows(logL):
    # the in-place first pass pairs n2 with S - n2 (0 with S/2): between them the pair reads exactly
    # the rows it writes, so pairs never touch another pair's rows, and together they form every
    # row of blocks 0..R/2
    L, R = 1 << logL, 1 << logradix(logL, 0)
    S, H = L // R, R // 2
    rows = (H + 1) * S
    seen = set()
    for t in range(S // 2):
        na, nb = (0, S // 2) if t == 0 else (t, S - t)
        reads = ({S * u for u in range(1, H)} | {S // 2 + S * u for u in range(H)} if t == 0 else
                 {t + S * u for u in range(H)} | {S * s - t for s in range(1, H + 1)})
        writes = {na + S * q for q in range(H + 1)} | {nb + S * q for q in range(H + 1)}
        assert reads <= writes and max(reads) <= L // 2 and max(writes) < rows
        assert not (writes & seen)
        seen |= writes
    assert seen == set(range(rows))
