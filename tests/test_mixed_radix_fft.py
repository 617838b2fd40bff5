"""CPU test of the pass structure of the shared-memory FFT for lengths L = 2^a 5^b (csrc/fft.cuh:
b radix-5 passes, then the power-of-two schedule; in-place decimation in frequency; the forward
leaves a digit-reversed spectrum, position fft_pos(j) holding frequency j, that the inverse
consumes). The passes, the twiddle indices and the position map are written out in numpy with the
kernels' index arithmetic and compared with numpy's FFT."""
import numpy as np
import pytest


def npass_pow2(P, maxlog):
    e = P.bit_length() - 1
    return (e + maxlog - 1) // maxlog


def radix_pow2(P, i, maxlog):
    e = P.bit_length() - 1
    np_ = (e + maxlog - 1) // maxlog
    return 1 << (e // np_ + (1 if i < e % np_ else 0))


def schedule(L, maxlog=4):
    b, P = 0, L
    while P % 5 == 0:
        P //= 5
        b += 1
    return [5] * b + [radix_pow2(P, i, maxlog) for i in range(npass_pow2(P, maxlog) if P > 1 else 0)]


def pos(j, L, maxlog=4):
    p, Ls = 0, L
    for R in schedule(L, maxlog):
        q = j % R
        j //= R
        Ls //= R
        p += q * Ls
    return p


def forward(x, maxlog=4):
    L = len(x)
    X = x.astype(complex).copy()
    tw = np.exp(-2j * np.pi * np.arange(L) / L)
    Ls = L
    for R in schedule(L, maxlog):
        S, tstep = Ls // R, L // Ls
        for g in range(L // R):
            blk, n2 = divmod(g, S)
            base = blk * Ls + n2
            idx = base + S * np.arange(R)
            v = X[idx]
            y = np.array([np.sum(v * np.exp(-2j * np.pi * np.arange(R) * q / R)) for q in range(R)])
            y[1:] *= tw[n2 * np.arange(1, R) * tstep]
            X[idx] = y
        Ls //= R
    return X


def inverse(X, maxlog=4):
    L = len(X)
    X = X.copy()
    tw = np.exp(-2j * np.pi * np.arange(L) / L)
    sched = schedule(L, maxlog)
    Ls = 1
    for R in reversed(sched):
        Ls *= R
        S, tstep = Ls // R, L // Ls
        for g in range(L // R):
            blk, n2 = divmod(g, S)
            idx = blk * Ls + n2 + S * np.arange(R)
            v = X[idx].copy()
            v[1:] *= np.conj(tw[n2 * np.arange(1, R) * tstep])
            X[idx] = np.array([np.sum(v * np.exp(2j * np.pi * np.arange(R) * q / R)) for q in range(R)])
    return X


@pytest.mark.parametrize("L", [10, 20, 40, 100, 200, 250, 2000])
@pytest.mark.parametrize("maxlog", [3, 4])
def test_mixed_radix_passes_match_numpy(L, maxlog):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    X = forward(x, maxlog)
    perm = np.array([pos(j, L, maxlog) for j in range(L)])
    assert sorted(perm) == list(range(L))              # a permutation of the rows
    ref = np.fft.fft(x)
    assert np.max(np.abs(X[perm] - ref)) <= 1e-10 * np.max(np.abs(ref))
    # the inverse takes the permuted spectrum back to L x the data in natural order
    assert np.max(np.abs(inverse(X, maxlog) / L - x)) <= 1e-12 * np.max(np.abs(x))


def test_twiddle_indices_stay_below_L():
    for L in (100, 200, 2000, 4000):
        Ls = L
        for R in schedule(L):
            S = Ls // R
            assert (S - 1) * (R - 1) * (L // Ls) < L
            Ls //= R
