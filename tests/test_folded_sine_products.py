"""The tensor-core form of the x sine transform (lines of 255 and of 127 points) written out in
numpy: the folded sine matrices (255) or the padded 128 x 128 matrix (127), the FP16 splitting with
the per-line power-of-two scale, the three products per term, and the -2i output convention,
checked against the sine transform computed directly. No GPU is involved; the CUDA kernels
themselves are compared with the FFT form and the oracle in the GPU tests (tests/test_gpu_dst_tc.py).

The transform of a line X_1..X_255 is Y_k = -2i sum_x X_x sin(pi k x / 256), k = 1..255 (the
output of the odd-extension FFT). With e_x = X_x - X_{256-x} and o_x = X_x + X_{256-x}:
  Y_{2k'}   = -2i sum_{x=1}^{127} e_x sin(pi k' x / 128),        k' = 1..127
  Y_{2k'+1} = -2i sum_{x=1}^{128} o_x sin(pi (2k'+1) x / 256),   o_128 = X_128."""
import numpy as np
import pytest

N_PTS = 255
L = N_PTS + 1          # 256
H = L // 2             # 128


def direct(X):
    """-2i times the sine transform, by the definition (float64)."""
    x = np.arange(1, N_PTS + 1)
    S = np.sin(np.pi * np.outer(x, x) / L)          # [k][x], both 1..255
    return -2j * (X @ S.T)


def matrices():
    """The two folded 128 x 128 matrices, scaled by 16 (row = output, column = input x - 1)."""
    r = np.arange(H)[:, None]
    q = np.arange(H)[None, :]
    x = q + 1
    kp = r + 1
    even = 16.0 * np.sin(np.pi * ((kp * x) % 256) / 128.0)
    even[(kp[:, 0] == 128), :] = 0.0
    even[:, (x[0] == 128)] = 0.0
    odd = 16.0 * np.sin(np.pi * (((2 * r + 1) * x) % 512) / 256.0)
    odd[:, H - 1] *= 0.5                            # the folded input at x = 128 is 2 X_128
    return even, odd


def fold(X):
    """e and o (complex, float32 arithmetic as the kernel), columns x = 1..128."""
    X = X.astype(np.complex64)
    a = X[:, :H]                                    # X_1 .. X_128
    b = X[:, ::-1][:, :H]                           # X_255 .. X_128 = X_{256-x}
    return (a - b).astype(np.complex64), (a + b).astype(np.complex64)


def veltkamp_f16(v):
    """v = hi + lo with hi of 11 significant bits (factor 2^13 + 1, float32 steps), both as FP16."""
    v = v.astype(np.float32)
    c = (v * np.float32(8193.0)).astype(np.float32)
    hi = (c - (c - v).astype(np.float32)).astype(np.float32)
    lo = (v - hi).astype(np.float32)
    return hi.astype(np.float16).astype(np.float64), lo.astype(np.float16).astype(np.float64)


def line_scale(X):
    """Per line: 2^sh with the largest |re|, |im| brought to [2^13, 2^14)."""
    m = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=1).astype(np.float32)
    E = np.where(m > 0, np.frexp(np.where(m > 0, m, 1.0))[1], 14)
    sh = np.clip(14 - E, -100, 100)
    return np.ldexp(np.float32(1.0), sh).astype(np.float32), sh


def products(B, A):
    """sum over K of hi hi + hi lo + lo hi for B [rows][K] (data) and A [outputs][K] (matrix)."""
    bh, bl = veltkamp_f16(B)
    ah, al = veltkamp_f16(A)
    return bh @ ah.T + bh @ al.T + bl @ ah.T


def tensor_core_form(X):
    even, odd = matrices()
    e, o = fold(X)
    sc, sh = line_scale(X)
    out = np.zeros((X.shape[0], N_PTS), dtype=np.complex128)
    for half, data, mat in ((0, e, even), (1, o, odd)):
        re = products((data.real * sc[:, None]).astype(np.float32), mat)
        im = products((data.imag * sc[:, None]).astype(np.float32), mat)
        z = (re + 1j * im) / (16.0 * np.ldexp(1.0, sh))[:, None]
        y = -2j * z
        if half == 0:
            out[:, 1::2] = y[:, :127]                # k = 2k', k' = 1..127 -> index 2k' - 1
        else:
            out[:, 0::2] = y                          # k = 2k' + 1, k' = 0..127 -> index 2k'
    return out


def lines(rng, n=24):
    X = rng.standard_normal((n, N_PTS)) + 1j * rng.standard_normal((n, N_PTS))
    X *= np.exp(rng.uniform(-30, 30, size=(n, 1)))  # lines of very different magnitudes
    X[3] = 0.0                                        # an empty line
    X[5, 1:] = 0.0                                    # a single nonzero value
    return X


def test_folded_matrices_are_the_sine_transform_exactly():
    """In float64 and without splitting, the folded form equals the direct transform."""
    rng = np.random.default_rng(1)
    X = lines(rng)
    even, odd = matrices()
    Xd = X.astype(np.complex128)
    a, b = Xd[:, :H], Xd[:, ::-1][:, :H]
    out = np.zeros_like(Xd)
    out[:, 1::2] = (-2j * ((a - b) @ even.T) / 16.0)[:, :127]
    out[:, 0::2] = -2j * ((a + b) @ odd.T) / 16.0
    ref = direct(Xd)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_split_products_reach_fp32_accuracy_per_line():
    rng = np.random.default_rng(2)
    X = lines(rng).astype(np.complex64)
    got = tensor_core_form(X)
    ref = direct(X.astype(np.complex128))
    for i in range(X.shape[0]):
        nrm = np.linalg.norm(ref[i])
        if nrm == 0.0:
            assert np.all(got[i] == 0.0)
            continue
        assert np.linalg.norm(got[i] - ref[i]) <= 5e-7 * nrm, i


def test_without_the_line_scale_fp16_fails():
    """The scale is needed: unscaled lines of magnitude ~1e-6 lose their low parts to FP16's range."""
    rng = np.random.default_rng(3)
    X = (1e-6 * (rng.standard_normal((4, N_PTS)) + 1j * rng.standard_normal((4, N_PTS)))).astype(np.complex64)
    even, odd = matrices()
    e, _ = fold(X)
    z = products(e.real.astype(np.float32), even) / 16.0
    ref = (e.real.astype(np.float64) @ even.T) / 16.0
    assert np.linalg.norm(z - ref) > 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("pieces", ["bf16"])
def test_bf16_pieces_are_not_enough(pieces):
    """With BF16 pieces (8 significant bits each) the error is ~1e-5, far above FP32's."""
    def bf16(v):
        b = v.astype(np.float32).view(np.uint32)
        r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        return r.view(np.float32).astype(np.float64)

    rng = np.random.default_rng(4)
    X = rng.standard_normal((8, N_PTS)).astype(np.float32)
    even, _ = matrices()
    e = (X[:, :H] - X[:, ::-1][:, :H]).astype(np.float32)
    eh = bf16(e)
    el = bf16(e - eh)
    mh = bf16(even)
    ml = bf16(even - mh)
    z = eh @ mh.T + eh @ ml.T + el @ mh.T
    ref = e.astype(np.float64) @ even.T
    assert np.linalg.norm(z - ref) > 1e-6 * np.linalg.norm(ref)


# ---- lines of 127 points: the sine matrix itself, padded to 128 x 128 (no fold) ----
N127 = 127


def direct127(X):
    x = np.arange(1, N127 + 1)
    S = np.sin(np.pi * np.outer(x, x) / (N127 + 1))
    return -2j * (X @ S.T)


def matrix127():
    """16 sin(pi k x / 128) for k, x = 1..127, row 128 and column 128 zero (row = k - 1, column = x - 1)."""
    k = np.arange(1, 129)[:, None]
    x = np.arange(1, 129)[None, :]
    S = 16.0 * np.sin(np.pi * ((k * x) % 256) / 128.0)
    S[127, :] = 0.0
    S[:, 127] = 0.0
    return S


def tensor_core_form127(X):
    S = matrix127()
    sc, sh = line_scale(X.astype(np.complex64))
    B = np.zeros((X.shape[0], 128), dtype=np.complex64)
    B[:, :N127] = X.astype(np.complex64)                  # the padding input x = 128 is zero
    re = products((B.real * sc[:, None]).astype(np.float32), S)
    im = products((B.imag * sc[:, None]).astype(np.float32), S)
    z = (re + 1j * im) / (16.0 * np.ldexp(1.0, sh))[:, None]
    return (-2j * z)[:, :N127]                            # output k = row + 1; row 128 is zero


def lines127(rng, n=24):
    X = rng.standard_normal((n, N127)) + 1j * rng.standard_normal((n, N127))
    X *= np.exp(rng.uniform(-30, 30, size=(n, 1)))
    X[2] = 0.0
    X[7, :-1] = 0.0                                       # only the last point (x = 127) nonzero
    return X


def test_padded_127_matrix_is_the_sine_transform_exactly():
    rng = np.random.default_rng(5)
    X = lines127(rng)
    S = matrix127()
    B = np.zeros((X.shape[0], 128), dtype=np.complex128)
    B[:, :N127] = X
    out = (-2j * (B @ S.T) / 16.0)[:, :N127]
    ref = direct127(X)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.all(S[127] == 0.0) and np.all(S[:, 127] == 0.0)


def test_split_products_127_reach_fp32_accuracy_per_line():
    rng = np.random.default_rng(6)
    X = lines127(rng).astype(np.complex64)
    got = tensor_core_form127(X)
    ref = direct127(X.astype(np.complex128))
    for i in range(X.shape[0]):
        nrm = np.linalg.norm(ref[i])
        if nrm == 0.0:
            assert np.all(got[i] == 0.0)
            continue
        assert np.linalg.norm(got[i] - ref[i]) <= 5e-7 * nrm, i


def test_127_transform_applied_twice_is_the_scaled_identity():
    """DST-I is its own inverse up to (n + 1) / 2: with the -2i convention, two transforms give
    -2 (n + 1) X = -256 X (the factor the 3D and 2D divisors account for)."""
    rng = np.random.default_rng(7)
    X = (rng.standard_normal((6, N127)) + 1j * rng.standard_normal((6, N127))).astype(np.complex64)
    Y = tensor_core_form127(X)
    Z = tensor_core_form127(Y.astype(np.complex64))
    assert np.linalg.norm(Z + 256.0 * X) <= 1e-6 * 256.0 * np.linalg.norm(X)
