"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check ties the oracle to something other than itself: the paper's own
matrices (Sec. 3, Eq. 4) multiplied out, the printed worked example (Sec. 4),
the operation counts (Sec. 5, Eqs. 6-7), closed forms of the DFT, a library FFT
and brute-force dense products.  The last test plants plausible mistakes in
the oracle's output and checks that the pins catch each one.
"""
import os

import numpy as np
import pytest

from oracle import matrices as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example_n8.txt")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _cplx(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def _per_window_fft(x, m):
    """Library FFT (numpy pocketfft) applied window by window: Eq. 1 per level."""
    return np.stack([np.fft.fft(x.reshape(-1, 1 << i), axis=1).reshape(-1)
                     for i in range(1, m + 1)])


def _read_golden():
    sections, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line[1:-1]
                sections[cur] = []
            else:
                sections[cur].append(line.split())
    return sections


def _diag_from_tokens(tokens):
    vals = []
    for t in tokens:
        if t == "1":
            vals.append(1.0 + 0j)
        else:
            L, e = t.split(":")
            vals.append(complex(M.w(int(L), int(e))))
    return np.diag(np.array(vals))


# ----------------------------------------------------------- Sec. 3 / Eq. 4

@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_eq4_product_equals_eq1(m):
    """The rationalised factorisation (Eq. 4) multiplies out to Eq. 1."""
    np.testing.assert_allclose(M.eq4(m), M.eq1(m), atol=1e-12, rtol=0)


@pytest.mark.parametrize("m", [2, 3, 4])
def test_eq1_printed_identity_is_not_square(m):
    """Eq. 1 as printed (I_{2^{m-1}}) gives blocks that are not N x N for i > 1;
    the reading I_{2^{m-i}} is the one that does."""
    N = 1 << m
    for i in range(2, m + 1):
        assert M.eq1_block_literal(m, i).shape != (N, N)
        assert np.kron(M.I(1 << (m - i)), M.E(1 << i)).shape == (N, N)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_eq1_matrix_matches_oracle(oracle, m):
    x = _cplx(_rng(m), 1 << m)
    y = (M.eq1(m) @ x).reshape(m, -1)
    np.testing.assert_allclose(oracle.forward(x, "direct"), y, atol=1e-12, rtol=0)
    np.testing.assert_allclose(oracle.forward(x, "fft"), y, atol=1e-12, rtol=0)


# --------------------------------------------------- Sec. 4 worked example

def test_worked_example_permutations():
    g = _read_golden()
    for name, i in (("T2", 1), ("T4", 2), ("T8", 3)):
        printed = np.array(g[name], dtype=float)
        np.testing.assert_array_equal(printed, M.T(i).real)
    G = M.Gamma(3)
    assert G.shape == (24, 24)
    np.testing.assert_array_equal(G[16:, 16:].real, np.array(g["T8"], dtype=float))


def test_worked_example_twiddles():
    g = _read_golden()
    np.testing.assert_allclose(M.Dtilde(3), _diag_from_tokens(g["Dtilde_8_level3"][0]), atol=1e-15)
    np.testing.assert_allclose(M.Dtilde(2), _diag_from_tokens(g["Dtilde_4_level2"][0]), atol=1e-15)
    np.testing.assert_allclose(M.Dtilde(1), _diag_from_tokens(g["Dtilde_2_level1"][0]), atol=1e-15)
    np.testing.assert_allclose(M.W(3, 1), _diag_from_tokens(g["W_4_j1_level3"][0]), atol=1e-15)
    np.testing.assert_allclose(M.W(3, 2), _diag_from_tokens(g["W_4_j2_level3"][0]), atol=1e-15)
    # S_4^(1) = H_2 (x) I_2 and S_4^(2) = I_2 (x) H_2 (Sec. 4)
    np.testing.assert_array_equal(M.S(3, 1), np.kron(M.H2, M.I(2)))
    np.testing.assert_array_equal(M.S(3, 2), np.kron(M.I(2), M.H2))
    # R_2^(2) = W_2^(1) S_2^(1) = (I_1 (+) w_2^0) H_2 = H_2
    np.testing.assert_allclose(M.R(2), M.H2, atol=1e-15)


def test_worked_example_shapes():
    """Matrix sizes of Eq. 5 (N = 8): P^(1) 24x8, P^(i) 32x24, A^(i) 24x32."""
    assert M.P1(3).shape == (24, 8)
    assert M.Pi(3, 2).shape == (32, 24) and M.Pi(3, 3).shape == (32, 24)
    assert M.A1(3).shape == (24, 24)
    assert M.Ai(3, 2).shape == (24, 32) and M.Ai(3, 3).shape == (24, 32)
    assert M.D(3, 2).shape == (24, 24) and M.F(3, 3).shape == (24, 24)


def test_R_is_bit_reversed_dft():
    """F's core R^(i) is a DFT of size 2^(i-1) with bit-reversed output."""
    for i in range(2, 7):
        h = 1 << (i - 1)
        np.testing.assert_allclose(M.R(i), M.T(i - 1).T @ M.E(h), atol=1e-12)


# ---------------------------------------------------------- Sec. 5 counts

@pytest.mark.parametrize("m", list(range(1, 21)))
def test_operation_counts_eq6_eq7(oracle, m):
    _, c = oracle.rationalized(m=m, compute=False)
    for i in range(1, m + 1):
        mul, mul_nt, add = (int(v) for v in c[i - 1])
        # Eq. 6: beta^(i) = (i+1) 2^(m-2); Eq. 7: 0 at i = 1, else (i-2) 2^(m-2)
        assert 4 * mul == (i + 1) * 2 ** m
        assert 4 * mul_nt == (0 if i == 1 else (i - 2) * 2 ** m)
        assert add == 2 * mul
    tot, tot_nt = int(c[:, 0].sum()), int(c[:, 1].sum())
    # beta = m(m+3) 2^(m-3), beta~ = (m-1)(m-2) 2^(m-3)  (Sec. 5)
    assert 8 * tot == m * (m + 3) * 2 ** m
    assert 8 * tot_nt == (m - 1) * (m - 2) * 2 ** m
    assert int(c[:, 2].sum()) == 2 * tot


def test_operation_counts_computed_equals_counted(oracle):
    x = _cplx(_rng(7), 1 << 9)
    _, c1 = oracle.rationalized(x)
    _, c2 = oracle.rationalized(m=9, compute=False)
    np.testing.assert_array_equal(c1, c2)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 10, 13])
def test_rationalized_reaches_definition(oracle, m):
    x = _cplx(_rng(100 + m), 1 << m)
    y, _ = oracle.rationalized(x)
    ref = oracle.forward(x, "direct" if m <= 10 else "fft")
    scale = np.linalg.norm(x) * np.sqrt(1 << m)
    assert np.abs(y - ref).max() <= 1e-13 * scale


# ------------------------------------------------------- library / brute force

@pytest.mark.parametrize("m", [1, 2, 3, 6, 9, 12])
def test_oracle_matches_library_fft(oracle, m):
    x = _cplx(_rng(200 + m), 1 << m)
    ref = _per_window_fft(x, m)
    scale = np.linalg.norm(x) * np.sqrt(1 << m)
    for method in ("direct", "fft"):
        assert np.abs(oracle.forward(x, method) - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("m", [13, 15])
def test_oracle_fft_path_large(oracle, m):
    x = _cplx(_rng(300 + m), 1 << m)
    ref = _per_window_fft(x, m)
    scale = np.linalg.norm(x) * np.sqrt(1 << m)
    assert np.abs(oracle.forward(x, "fft") - ref).max() <= 1e-12 * scale


def test_direct_and_fft_agree_to_1e12(oracle):
    x = _cplx(_rng(5), 1 << 12)
    yd, yf = oracle.forward(x, "direct"), oracle.forward(x, "fft")
    for i in range(12):
        assert np.linalg.norm(yd[i] - yf[i]) <= 1e-12 * np.linalg.norm(yd[i])


def test_bin_and_level(oracle):
    x = _cplx(_rng(9), 1 << 11)
    y = oracle.forward(x, "direct")
    for (i, p) in [(1, 0), (1, 2047), (5, 33), (11, 0), (11, 1), (11, 2047), (7, 1000)]:
        assert abs(oracle.bin_value(x, i, p) - y[i - 1, p]) <= 1e-11
    for i in (1, 6, 11):
        np.testing.assert_allclose(oracle.forward_level(x, i), y[i - 1], atol=1e-11)


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("m", [3, 8])
def test_impulse(oracle, m):
    N = 1 << m
    for p in (0, 1, 5, N - 1):
        x = np.zeros(N, complex)
        x[p] = 1.0
        y = oracle.forward(x)
        for i in range(1, m + 1):
            L = 1 << i
            w, off = divmod(p, L)
            k = np.arange(L)
            expect = np.zeros(N, complex)
            expect[w * L:(w + 1) * L] = np.exp(-2j * np.pi * off * k / L)
            np.testing.assert_allclose(y[i - 1], expect, atol=1e-12)
            if off == 0:  # impulse at a window start: all-ones spectrum
                np.testing.assert_allclose(y[i - 1][w * L:(w + 1) * L], 1.0, atol=1e-12)


def test_constant(oracle):
    m, c = 7, 0.75 - 0.25j
    y = oracle.forward(np.full(1 << m, c))
    for i in range(1, m + 1):
        L = 1 << i
        blk = y[i - 1].reshape(-1, L)
        np.testing.assert_allclose(blk[:, 0], c * L, atol=1e-12)
        np.testing.assert_allclose(blk[:, 1:], 0, atol=1e-12)


def test_on_bin_cosine(oracle):
    """cos(2 pi n / 2^j): lines of height 2^(i-1) at k = 2^(i-j), 2^i - 2^(i-j)."""
    m, j = 9, 4
    n = np.arange(1 << m)
    y = oracle.forward(np.cos(2 * np.pi * n / (1 << j)).astype(complex))
    for i in range(j, m + 1):
        L = 1 << i
        f = 1 << (i - j)
        expect = np.zeros(L, complex)
        expect[f] += L / 2
        expect[L - f] += L / 2
        blk = y[i - 1].reshape(-1, L)
        np.testing.assert_allclose(blk, np.broadcast_to(expect, blk.shape), atol=1e-9)


def test_parseval_per_window(oracle):
    m = 10
    x = _cplx(_rng(11), 1 << m)
    y = oracle.forward(x)
    for i in range(1, m + 1):
        L = 1 << i
        lhs = (np.abs(y[i - 1].reshape(-1, L)) ** 2).sum(axis=1)
        rhs = L * (np.abs(x.reshape(-1, L)) ** 2).sum(axis=1)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_even_bins_are_child_sums(oracle):
    """Eq. 2: Y_i[2k] of a window = sum of its two children's Y_{i-1}[k]."""
    m = 9
    x = _cplx(_rng(12), 1 << m)
    y = oracle.forward(x)
    for i in range(2, m + 1):
        L, h = 1 << i, 1 << (i - 1)
        par = y[i - 1].reshape(-1, L)
        ch = y[i - 2].reshape(-1, 2, h)
        np.testing.assert_allclose(par[:, 0::2], ch[:, 0] + ch[:, 1], atol=1e-10)


def test_odd_bins_are_fft_of_twiddled_difference(oracle):
    """Eq. 3 with D and F: Y_i[2k+1] = DFT_h((a - b) w_{2^i}^n)[k]."""
    m = 8
    x = _cplx(_rng(13), 1 << m)
    y = oracle.forward(x)
    for i in range(1, m + 1):
        L, h = 1 << i, 1 << (i - 1)
        xw = x.reshape(-1, L)
        z = (xw[:, :h] - xw[:, h:]) * np.exp(-2j * np.pi * np.arange(h) / L)
        np.testing.assert_allclose(y[i - 1].reshape(-1, L)[:, 1::2], np.fft.fft(z, axis=1), atol=1e-10)


def test_linearity(oracle):
    rng = _rng(14)
    a, b = _cplx(rng, 256), _cplx(rng, 256)
    al, be = 0.3 - 1.1j, -2.0 + 0.5j
    np.testing.assert_allclose(oracle.forward(al * a + be * b),
                               al * oracle.forward(a) + be * oracle.forward(b), atol=1e-11)


# ----------------------------------------------------------------- adjoint

@pytest.mark.parametrize("m", [1, 2, 4, 6])
def test_adjoint_is_conjugate_transpose(oracle, m):
    g = _cplx(_rng(400 + m), m << m).reshape(m, -1)
    dense = M.eq1(m).conj().T @ g.reshape(-1)
    for method in ("direct", "fft"):
        np.testing.assert_allclose(oracle.adjoint(g, method), dense, atol=1e-12)


@pytest.mark.parametrize("m", [5, 10, 14])
def test_adjoint_dot_product(oracle, m):
    rng = _rng(500 + m)
    x = _cplx(rng, 1 << m)
    g = _cplx(rng, m << m).reshape(m, -1)
    lhs = np.vdot(g, oracle.forward(x))          # <g, M x>
    rhs = np.vdot(oracle.adjoint(g), x)          # <M^H g, x>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-9


def test_adjoint_finite_differences(oracle):
    """Real loss L = sum_i w_i ||Y_i - T_i||^2; dL/dRe x + j dL/dIm x = 2 M^H (w (Y - T))."""
    m = 6
    rng = _rng(600)
    x = _cplx(rng, 1 << m)
    T = _cplx(rng, m << m).reshape(m, -1)
    wts = 2.0 ** -np.arange(1, m + 1)

    def loss(xx):
        return float((wts[:, None] * np.abs(oracle.forward(xx) - T) ** 2).sum())

    grad = oracle.adjoint(2 * wts[:, None] * (oracle.forward(x) - T))
    eps = 1e-6
    for p in range(1 << m):
        for unit in (1.0, 1j):
            e = np.zeros(1 << m, complex)
            e[p] = unit * eps
            fd = (loss(x + e) - loss(x - e)) / (2 * eps)
            an = grad[p].real if unit == 1.0 else grad[p].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


# ----------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(oracle):
    """Plausible oracle bugs, planted in its output, each fail a pin above."""
    m = 6
    x = _cplx(_rng(700), 1 << m)
    good = oracle.forward(x)
    ref = (M.eq1(m) @ x).reshape(m, -1)

    def bad_sign(y):        # exp(+j...) instead of exp(-j...)
        return np.stack([np.fft.ifft(x.reshape(-1, 1 << i), axis=1).reshape(-1) * (1 << i)
                         for i in range(1, m + 1)])

    def bad_order(y):       # bins left in bit-reversed order (Gamma dropped)
        out = y.copy()
        for i in range(1, m + 1):
            L = 1 << i
            perm = [M.bitrev(k, i) for k in range(L)]
            out[i - 1] = y[i - 1].reshape(-1, L)[:, perm].reshape(-1)
        return out

    def bad_level_shift(y):  # levels stored off by one
        return np.roll(y, 1, axis=0)

    def bad_odd_sign(y):    # b - a instead of a - b in V (Eq. 3)
        out = y.copy()
        for i in range(1, m + 1):
            out[i - 1].reshape(-1, 1 << i)[:, 1::2] *= -1
        return out

    assert np.abs(good - ref).max() < 1e-12
    for mutate in (bad_sign, bad_order, bad_level_shift, bad_odd_sign):
        assert np.abs(mutate(good) - ref).max() > 1e-3, mutate.__name__
