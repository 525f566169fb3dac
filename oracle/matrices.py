"""Dense matrices of the paper's Sec. 2-4, built literally -- TEST INFRASTRUCTURE.

Each function builds one matrix of Andreatto & Cariow (arXiv:1507.02525) as a
dense complex128 numpy array, from the paper's Kronecker-product / direct-sum
formulas, for small m (the matrices are mN x mN).  The tests multiply them out
and compare the product of Eq. 4 with the definition, Eq. 1.  Nothing here is
used by the product path.

Readings of garbled or ambiguous passages (each one pinned by a test):
  * Eq. 1 prints I_{2^{m-1}}; it is read as I_{2^{m-i}} (N/2^i windows at
    level i) -- the printed form does not give an N x N block for i > 1.
  * T_{2^i} (Sec. 3): t_{k, <k>} = 1 with <.> the bit reversal over i bits;
    the printed T_4 and T_8 of Sec. 4 fix this reading.
  * In A^(i), U acts on the duplicated level-(i-1) block and V on the i-th
    copy of X (Sec. 3, P^(i) and A^(i) dimensions).
"""
from __future__ import annotations

import numpy as np


def w(L: int, e) -> np.ndarray:
    """Twiddle factor w_L^e = exp(-j 2 pi e / L) (Sec. 3, after D~)."""
    return np.exp(-2j * np.pi * np.asarray(e, dtype=np.float64) / L)


def I(n: int) -> np.ndarray:
    return np.eye(n, dtype=np.complex128)


def Z(r: int, c: int) -> np.ndarray:
    return np.zeros((r, c), dtype=np.complex128)


def ones(r: int, c: int) -> np.ndarray:
    return np.ones((r, c), dtype=np.complex128)


H2 = np.array([[1, 1], [1, -1]], dtype=np.complex128)


def dsum(*blocks) -> np.ndarray:
    """Direct sum (block diagonal) of possibly rectangular blocks."""
    blocks = [b for b in blocks if b.size or b.shape != (0, 0)]
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    out = np.zeros((rows, cols), dtype=np.complex128)
    r = c = 0
    for b in blocks:
        out[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return out


def E(L: int) -> np.ndarray:
    """DEF matrix E_L, element (n, k) = w_L^{n k} (Sec. 2)."""
    n = np.arange(L)
    return w(L, np.outer(n, n) % L)


def P_def(m: int) -> np.ndarray:
    """P_{mN x N} = 1_{m x 1} (x) I_N (Sec. 2)."""
    return np.kron(ones(m, 1), I(1 << m))


def eq1(m: int) -> np.ndarray:
    """Eq. 1 with I_{2^{m-i}}: [(+)_i (I_{2^{m-i}} (x) E_{2^i})] P."""
    blocks = [np.kron(I(1 << (m - i)), E(1 << i)) for i in range(1, m + 1)]
    return dsum(*blocks) @ P_def(m)


def eq1_block_literal(m: int, i: int) -> np.ndarray:
    """Level-i block of Eq. 1 exactly as printed, I_{2^{m-1}} (x) E_{2^i}."""
    return np.kron(I(1 << (m - 1)), E(1 << i))


def P1(m: int) -> np.ndarray:
    """P^(1)_{mN x N} = 1_{m x 1} (x) I_N."""
    return np.kron(ones(m, 1), I(1 << m))


def Pi(m: int, i: int) -> np.ndarray:
    """P^(i)_{(m+1)N x mN} = I_{(i-2)N} (+) (1_{2x1} (x) I_N) (+) I_{(m-i+1)N}."""
    N = 1 << m
    return dsum(I((i - 2) * N), np.kron(ones(2, 1), I(N)), I((m - i + 1) * N))


def A1(m: int) -> np.ndarray:
    """A^(1)_{mN} = (I_{2^{m-1}} (x) H_2) (+) I_{(m-1)N}."""
    N = 1 << m
    return dsum(np.kron(I(1 << (m - 1)), H2), I((m - 1) * N))


def U(m: int, i: int) -> np.ndarray:
    """Eq. 2: U_N^(i) = I_{2^{m-i}} (x) [1_{1x2} (x) I_{2^{i-1}} ; 0]."""
    h = 1 << (i - 1)
    blk = np.vstack([np.kron(ones(1, 2), I(h)), Z(h, 2 * h)])
    return np.kron(I(1 << (m - i)), blk)


def V(m: int, i: int) -> np.ndarray:
    """Eq. 3: V_N^(i) = I_{2^{m-i}} (x) [0 ; I_{2^{i-1}} | -I_{2^{i-1}}]."""
    h = 1 << (i - 1)
    blk = np.vstack([Z(h, 2 * h), np.hstack([I(h), -I(h)])])
    return np.kron(I(1 << (m - i)), blk)


def Ai(m: int, i: int) -> np.ndarray:
    """A^(i)_{mN x (m+1)N} = I_{(i-1)N} (+) [U | V] (+) I_{(m-i)N}."""
    N = 1 << m
    return dsum(I((i - 1) * N), np.hstack([U(m, i), V(m, i)]), I((m - i) * N))


def Dtilde(i: int) -> np.ndarray:
    """D~_{2^i}^(i) = I_{2^{i-1}} (+) diag(w_{2^i}^0 .. w_{2^i}^{2^{i-1}-1})."""
    h = 1 << (i - 1)
    return dsum(I(h), np.diag(w(1 << i, np.arange(h))))


def D(m: int, i: int) -> np.ndarray:
    """D^(i)_{mN} = I_{(i-1)N} (+) (I_{2^{m-i}} (x) D~^(i)) (+) I_{(m-i)N}."""
    N = 1 << m
    return dsum(I((i - 1) * N), np.kron(I(1 << (m - i)), Dtilde(i)), I((m - i) * N))


def S(i: int, j: int) -> np.ndarray:
    """S^(j)_{2^{i-1}} = I_{2^{j-1}} (x) (H_2 (x) I_{2^{i-j-1}})."""
    return np.kron(I(1 << (j - 1)), np.kron(H2, I(1 << (i - j - 1))))


def W(i: int, j: int) -> np.ndarray:
    """W^(j)_{2^{i-1}} = I_{2^{j-1}} (x) [I_{2^{i-j-1}} (+) diag(w_{2^{i-j}}^n)]."""
    half = 1 << (i - j - 1)
    blk = dsum(I(half), np.diag(w(1 << (i - j), np.arange(half))))
    return np.kron(I(1 << (j - 1)), blk)


def R(i: int) -> np.ndarray:
    """R^(i)_{2^{i-1}} = (W^(i-1) S^(i-1)) (W^(i-2) S^(i-2)) ... (W^(1) S^(1))."""
    out = I(1 << (i - 1))
    for j in range(1, i):
        out = W(i, j) @ S(i, j) @ out
    return out


def F(m: int, i: int) -> np.ndarray:
    """F^(1) = I_{mN}; F^(i) = I_{(i-1)N} (+) (I_{2^{m-i}} (x) R~^(i)) (+) I_{(m-i)N}."""
    N = 1 << m
    if i == 1:
        return I(m * N)
    Rt = dsum(I(1 << (i - 1)), R(i))
    return dsum(I((i - 1) * N), np.kron(I(1 << (m - i)), Rt), I((m - i) * N))


def bitrev(v: int, bits: int) -> int:
    r = 0
    for b in range(bits):
        r |= ((v >> b) & 1) << (bits - 1 - b)
    return r


def T(i: int) -> np.ndarray:
    """T_{2^i}^(i): t_{k, <k>} = 1, <.> = bit reversal over i bits (Sec. 3)."""
    L = 1 << i
    out = np.zeros((L, L), dtype=np.complex128)
    for k in range(L):
        out[k, bitrev(k, i)] = 1
    return out


def Gamma(m: int) -> np.ndarray:
    """Gamma_{mN} = (+)_{i=1..m} (I_{2^{m-i}} (x) T_{2^i}^(i))."""
    return dsum(*[np.kron(I(1 << (m - i)), T(i)) for i in range(1, m + 1)])


def eq4(m: int) -> np.ndarray:
    """Eq. 4: Gamma (F^(m) D^(m) A^(m) P^(m)) ... (F^(1) D^(1) A^(1) P^(1))."""
    acc = F(m, 1) @ D(m, 1) @ A1(m) @ P1(m)
    for i in range(2, m + 1):
        acc = F(m, i) @ D(m, i) @ Ai(m, i) @ Pi(m, i) @ acc
    return Gamma(m) @ acc
