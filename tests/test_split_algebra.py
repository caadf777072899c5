"""The index algebra of the split column transform (CPU, numpy): the
factorisation the GPU's fused column kernels follow, written out with their
thread roles, against numpy's FFT.

Forward (k_colstack after cuFFT's first column factor): with n = N1 * 16,
row v = 16 a + b and output row y = f1 + N1 f2,
    Y[16 f1 + b] = sum_a x[16 a + b] w_N1^(a f1)                 (cuFFT)
    X[f1 + N1 f2] = sum_b w_16^(b f2) w_n^(b f1) Y[16 f1 + b]     (kernel)
with the 16-point factor as two 4-point passes (b = 4 b1 + b0,
f2 = g0 + 4 g1): over b1 for each b0, times w_16^(b0 g0), then over b0.
Adjoint (k_spreadcol before cuFFT's forward first column factor): the same
steps in reverse order with conjugate twiddles and the minus sign.  The
unnormalised inverse column DFT (exponent +) and its adjoint, the forward
DFT (exponent -), are the references."""
import numpy as np
import pytest

Q, N2 = 4, 16


def _w(m, e):
    return np.exp(2j * np.pi * e / m)


def _dft4(v, sign):
    k = np.arange(Q)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / Q) @ v


def forward_split(x, n1):
    """Inverse (exponent +) transform of one column through the split."""
    n = n1 * N2
    y = np.empty(n, complex)
    for b in range(N2):  # first factor, in place: rows 16 f1 + b
        y[b::N2] = np.exp(2j * np.pi * np.outer(np.arange(n1), np.arange(n1)) / n1) @ x[b::N2]
    out = np.empty(n, complex)
    for f1 in range(n1):
        ex = np.empty((Q, Q), complex)  # [g0][b0]
        for j in range(Q):  # pass 1: thread b0 = j
            tw = np.array([_w(n, ((Q * q + j) * f1) % n) for q in range(Q)])
            u = _dft4(y[[N2 * f1 + Q * q + j for q in range(Q)]] * tw, +1)
            ex[:, j] = u * np.array([_w(N2, (j * g) % N2) for g in range(Q)])
        for j in range(Q):  # pass 2: thread g0 = j
            z = _dft4(ex[j, :], +1)
            for g in range(Q):
                out[f1 + n1 * (j + Q * g)] = z[g]
    return out


def adjoint_split(r, n1):
    """Forward (exponent -) transform of one column through the adjoint split."""
    n = n1 * N2
    y = np.empty(n, complex)
    for f1 in range(n1):
        ex = np.empty((Q, Q), complex)  # [b0][g0]
        for j in range(Q):  # thread g0 = j: over g1 -> b0, times conj(w_16^(b0 g0))
            s = _dft4(np.array([r[f1 + n1 * (j + Q * g)] for g in range(Q)]), -1)
            ex[:, j] = s * np.conj(np.array([_w(N2, (j * q) % N2) for q in range(Q)]))
        for j in range(Q):  # thread b0 = j: over g0 -> b1, times conj(w_n^(b f1))
            t = _dft4(ex[j, :], -1)
            for q in range(Q):
                y[N2 * f1 + Q * q + j] = t[q] * np.conj(_w(n, ((Q * q + j) * f1) % n))
    x = np.empty(n, complex)
    for b in range(N2):  # cuFFT forward first factor along the columns
        x[b::N2] = np.exp(-2j * np.pi * np.outer(np.arange(n1), np.arange(n1)) / n1) @ y[b::N2]
    return x


@pytest.mark.parametrize("n1", [4, 8, 16, 64])
def test_forward_split_is_the_inverse_dft(n1):
    rng = np.random.default_rng(n1)
    x = rng.standard_normal(n1 * N2) + 1j * rng.standard_normal(n1 * N2)
    ref = np.fft.ifft(x) * x.size
    assert np.max(np.abs(forward_split(x, n1) - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n1", [4, 8, 16, 64])
def test_adjoint_split_is_the_forward_dft(n1):
    rng = np.random.default_rng(100 + n1)
    r = rng.standard_normal(n1 * N2) + 1j * rng.standard_normal(n1 * N2)
    ref = np.fft.fft(r)
    assert np.max(np.abs(adjoint_split(r, n1) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_the_two_splits_are_adjoint():
    """<F x, r> = <x, F^H r> for the two factorisations as written."""
    rng = np.random.default_rng(7)
    n1 = 8
    x = rng.standard_normal(n1 * N2) + 1j * rng.standard_normal(n1 * N2)
    r = rng.standard_normal(n1 * N2) + 1j * rng.standard_normal(n1 * N2)
    lhs = np.vdot(r, forward_split(x, n1))
    rhs = np.vdot(adjoint_split(r, n1), x)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
