"""The index algebra of the split column transform (CPU, numpy): the
factorisation the GPU's fused column kernels follow, written out with their
thread roles, against numpy's FFT.

Forward (k_colstack after k_colfft's first column factor): with n = N1 * 16,
row v = 16 a + b and output row y = f1 + N1 f2,
    Y[16 f1 + b] = sum_a x[16 a + b] w_N1^(a f1)                 (k_colfft)
    X[f1 + N1 f2] = sum_b w_16^(b f2) w_n^(b f1) Y[16 f1 + b]     (k_colstack)
with the 16-point factor as two 4-point passes (b = 4 b1 + b0,
f2 = g0 + 4 g1): over b1 for each b0, times w_16^(b0 g0), then over b0.
Adjoint (k_spreadcol before k_colfft's forward first column factor): the same
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
    for b in range(N2):  # first factor (k_colfft), in place: rows 16 f1 + b
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
    for b in range(N2):  # k_colfft's forward first factor along the columns
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


# -------------------------------------------------------------------------
# The first column factor as k_colfft computes it in shared memory: the
# N1-point DFT of the rows 16 a + b of one column, N1 = 16 Q, through its
# passes and in-block positions, written out with the kernel's thread roles.

def _dft(v, sign):
    k = np.arange(v.size)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / v.size) @ v


def colfft_block(x, sign):
    """x: the N1 samples x[16 a + b] of one (b, column), a = 0 .. N1-1.
    Returns Y indexed by f1 (what the kernel stores at row 16 f1 + b)."""
    n1 = x.size
    tw = np.exp(sign * 2j * np.pi * np.arange(n1) / n1)  # w_N1^e with the kernel's sign
    buf = x.astype(complex).copy()                       # shared memory, position a
    out = np.empty(n1, complex)
    if n1 < 16:                                          # one pass
        return _dft(buf, sign)
    q = n1 // 16
    for a2 in range(q):                                  # pass A: thread (x, a2)
        v = _dft(buf[[q * a1 + a2 for a1 in range(16)]], sign)
        for k1 in range(16):
            buf[q * k1 + a2] = v[k1] * tw[a2 * k1]
    if q <= 16:                                          # pass B: thread (x, k1)
        for k1 in range(16):
            v = _dft(buf[[q * k1 + a2 for a2 in range(q)]], sign) if q > 1 else buf[[k1]]
            for kq in range(q):
                out[k1 + 16 * kq] = v[kq]
        return out
    r = q // 16
    for k1 in range(16):                                 # pass B1: the warp owning block k1
        stage = {}
        for c2 in range(r):
            v = _dft(buf[[q * k1 + r * c1 + c2 for c1 in range(16)]], sign)
            for j1 in range(16):
                stage[q * k1 + 16 * c2 + (j1 ^ c2)] = v[j1] * tw[16 * c2 * j1]
        for pos, val in stage.items():                   # written after the warp's reads
            buf[pos] = val
    for k1 in range(16):                                 # pass B2: thread (x, k1, j1)
        for j1 in range(16):
            v = _dft(buf[[q * k1 + 16 * c2 + (j1 ^ c2) for c2 in range(r)]], sign)
            for j2 in range(r):
                out[k1 + 16 * (j1 + 16 * j2)] = v[j2]
    return out


@pytest.mark.parametrize("n1", [4, 8, 16, 32, 64, 128, 256, 512, 1024])
@pytest.mark.parametrize("sign", [1, -1])
def test_colfft_passes_are_the_n1_point_dft(n1, sign):
    rng = np.random.default_rng(n1 + (sign > 0))
    x = rng.standard_normal(n1) + 1j * rng.standard_normal(n1)
    ref = np.fft.ifft(x) * n1 if sign > 0 else np.fft.fft(x)
    assert np.max(np.abs(colfft_block(x, sign) - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_colfft_block_positions_are_a_permutation():
    """Every pass reads and writes each in-block position exactly once."""
    for n1 in (256, 512, 1024):
        q = n1 // 16
        pa = sorted(q * a1 + a2 for a2 in range(q) for a1 in range(16))
        assert pa == list(range(n1))
        if q > 16:
            r = q // 16
            reads = sorted(q * k1 + r * c1 + c2 for k1 in range(16) for c2 in range(r) for c1 in range(16))
            writes = sorted(q * k1 + 16 * c2 + (j1 ^ c2) for k1 in range(16) for c2 in range(r) for j1 in range(16))
            assert reads == writes == list(range(n1))


# -------------------------------------------------------------------------
# The planes' b-major row order of the split transform: grid row 16 a + b is
# memory row b N1 + a (GridCfg::row_perm / plane_row), so k_colfft reads and
# writes one contiguous run of N1 memory rows per b, and k_colstack reads the
# 16 memory rows b N1 + f1 (b = 0 .. 15) of each f1.

def plane_row(v, n1):
    return (v % N2) * n1 + v // N2


@pytest.mark.parametrize("n1", [4, 16, 64, 256, 1024])
def test_b_major_rows_are_a_permutation(n1):
    rows = [plane_row(v, n1) for v in range(n1 * N2)]
    assert sorted(rows) == list(range(n1 * N2))
    # the column factor's input rows of one b are the run b N1 .. b N1 + N1 - 1
    for b in (0, 5, N2 - 1):
        assert [plane_row(N2 * a + b, n1) for a in range(n1)] == list(range(b * n1, b * n1 + n1))


@pytest.mark.parametrize("n1", [4, 8, 64])
def test_column_transform_through_b_major_memory(n1):
    """A plane of 3 columns stored b-major; the first factor on each memory
    run (in place), then the last factor reading memory rows b N1 + f1: the
    inverse DFT of every column in natural order."""
    n = n1 * N2
    rng = np.random.default_rng(300 + n1)
    grid = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    mem = np.empty_like(grid)
    for v in range(n):
        mem[plane_row(v, n1)] = grid[v]
    for b in range(N2):  # k_colfft: block (b, columns) on its run, in place
        for col in range(3):
            mem[b * n1:(b + 1) * n1, col] = colfft_block(mem[b * n1:(b + 1) * n1, col], +1)
    out = np.empty_like(grid)
    for col in range(3):  # k_colstack's last factor on memory rows b N1 + f1
        y = np.empty(n, complex)
        for f1 in range(n1):
            for b in range(N2):
                y[N2 * f1 + b] = mem[b * n1 + f1, col]  # Y[16 f1 + b]
        for f1 in range(n1):
            for f2 in range(N2):
                out[f1 + n1 * f2, col] = sum(_w(N2, b * f2) * _w(n, b * f1) * y[N2 * f1 + b] for b in range(N2))
    ref = np.fft.ifft(grid, axis=0) * n
    assert np.max(np.abs(out - ref)) <= 1e-11 * np.max(np.abs(ref))
