"""CPU check of the index algebra that the spectral correction's warp FFT
rests on (n = 32 R points per line; lane j, register m).  Written from the
definitions, against numpy's FFT and the DCT-II sum, for every supported n:

* the four-step split n = R x 32: an R-point DFT over the registers, the
  twiddle e^{-2 pi i j a / n}, a 32-point DFT across the lanes by xor
  butterflies (decimation in frequency), leaves Z_{a + R brev5(j)} in lane j,
  register a; the transposed order (decimation in time across the lanes)
  takes that layout back to j + 32 m;
* the value at index n - k of that layout sits in lane j ^ 31, register
  R - a (a > 0), or in lane brev5((32 - brev5(j)) mod 32), register 0;
* Makhoul's reordering and rotation give the unnormalised DCT-II of two real
  lines from one complex FFT, and its inverse.
"""
import numpy as np
import pytest

LANES = np.arange(32)


def brev5(j):
    return int(format(j, "05b")[::-1], 2)


BREV = np.array([brev5(j) for j in range(32)])


def dft(v):
    """Plain DFT along axis 0 (the R registers): e^{-2 pi i q a / R}."""
    R = v.shape[0]
    W = np.exp(-2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    return W @ v


def fft_dif(v, n):
    """v[m, j] = z_{j + 32 m} -> v[a, j] = Z_{a + R brev5(j)}."""
    R = n // 32
    v = dft(v)
    v = v * np.exp(-2j * np.pi * np.outer(np.arange(R), LANES) / n)
    for st in range(4, -1, -1):
        h = 1 << st
        up = (LANES & h) != 0
        w = np.exp(-1j * np.pi * (LANES & (h - 1)) / h)
        p = v[:, LANES ^ h]
        v = np.where(up, (p - v) * w, v + p)
    return v


def fft_dit(v, n):
    """v[a, j] = u_{a + R brev5(j)} -> v[m, j] = U_{j + 32 m}."""
    R = n // 32
    for st in range(5):
        h = 1 << st
        up = (LANES & h) != 0
        w = np.exp(-1j * np.pi * (LANES & (h - 1)) / h)
        m = np.where(up, v * w, v)
        p = m[:, LANES ^ h]
        v = np.where(up, p - m, m + p)
    v = v * np.exp(-2j * np.pi * np.outer(np.arange(R), LANES) / n)
    return dft(v)


def layout_index(n):
    R = n // 32
    return np.arange(R)[:, None] + R * BREV[None, :]          # k held by [a, j]


def strided_index(n):
    return LANES[None, :] + 32 * np.arange(n // 32)[:, None]  # index held by [m, j]


def mirror(v, n):
    """c[a, j] = the value at index (n - k) mod n of the layout a + R brev5(j)."""
    R = n // 32
    c = np.empty_like(v)
    c[0] = v[0][[brev5((32 - BREV[j]) & 31) for j in range(32)]]
    for a in range(1, R):
        c[a] = v[R - a][LANES ^ 31]
    return c


def src(p, n):
    return np.where(p < n // 2, 2 * p, 2 * (n - 1 - p) + 1)


NS = [32, 64, 128, 256, 512]


@pytest.mark.parametrize("n", NS)
def test_four_step_split_and_its_transpose(n):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Z = np.fft.fft(z)
    got = fft_dif(z[strided_index(n)], n)
    assert np.abs(got - Z[layout_index(n)]).max() < 1e-9 * np.abs(Z).max()
    back = fft_dit(Z[layout_index(n)], n)                       # FFT of the spectrum
    assert np.abs(back - np.fft.fft(Z)[strided_index(n)]).max() < 1e-9 * n * np.abs(Z).max()


@pytest.mark.parametrize("n", NS)
def test_mirror_partner(n):
    k = layout_index(n)
    assert np.array_equal(mirror(k, n), (n - k) % n)


@pytest.mark.parametrize("n", NS)
def test_two_line_dct_and_inverse(n):
    rng = np.random.default_rng(100 + n)
    xa, xb = rng.standard_normal(n), rng.standard_normal(n)
    C = np.cos(np.pi * np.outer(np.arange(n), np.arange(n) + 0.5) / n)   # DCT-II, unnormalised
    k = layout_index(n)
    wm = np.exp(-1j * np.pi * k / (2 * n))
    # forward: v = Makhoul's reordering, Z = FFT(v_a + i v_b), split by Z_{n-k}
    p = strided_index(n)
    Z = fft_dif(xa[src(p, n)] + 1j * xb[src(p, n)], n)
    c = mirror(Z, n)
    va = 0.5 * (Z + np.conj(c))
    vb = -0.5j * (Z - np.conj(c))
    Xa, Xb = np.real(wm * va), np.real(wm * vb)
    assert np.abs(Xa - (C @ xa)[k]).max() < 1e-9 * n
    assert np.abs(Xb - (C @ xb)[k]).max() < 1e-9 * n
    # inverse: conj V_k = wm_k (X_k + i X_{n-k}) (X_n = 0), FFT of conj(V_a + i V_b)
    nk_a, nk_b = mirror(Xa, n), mirror(Xb, n)
    nk_a[0, 0] = nk_b[0, 0] = 0.0
    u = wm * (Xa + 1j * nk_a) - 1j * wm * (Xb + 1j * nk_b)
    r = fft_dit(u, n)
    ya, yb = np.empty(n), np.empty(n)
    ya[src(p, n)] = r.real / n
    yb[src(p, n)] = -r.imag / n
    assert np.abs(ya - xa).max() < 1e-10 * n
    assert np.abs(yb - xb).max() < 1e-10 * n
