"""The identities the packed residual passes rest on, checked in FP64 (CPU).

The IOTF iteration's intensity |v|^2 and residual G are real fields. The GPU
path carries two of their rows in one complex row and filters only the column
bins kx = 0..nx/2 (its packed row and column passes); these tests pin, with
numpy's FFT as the DFT, the exact statements those passes use:

* the row DFT of z = I(2y') + i I(2y'+1) gives both rows' spectra:
  X(2y', k) = (Z(k) + conj Z(-k)) / 2, X(2y'+1, k) = (Z(k) - conj Z(-k)) / (2i);
* the bins 0 and nx/2 of a real row's spectrum are real, so those two columns
  can travel as one complex column X0 + i Xh and be split after the column
  DFT by the same rule along ky;
* the 2-D residual spectrum r = W F{I} - F{y} of real fields under a real,
  even window W is Hermitian, so the columns kx and nx - kx carry the same
  sum of |r|^2 (Parseval with weight 2 for 0 < kx < nx/2), and the inverse
  column transforms of the mirrored columns are conjugates;
* the position map of a packed row (bin kx at kx for kx <= nx/2, at
  nx/2 + (nx - kx) above) is a permutation that puts the mirror of every
  aligned pair of bins kx, kx + 1 (kx even, 0 < kx < nx/2) in the aligned pair
  nx/2 + kx, nx/2 + kx + 1.
"""
import numpy as np
import pytest

TOL = 1e-12


def pk_pos(kx, n):
    return kx if kx <= n // 2 else 3 * n // 2 - kx


@pytest.fixture(scope="module")
def fields():
    rng = np.random.default_rng(20146)
    ny, nx = 48, 64
    I = rng.random((ny, nx)) + 0.5
    y = I * (1 + 0.05 * rng.standard_normal((ny, nx)))
    u = np.fft.fftfreq(ny)[:, None]
    v = np.fft.fftfreq(nx)[None, :]
    W = np.exp(-2 * np.pi ** 2 * 4.0 * (u ** 2 + v ** 2))  # real, even window (an IOTF)
    return I, y, W


def test_two_real_rows_share_one_complex_transform(fields):
    I, _, _ = fields
    X = np.fft.fft(I, axis=1)
    Z = np.fft.fft(I[0::2] + 1j * I[1::2], axis=1)
    Zm = np.conj(np.roll(Z[:, ::-1], 1, axis=1))  # conj Z(-k)
    assert np.max(np.abs((Z + Zm) / 2 - X[0::2])) <= TOL * np.max(np.abs(X))
    assert np.max(np.abs((Z - Zm) / 2j - X[1::2])) <= TOL * np.max(np.abs(X))
    # and back: the inverse row DFT of X(2y') + i X(2y'+1) is I(2y') + i I(2y'+1)
    back = np.fft.ifft(X[0::2] + 1j * X[1::2], axis=1)
    assert np.max(np.abs(back.real - I[0::2])) <= TOL and np.max(np.abs(back.imag - I[1::2])) <= TOL


def test_edge_columns_are_real_and_split_after_one_column_transform(fields):
    I, _, _ = fields
    ny, nx = I.shape
    X = np.fft.fft(I, axis=1)
    assert np.max(np.abs(X[:, 0].imag)) <= TOL * np.max(np.abs(X))
    assert np.max(np.abs(X[:, nx // 2].imag)) <= TOL * np.max(np.abs(X))
    Wc = np.fft.fft(X[:, 0].real + 1j * X[:, nx // 2].real)  # one complex column
    Wm = np.conj(np.roll(Wc[::-1], 1))
    X0, Xh = np.fft.fft(X[:, 0]), np.fft.fft(X[:, nx // 2])
    assert np.max(np.abs((Wc + Wm) / 2 - X0)) <= TOL * np.max(np.abs(X0))
    assert np.max(np.abs((Wc - Wm) / 2j - Xh)) <= TOL * np.max(np.abs(X0))


def test_residual_spectrum_is_hermitian_and_half_the_columns_carry_the_loss(fields):
    I, y, W = fields
    ny, nx = I.shape
    r = W * np.fft.fft2(I) - np.fft.fft2(y)
    rm = np.conj(np.roll(np.roll(r[::-1, ::-1], 1, axis=0), 1, axis=1))  # conj r(-ky, -kx)
    assert np.max(np.abs(r - rm)) <= TOL * np.max(np.abs(r))
    full = np.sum(np.abs(r) ** 2)
    col = np.sum(np.abs(r) ** 2, axis=0)
    half = col[0] + col[nx // 2] + 2 * np.sum(col[1:nx // 2])
    assert abs(half - full) <= TOL * full
    # Parseval: the loss of Eq. (2) of the filtered intensity
    L = np.sum((np.fft.ifft2(W * np.fft.fft2(I)).real - y) ** 2)
    assert abs(half / (ny * nx) - L) <= 1e-10 * L
    # the inverse column transforms of the mirrored columns are conjugates
    g = np.fft.ifft(r, axis=0)
    for kx in (1, 5, nx // 2 - 1):
        assert np.max(np.abs(g[:, nx - kx] - np.conj(g[:, kx]))) <= TOL * np.max(np.abs(g))


@pytest.mark.parametrize("n", [16, 64, 96, 768, 1024, 1536, 2048])
def test_packed_positions_pair_aligned_bins_with_aligned_mirrors(n):
    pos = [pk_pos(k, n) for k in range(n)]
    assert sorted(pos) == list(range(n))  # a permutation of the row
    h = n // 2
    for kx in range(2, h, 2):  # aligned pairs of the front half, bin 0's pair aside
        a, b = pk_pos(n - kx, n), pk_pos(n - kx - 1, n)
        assert (a, b) == (h + kx, h + kx + 1) and a % 2 == 0
    # bin 0's pair: bin 1's mirror sits next to bin nx/2, both self-mirrored bins in one aligned pair
    assert pk_pos(0, n) == 0 and pk_pos(h, n) == h and pk_pos(n - 1, n) == h + 1
