"""Fourier and Chebyshev bases in plain FP64 (oracle; test infrastructure only).

Conventions, each restated from the paper:

Fourier (Sec. "Fourier basis"): modes exp(i k x) on [0, L); grid
x_i = L i / N_g; a real field keeps only k >= 0 and drops the Nyquist mode;
coefficients are mode amplitudes f_k = (1/N_g) sum_i f(x_i) exp(-i k x_i).
With N_c modes the stored wavenumbers are n = 0 .. N_c/2 - 1, k = 2 pi n / L.

Chebyshev (Sec. "Chebyshev basis"): T_n(x) = cos(n arccos x) on the native
interval [-1, 1]; Gauss grid x_i = -cos(pi (i + 1/2) / N_g) (ascending);
f_n = (2 - delta_n0) / N_g * sum_i f(x_i) T_n(x_i).  The problem interval
[a, b] maps affinely, z = a + (b - a)(x + 1)/2, so d/dz = 2/(b - a) d/dx.

Scaled transforms (Sec. "Scaled transforms & dealiasing"): a backward
transform to N_g = s N_c points pads the coefficients with zeros; a forward
transform from N_g points keeps the first N_c coefficients.

Operator matrices (Appendix "Differentiation and conversion matrices",
"Dirichlet recombination matrices"), all on the native interval:
  D^TT_ij = 2 j ((j - i) mod 2) / (1 + delta_i0) [i < j]   (T-to-T derivative)
  D^TU_ij = j delta_{i, j-1}                               (T-to-U derivative)
  P^L_ij  = (delta_ij - delta_{i, j-2}) / (2 - delta_j0)   (T-to-U conversion)
  P^R_ij  = delta_ij - delta_{i, j-2} [j > 1]              (Dirichlet basis)
  T_n(-1) = (-1)^n,  T_n(1) = 1                            (interpolation)

Pins: ``tests/test_oracle_bases.py``.
"""
import numpy as np


# ----------------------------------------------------------------------------
# Fourier
# ----------------------------------------------------------------------------

def fourier_grid(n_grid, length):
    """x_i = L i / N_g, i = 0 .. N_g - 1 (Sec. "Fourier basis")."""
    return length * np.arange(n_grid) / n_grid


def fourier_wavenumbers(n_coeff, length):
    """Physical wavenumbers of the stored k >= 0 modes, Nyquist dropped."""
    return 2.0 * np.pi * np.arange(n_coeff // 2) / length


def fourier_forward(g, n_coeff, axis=-1):
    """Grid values (real, N_g points along ``axis``) -> N_c/2 complex amplitudes.

    f_k = (1/N_g) sum_i g(x_i) exp(-i k x_i), kept for k < N_c/2 (the Nyquist
    bin and everything above it are discarded).
    """
    g = np.asarray(g, dtype=np.float64)
    n_grid = g.shape[axis]
    f = np.fft.rfft(g, axis=axis) / n_grid
    f = np.take(f, np.arange(n_coeff // 2), axis=axis)
    return f


def fourier_backward(f, n_grid, axis=-1):
    """N_c/2 complex amplitudes (k >= 0) -> real grid values on N_g points.

    g(x_i) = sum_{|k| <= k_m} f_k exp(i k x_i) with f_{-k} = conj(f_k); bins
    above the stored ones (and the Nyquist bin) are zero.
    """
    f = np.asarray(f, dtype=np.complex128)
    f = np.moveaxis(f, axis, -1)
    full = np.zeros(f.shape[:-1] + (n_grid // 2 + 1,), dtype=np.complex128)
    full[..., : f.shape[-1]] = f
    g = np.fft.irfft(full, n=n_grid, axis=-1) * n_grid
    return np.moveaxis(g, -1, axis)


def fourier_c_modes(n_coeff):
    """Signed mode numbers of the N_c stored slots of a complex Fourier axis,
    in FFT order: slot s holds n = s for s < N_c/2 and n = s - N_c above;
    the Nyquist slot s = N_c/2 is kept at zero (Sec. "Fourier basis")."""
    s = np.arange(n_coeff)
    return np.where(s < n_coeff // 2, s, s - n_coeff)


def fourier_c_wavenumbers(n_coeff, length):
    """Physical wavenumbers 2 pi n / L of the stored slots of a complex axis."""
    return 2.0 * np.pi * fourier_c_modes(n_coeff) / length


def fourier_c_forward(g, n_coeff, axis=-1):
    """Complex grid values on N_g points -> N_c complex amplitudes in FFT order,
    f_n = (1/N_g) sum_i g(y_i) exp(-i n y_i) for |n| < N_c/2; Nyquist slot zero."""
    g = np.moveaxis(np.asarray(g, dtype=np.complex128), axis, -1)
    n_grid = g.shape[-1]
    full = np.fft.fft(g, axis=-1) / n_grid
    n = fourier_c_modes(n_coeff)
    f = full[..., n % n_grid]
    f[..., n_coeff // 2] = 0.0
    return np.moveaxis(f, -1, axis)


def fourier_c_backward(f, n_grid, axis=-1):
    """N_c amplitudes in FFT order -> complex grid values on N_g >= N_c points,
    g(y_i) = sum_{|n| < N_c/2} f_n exp(i n y_i) (Nyquist slot ignored)."""
    f = np.moveaxis(np.asarray(f, dtype=np.complex128), axis, -1)
    n_coeff = f.shape[-1]
    n = fourier_c_modes(n_coeff)
    keep = np.arange(n_coeff) != n_coeff // 2
    full = np.zeros(f.shape[:-1] + (n_grid,), dtype=np.complex128)
    full[..., n[keep] % n_grid] = f[..., keep]
    g = np.fft.ifft(full, axis=-1) * n_grid
    return np.moveaxis(g, -1, axis)


# ----------------------------------------------------------------------------
# Chebyshev
# ----------------------------------------------------------------------------

def chebyshev_native_grid(n_grid):
    """x_i = -cos(pi (i + 1/2) / N_g), ascending in [-1, 1]."""
    i = np.arange(n_grid)
    return -np.cos(np.pi * (i + 0.5) / n_grid)


def chebyshev_grid(n_grid, a=0.0, b=1.0):
    """Gauss grid mapped to the problem interval [a, b]."""
    return a + (b - a) * (chebyshev_native_grid(n_grid) + 1.0) / 2.0


def chebyshev_T_matrix(n_coeff, n_grid):
    """Dense matrix T[i, n] = T_n(x_i) = cos(n arccos x_i) at the Gauss nodes."""
    x = chebyshev_native_grid(n_grid)
    n = np.arange(n_coeff)
    return np.cos(np.outer(np.arccos(x), n))


def chebyshev_forward(g, n_coeff, axis=-1):
    """Grid values on N_g Gauss nodes -> first N_c Chebyshev coefficients.

    c_n = (2 - delta_n0) / N_g * sum_i g_i T_n(x_i)   (dense quadrature).
    Works for real or complex data (real and imaginary parts independently).
    """
    g = np.moveaxis(np.asarray(g), axis, -1)
    n_grid = g.shape[-1]
    T = chebyshev_T_matrix(n_coeff, n_grid)
    w = np.full(n_coeff, 2.0 / n_grid)
    w[0] = 1.0 / n_grid
    c = (g @ T) * w
    return np.moveaxis(c, -1, axis)


def chebyshev_backward(c, n_grid, axis=-1):
    """Chebyshev coefficients -> values on N_g Gauss nodes (zero padding above)."""
    c = np.moveaxis(np.asarray(c), axis, -1)
    T = chebyshev_T_matrix(c.shape[-1], n_grid)
    g = c @ T.T
    return np.moveaxis(g, -1, axis)


def chebyshev_forward_dct(g, n_coeff, axis=-1):
    """Same definition as chebyshev_forward, computed with scipy's DCT-II.

    With T_n(x_i) = (-1)^n cos(pi n (2i+1) / (2 N_g)) and scipy's
    DCT-II y_n = 2 sum_i g_i cos(pi n (2i+1) / (2 N_g)):
    c_n = (-1)^n (2 - delta_n0) / (2 N_g) y_n.  A second summation order,
    used only to measure the rounding floor between two FP64 evaluations.
    """
    import scipy.fft as sf
    g = np.moveaxis(np.asarray(g), axis, -1)
    n_grid = g.shape[-1]
    y = sf.dct(g, type=2, axis=-1)
    w = np.full(n_grid, 1.0 / n_grid)
    w[0] = 0.5 / n_grid
    c = (y * w * (-1.0) ** np.arange(n_grid))[..., :n_coeff]
    return np.moveaxis(c, -1, axis)


def chebyshev_backward_dct(c, n_grid, axis=-1):
    """Same definition as chebyshev_backward, computed with scipy's DCT-III
    (y_k = d_0 + 2 sum_{n>=1} d_n cos(pi n (2k+1) / (2 N_g)), d_n = (-1)^n c_n)."""
    import scipy.fft as sf
    c = np.moveaxis(np.asarray(c), axis, -1)
    n_c = c.shape[-1]
    d = np.zeros(c.shape[:-1] + (n_grid,), dtype=np.result_type(c, np.float64))
    d[..., :n_c] = c * (-1.0) ** np.arange(n_c)
    d[..., 0] *= 2.0
    g = sf.dct(d, type=3, axis=-1) / 2.0
    return np.moveaxis(g, -1, axis)


def cheb_D_TT(n):
    """T-to-T derivative matrix on [-1, 1] (dense upper triangular)."""
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if (j - i) % 2 == 1:
                D[i, j] = 2.0 * j / (1.0 + (i == 0))
    return D


def cheb_D_TU(n):
    """T-to-U derivative on [-1, 1]: dT_j/dx = j U_{j-1}."""
    D = np.zeros((n, n))
    for j in range(1, n):
        D[j - 1, j] = float(j)
    return D


def cheb_P_L(n):
    """T-to-U conversion: P^L_ij = (delta_ij - delta_{i,j-2}) / (2 - delta_j0)."""
    P = np.zeros((n, n))
    for j in range(n):
        P[j, j] = 1.0 / (2.0 - (j == 0))
        if j >= 2:
            P[j - 2, j] = -1.0 / (2.0 - (j == 0))
    return P


def cheb_P_R(n):
    """Dirichlet recombination: P^R_ij = delta_ij - delta_{i,j-2} [j > 1]."""
    P = np.eye(n)
    for j in range(2, n):
        P[j - 2, j] = -1.0
    return P


def cheb_left_vector(n):
    """Row vector of T_n(-1) = (-1)^n (interpolation to the left endpoint)."""
    return (-1.0) ** np.arange(n)


def cheb_right_vector(n):
    """Row vector of T_n(+1) = 1 (interpolation to the right endpoint)."""
    return np.ones(n)


def cheb_integrate_vector(n):
    """Row vector of int_{-1}^{1} T_n dx = 2/(1 - n^2) for even n, 0 for odd n."""
    v = np.zeros(n)
    for k in range(0, n, 2):
        v[k] = 2.0 / (1.0 - k * k)
    return v


def chebyshev_derivative(c, a=0.0, b=1.0, axis=-1):
    """Coefficients of d/dz of a Chebyshev series on [a, b], via the dense D^TT."""
    c = np.moveaxis(np.asarray(c), axis, -1)
    D = cheb_D_TT(c.shape[-1]) * (2.0 / (b - a))
    return np.moveaxis(c @ D.T, -1, axis)
