"""The method's steps, in the paper's order, in plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions.  The band-limit ``L`` is exclusive (coefficients for 0 <= l < L);
the paper's inclusive band-limit is Lp = L - 1 and its torus has N = 2 Lp + 1
samples per axis (Sec. 3.4.1, eqns nodes_theta and nodes_phi).  The sphere grid
keeps the L rings t = 0..Lp with theta_t <= pi (the ring theta_{Lp} = pi is a
sphere point) and all N longitudes.  Coefficients are stored at index
l*l + l + m.  Torus arrays are ``T[b, m + Lp, m' + Lp]`` with m the phi frequency
and m' the theta frequency.

The O(L^3) sums (Risbo recursion, eqn fourier_coeff, the harmonic projection,
the weight convolution, the paper's triangular solve) run in ``ssht_oracle.c``;
the discrete Fourier transforms use numpy.fft.
"""
import numpy as np

from . import _lib


def sizes(L):
    Lp = L - 1
    return Lp, 2 * Lp + 1


def thetas(L):
    """Colatitudes theta_t = pi (2t+1) / (2 Lp + 1) for t = 0..Lp (eqn nodes_theta, theta <= pi)."""
    Lp, N = sizes(L)
    return np.pi * (2.0 * np.arange(L) + 1.0) / N


def phis(L):
    """Longitudes phi_p = pi (2p+1) / (2 Lp + 1), p = 0..2Lp (eqn nodes_phi)."""
    Lp, N = sizes(L)
    return np.pi * (2.0 * np.arange(N) + 1.0) / N


def _as_batch(x, ndim):
    x = np.asarray(x)
    single = x.ndim == ndim - 1
    if single:
        x = x[None]
    return np.ascontiguousarray(x.astype(np.complex128)), single


# ---------------------------------------------------------------------------
# Wigner d (Risbo recursion, Sec. 2.2)
# ---------------------------------------------------------------------------

def wigner_full(tj, beta=np.pi / 2):
    """Full matrix d^{j}(beta), j = tj/2, rows/cols m, n = -j..j (Risbo recursion)."""
    out = np.zeros((tj + 1, tj + 1))
    _lib.check(_lib.lib().oracle_wigner_full(tj, beta, _lib.ptr(out)), "wigner_full")
    return out


def delta_offsets(L):
    """offset(l) = sum_{k<l} (k+1)^2: start of degree l in the quadrant table (Sec. 4.1)."""
    l = np.arange(L + 1)
    return l * (l + 1) * (2 * l + 1) // 6


def delta_quadrant(L, beta=np.pi / 2):
    """Quadrant table Delta^l_{m' m}, 0 <= m', m <= l, l < L; entry (l, m', m) at offset(l) + m'(l+1) + m."""
    out = np.zeros(int(delta_offsets(L)[L]))
    _lib.check(_lib.lib().oracle_delta_quadrant(L, beta, _lib.ptr(out)), "delta_quadrant")
    return out


def delta_slab(table, l):
    """(l+1) x (l+1) matrix [m', m] of one degree from a quadrant table."""
    off = int(delta_offsets(l + 1)[l])
    return table[off:off + (l + 1) ** 2].reshape(l + 1, l + 1)


# ---------------------------------------------------------------------------
# Inverse transform (Sec. 3.4.3)
# ---------------------------------------------------------------------------

def fourier_coeff(flm, L, s):
    """Eqn fourier_coeff: torus Fourier coefficients F_{m m'} for all m, m' in [-Lp, Lp]."""
    flm, single = _as_batch(flm, 2)
    B = flm.shape[0]
    assert flm.shape[1] == L * L
    Lp, N = sizes(L)
    F = np.zeros((B, N, N), dtype=np.complex128)
    _lib.check(_lib.lib().oracle_fourier_coeff(L, s, B, _lib.ptr(flm), _lib.ptr(F)), "fourier_coeff")
    return F[0] if single else F


def torus_synthesis(F, L):
    """Eqn idft_spatial: samples of sum_{m,m'} F_{m m'} e^{i(m phi + m' theta)} on the N x N torus,
    returned as [b, t, p] (theta index t, phi index p), via the 2-D inverse DFT with the phase
    e^{i pi (m + m') / N} and the inverse fft-shift."""
    F, single = _as_batch(F, 3)
    Lp, N = sizes(L)
    m = np.arange(-Lp, Lp + 1)
    ph = np.exp(1j * np.pi * (m[:, None] + m[None, :]) / N)
    X = np.transpose(F * ph[None], (0, 2, 1))          # [b, m', m]: theta frequency first
    X = np.fft.ifftshift(X, axes=(1, 2))
    ft = N * N * np.fft.ifft2(X, axes=(1, 2))
    return ft[0] if single else ft


def inverse(flm, L, s):
    """Inverse spin transform (Sec. 3.4.3): eqn fourier_coeff, then eqn idft_spatial; keep the
    rings with theta <= pi.  Returns f[b, t, p] on the L x N sphere grid."""
    F = fourier_coeff(flm, L, s)
    ft = torus_synthesis(F, L)
    return ft[..., :L, :]


# ---------------------------------------------------------------------------
# Forward transform pieces
# ---------------------------------------------------------------------------

def phi_analysis(f, L):
    """f_m(theta_t) = (1/N) sum_p f[t, p] e^{-i m phi_p} for m in [-Lp, Lp]; returns [b, t, m + Lp]."""
    f, single = _as_batch(f, 3)
    Lp, N = sizes(L)
    m = np.arange(-Lp, Lp + 1)
    fm = np.fft.fftshift(np.fft.fft(f, axis=2), axes=2) / N
    fm = fm * np.exp(-1j * np.pi * m / N)[None, None, :]
    return fm[0] if single else fm


def torus_extend(fm, L, s, parity="spin"):
    """Extension of each phi-frequency column to theta in [0, 2 pi) (Sec. 3.2):
    f~_m(2 pi - theta) = sigma_m f~_m(theta), i.e. f~_m[t] = sigma_m f_m[N-1-t] for t >= L.
    ``parity='spin'`` takes sigma_m = (-1)^{m+s} (even extension for even m+s, odd for odd);
    ``'even'`` / ``'odd'`` apply one extension to every column (the paper's f~^e, f~^o).
    For an odd column the sample on theta = pi (t = Lp) is set to zero, which an odd
    2 pi-periodic function must satisfy.  Input/output [b, t, m + Lp]."""
    fm, single = _as_batch(fm, 3)
    Lp, N = sizes(L)
    B = fm.shape[0]
    m = np.arange(-Lp, Lp + 1)
    if parity == "spin":
        sig = np.where((m + s) % 2 == 0, 1.0, -1.0)
    elif parity == "even":
        sig = np.ones(N)
    else:
        sig = -np.ones(N)
    ext = np.zeros((B, N, N), dtype=np.complex128)
    ext[:, :L, :] = fm[:, :L, :]
    ext[:, Lp, :] = np.where(sig > 0, fm[:, Lp, :], 0.0)
    t = np.arange(L, N)
    ext[:, L:, :] = sig[None, None, :] * fm[:, N - 1 - t, :]
    return ext[0] if single else ext


def theta_analysis(ext, L):
    """F_{m m'} = (1/N) sum_{t<N} f~_m[t] e^{-i m' theta_t} (eqn dft_spatial along theta);
    input [b, t, m + Lp], output F[b, m + Lp, m' + Lp]."""
    ext, single = _as_batch(ext, 3)
    Lp, N = sizes(L)
    mp = np.arange(-Lp, Lp + 1)
    Fm = np.fft.fftshift(np.fft.fft(ext, axis=1), axes=1) / N
    Fm = Fm * np.exp(-1j * np.pi * mp / N)[None, :, None]
    F = np.ascontiguousarray(np.transpose(Fm, (0, 2, 1)))
    return F[0] if single else F


def torus_coeffs(f, L, s, parity="spin"):
    """Torus Fourier coefficients of the extended samples: phi DFT, extension, theta DFT
    (Secs. 3.2 and 3.4.1; equal to eqn dft_spatial applied to the extended function)."""
    return theta_analysis(torus_extend(phi_analysis(f, L), L, s, parity), L)


def weight_conv(F, L):
    """G_{m m'} = 2 pi sum_{m''} F_{m m''} w(m'' - m'), w(p) = int_0^pi sin(theta) e^{i p theta} d theta."""
    F, single = _as_batch(F, 3)
    B = F.shape[0]
    G = np.zeros_like(F)
    _lib.check(_lib.lib().oracle_weight_conv(L, B, _lib.ptr(F), _lib.ptr(G)), "weight_conv")
    return G[0] if single else G


def harmonic_project(X, L, s):
    """sf_lm = (-1)^s i^{m+s} sqrt((2l+1)/4pi) sum_{m'=-l}^{l} Delta^l_{m'm} Delta^l_{m',-s} X_{m m'}."""
    X, single = _as_batch(X, 3)
    B = X.shape[0]
    flm = np.zeros((B, L * L), dtype=np.complex128)
    _lib.check(_lib.lib().oracle_harmonic_project(L, s, B, _lib.ptr(X), _lib.ptr(flm)), "harmonic_project")
    return flm[0] if single else flm


def forward(f, L, s):
    """Forward spin transform by exact quadrature of eqn ssht_fwd on the torus: phi DFT, per-m
    parity extension, theta DFT (F), the sin(theta) weight convolution (G), harmonic projection.
    Exact for band-limited f (the product sin(theta) f_m(theta) e^{-i m' theta} is integrated
    exactly because F holds every Fourier mode of f_m)."""
    F = torus_coeffs(f, L, s)
    G = weight_conv(F, L)
    return harmonic_project(G, L, s)


def adjoint(g, L, s):
    """Adjoint of ``inverse``: H_{m m'} = sum_{t<L, p} g[t, p] e^{-i(m' theta_t + m phi_p)}
    (no extension, no weight), then the conjugate transpose of eqn fourier_coeff."""
    g, single = _as_batch(g, 3)
    Lp, N = sizes(L)
    B = g.shape[0]
    X = phi_analysis(g, L) * N                       # sum_p g e^{-i m phi_p}: [b, t, m]
    pad = np.zeros((B, N, N), dtype=np.complex128)
    pad[:, :L, :] = X
    H = theta_analysis(pad, L) * N                   # sum_{t<L} X e^{-i m' theta_t}: [b, m, m']
    flm = harmonic_project(H, L, s)
    return flm[0] if single else flm


def forward_triangular(f, L, s):
    """The paper's forward transform (Sec. 3.4.2): F^e and F^o from the even and odd torus
    extensions (eqn dft_spatial), then per m the triangular system eqn matrix_fwd solved by
    back substitution, taking F^e for even m+s and F^o for odd m+s."""
    f, single = _as_batch(f, 3)
    B = f.shape[0]
    Fe = np.ascontiguousarray(torus_coeffs(f, L, s, "even"))
    Fo = np.ascontiguousarray(torus_coeffs(f, L, s, "odd"))
    if Fe.ndim == 2:
        Fe, Fo = Fe[None], Fo[None]
    flm = np.zeros((B, L * L), dtype=np.complex128)
    _lib.check(_lib.lib().oracle_triangular_forward(L, s, B, _lib.ptr(Fe), _lib.ptr(Fo), _lib.ptr(flm)),
               "triangular_forward")
    return flm[0] if single else flm


def triangular_matrix(L, s, m):
    """Matrix of eqn matrix_fwd for one m: rows m' = 0..Lp, columns l = 0..Lp."""
    D = np.zeros((L, L), dtype=np.complex128)
    _lib.check(_lib.lib().oracle_triangular_matrix(L, s, m, _lib.ptr(D)), "triangular_matrix")
    return D


def num_threads():
    return _lib.lib().oracle_num_threads()


# ---------------------------------------------------------------------------
# Error metrics of Sec. 4.2
# ---------------------------------------------------------------------------

def error_metrics(f, g):
    """The five error metrics of Sec. 4.2 between coefficient sets f (original) and g
    (reconstructed), plus the max-norm relative error max|f-g| / max|f|."""
    d = np.abs(np.asarray(f) - np.asarray(g)).ravel()
    fa = np.abs(np.asarray(f)).ravel()
    return {
        "max": float(d.max()),
        "mean": float(d.mean()),
        "median": float(np.median(d)),
        "rms": float(np.sqrt(np.mean(d * d))),
        "rel_rms": float(np.sqrt(np.sum(d * d) / np.sum(fa * fa))),
        "rel_max": float(d.max() / fa.max()),
    }
