"""Brute-force and closed-form checks for the Wilson-Dirac oracle (test infrastructure).

* dense_wilson(): the 12V x 12V matrix of M, built entry block by entry block
  from the definition with pure-Python site loops (tiny lattices only).
* gammas(): the chiral gamma matrices as Kronecker products of Pauli matrices
  (a construction independent of the C oracle's element-wise tables).
* free_eigenvalues(): closed-form spectrum of M at unit links.
* free_solve_fft(): exact solve of M x = b at unit links by Fourier transform.

Convention (textbook Wilson, r = 1; the paper fixes none):
  M = 1 - kappa sum_mu [ eta (1 - g_mu) U_mu(x) delta_{y,x+mu}
                        + eta (1 + g_mu) U_mu(x-mu)^dag delta_{y,x-mu} ]
with eta = t_bc on hops across the t boundary.
"""
from __future__ import annotations

import itertools

import numpy as np

_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def gammas():
    """g_1..g_3 = sigma_y (x) sigma_k, g_4 = sigma_x (x) 1; returns (g[4], g5)."""
    g = [np.kron(_SY, _SX), np.kron(_SY, _SY), np.kron(_SY, _SZ), np.kron(_SX, _I2)]
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def _coords(dims):
    lx, ly, lz, lt = dims
    for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        yield (x, y, z, t)


def _index(dims, c):
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def dense_wilson(dims, U, kappa, t_bc=-1, mu=0.0):
    """Dense M (12V x 12V); row index = 12*site + 3*spin + colour. mu != 0 adds the
    twisted-mass term 2 i kappa mu g5 on the diagonal."""
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(V, 4, 3, 3)
    g, g5 = gammas()
    one = np.eye(4, dtype=np.complex128)
    M = np.eye(12 * V, dtype=np.complex128)
    if mu != 0.0:
        M = M + np.kron(np.eye(V), np.kron(2j * kappa * mu * g5, np.eye(3)))
    for c in _coords(dims):
        s = _index(dims, c)
        for mu in range(4):
            fwd = list(c)
            fwd[mu] = (c[mu] + 1) % dims[mu]
            bwd = list(c)
            bwd[mu] = (c[mu] - 1) % dims[mu]
            eta_f = t_bc if (mu == 3 and c[3] == dims[3] - 1) else 1
            eta_b = t_bc if (mu == 3 and c[3] == 0) else 1
            sf = _index(dims, fwd)
            sb = _index(dims, bwd)
            blk_f = -kappa * eta_f * np.kron(one - g[mu], U[s, mu])
            blk_b = -kappa * eta_b * np.kron(one + g[mu], np.conj(U[sb, mu]).T)
            M[12 * s:12 * s + 12, 12 * sf:12 * sf + 12] += blk_f
            M[12 * s:12 * s + 12, 12 * sb:12 * sb + 12] += blk_b
    return M


def parity_mask(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1)


def momenta(dims, t_antiperiodic=True):
    """All lattice momenta p = (2 pi n_k / L_k, (2 pi n_t + pi) / L_t)."""
    lx, ly, lz, lt = dims
    shift = np.pi if t_antiperiodic else 0.0
    out = []
    for nt, nz, ny, nx in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        out.append((2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz,
                    (2 * np.pi * nt + shift) / lt))
    return np.array(out)


def free_eigenvalues(dims, kappa, t_antiperiodic=True, mu=0.0):
    """1 - 2 kappa sum cos p +- 2 i kappa sqrt(sum sin^2 p + mu^2), each 6-fold: with
    K = sum g_mu sin p_mu + mu g5, K^2 = (sum sin^2 p + mu^2) 1 since g5 anticommutes
    with every g_mu."""
    ev = []
    for p in momenta(dims, t_antiperiodic):
        a = 1 - 2 * kappa * np.sum(np.cos(p))
        b = 2 * kappa * np.sqrt(np.sum(np.sin(p) ** 2) + mu * mu)
        ev += [a + 1j * b] * 6 + [a - 1j * b] * 6
    return np.array(ev)


def free_symbol(p, kappa):
    """4x4 spin matrix M(p) = 1 - 2 kappa sum cos p_mu + 2 i kappa sum g_mu sin p_mu."""
    g, _ = gammas()
    m = (1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu]) * g[mu]
    return m


def free_solve_fft(dims, kappa, b, t_antiperiodic=True):
    """Exact M^{-1} b at unit links: twist t to periodic, FFT, invert M(p) per momentum."""
    lx, ly, lz, lt = dims
    b = np.asarray(b).reshape(lt, lz, ly, lx, 4, 3)
    tt = np.arange(lt).reshape(lt, 1, 1, 1, 1, 1)
    shift = np.pi / lt if t_antiperiodic else 0.0
    phi = b * np.exp(-1j * shift * tt)
    phik = np.fft.fftn(phi, axes=(0, 1, 2, 3))
    kt = 2 * np.pi * np.fft.fftfreq(lt) * 1.0
    kz = 2 * np.pi * np.fft.fftfreq(lz)
    ky = 2 * np.pi * np.fft.fftfreq(ly)
    kx = 2 * np.pi * np.fft.fftfreq(lx)
    g, _ = gammas()
    PT, PZ, PY, PX = np.meshgrid(kt + shift, kz, ky, kx, indexing="ij")
    m = np.zeros((lt, lz, ly, lx, 4, 4), dtype=np.complex128)
    cs = np.cos(PX) + np.cos(PY) + np.cos(PZ) + np.cos(PT)
    m += (1 - 2 * kappa * cs)[..., None, None] * np.eye(4)
    for mu, P in enumerate((PX, PY, PZ, PT)):
        m += (2j * kappa * np.sin(P))[..., None, None] * g[mu]
    xk = np.linalg.solve(m, phik)  # solves per momentum, colour as extra rhs columns
    x = np.fft.ifftn(xk, axes=(0, 1, 2, 3)) * np.exp(1j * shift * tt)
    return x.reshape(-1, 4, 3)


def gauge_transform_links(dims, U, g):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    dims = tuple(int(d) for d in dims)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    U = np.asarray(U).reshape(lt, lz, ly, lx, 4, 3, 3)
    G = np.asarray(g).reshape(lt, lz, ly, lx, 3, 3)
    out = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> array axis
    for mu in range(4):
        Gf = np.roll(G, -1, axis=axes[mu])  # g(x + mu)
        out[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gf, -1, -2))
    return out.reshape(V, 4, 3, 3)


def gauge_transform_spinor(g, psi):
    """(g psi)(x) = g(x) psi(x) on colour."""
    return np.einsum("sab,sib->sia", g, psi)
