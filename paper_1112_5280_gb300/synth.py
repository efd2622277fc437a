"""Seeded synthetic inputs for the Wilson-Dirac solver: gauge links, spinors, sources.

This module is the only code shared by the oracle and the CUDA path. It draws
random numbers and builds input arrays; it holds none of the operator's
arithmetic (no hopping term, no gamma matrices, no solver step).

Host layout (the library's interchange format, also used by the oracle):
  * site index  s = x + Lx*(y + Ly*(z + Lz*t)),   x fastest, t slowest
  * links       U[s, mu, row, col]  complex128, mu = 0..3 for x, y, z, t;
                U[s, mu] sits on the bond s -> s + mu_hat
  * spinors     psi[s, spin, colour] complex128

Workload recipe (Section 3 of the paper reports the even-odd Dslash on
synthetic-size lattices; the link ensemble itself is not specified there):
  * link U = exp(i*eps*H), H = (A + A^dag)/2 - tr(.)/3, A with i.i.d. N(0,1)
    real and imaginary parts, exponentiated through a Hermitian
    eigendecomposition and re-unitarised (Gram-Schmidt on rows 0 and 1,
    row 2 = conj(row0 x row1)) so that det U = 1 to rounding;
  * spinor entries: real and imaginary parts i.i.d. N(0,1).
"""
from __future__ import annotations

import numpy as np

SEED_LINKS = 1001
SEED_SOURCE = 2002
SEED_POINT_SITE = 3003
SEED_ARRIVALS = 4004


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def site_index(dims, x, y, z, t) -> int:
    lx, ly, lz, _ = dims
    return x + lx * (y + ly * (z + lz * t))


def site_coords(dims, s):
    lx, ly, lz, _ = dims
    x = s % lx
    s //= lx
    y = s % ly
    s //= ly
    z = s % lz
    t = s // lz
    return x, y, z, t


def parity_of_sites(dims) -> np.ndarray:
    """Checkerboard parity (x+y+z+t) mod 2 for every site, in host order."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1).astype(np.int8)


def _gaussian_complex(rng, shape) -> np.ndarray:
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt rows 0 and 1, then row 2 = conj(row0 x row1) (det = 1)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(n: int, eps: float, rng) -> np.ndarray:
    """n matrices exp(i*eps*H) with H random traceless Hermitian, re-unitarised."""
    a = _gaussian_complex(rng, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    chunk = 1 << 20
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        w, v = np.linalg.eigh(h[lo:hi])
        ph = np.exp(1j * eps * w)
        out[lo:hi] = np.einsum("nij,nj,nkj->nik", v, ph, np.conj(v))
    return _reunitarise(out)


def random_links(dims, eps: float, seed: int = SEED_LINKS) -> np.ndarray:
    """Gauge field U[V, 4, 3, 3] with U = exp(i*eps*H) per link."""
    rng = np.random.default_rng(seed)
    v = volume(dims)
    return random_su3(4 * v, eps, rng).reshape(v, 4, 3, 3)


def unit_links(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gaussian_spinor(dims, seed: int = SEED_SOURCE) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _gaussian_complex(rng, (volume(dims), 4, 3))


def gaussian_momenta(dims, seed: int) -> np.ndarray:
    """HMC momenta P[V, 4, 3, 3]: P = i H, H traceless Hermitian with density
    ~ exp(-Tr(H^2) / 2) (a GUE sample with its trace removed), so that
    ~ exp(-sum |P_ij|^2 / 2)."""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    a = _gaussian_complex(rng, (V, 4, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    h = h - (np.trace(h, axis1=-2, axis2=-1) / 3)[..., None, None] * np.eye(3)
    return 1j * h


def gauge_transform_field(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix g(x) per site, for gauge-covariance checks."""
    rng = np.random.default_rng(seed)
    return random_su3(volume(dims), np.pi, rng)


def point_site(dims, seed: int = SEED_POINT_SITE) -> int:
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, volume(dims)))


def point_source(dims, site: int, spin: int, colour: int) -> np.ndarray:
    b = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def plane_wave(dims, n, chi: np.ndarray, t_antiperiodic: bool = True) -> np.ndarray:
    """psi(x) = exp(i p.x) chi with p_k = 2 pi n_k / L_k (t: +pi/L_t if antiperiodic)."""
    lx, ly, lz, lt = dims
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
         (2 * np.pi * n[3] + (np.pi if t_antiperiodic else 0.0)) / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t)).reshape(-1)
    return phase[:, None, None] * chi[None, :, :], p


def lattice_sample(rng, sizes, weights):
    """Draw one lattice shape from a weighted list."""
    i = rng.choice(len(sizes), p=np.asarray(weights) / np.sum(weights))
    return tuple(sizes[i])
