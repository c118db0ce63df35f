"""Seeded synthetic input fields shaped like the paper's 2D and 3D tests.

This module produces only *inputs*: per-site density matrices (as Pauli
densities), velocities, internal energies and raw population arrays.  It
holds none of the lattice Boltzmann arithmetic (no weights, no lattice
constant, no equilibrium), so the CUDA library and the test oracle can both
consume its output without sharing any of the method's code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
evaluated as ``mix(seed_key + (counter + 1) * 0x9E3779B97F4A7C15)``; uniform
doubles take the top 53 bits and normals use the Box-Muller transform.

Workloads (site index = x + nx*(y + ny*z); arrays are SoA, site fastest):
  * ``blob2d``   -- 2D periodic: n = 1 + 0.05 sin(2 pi x / nx), a Gaussian
                    spin-polarised blob |r| = 0.1 n exp(-|x-c|^2 / (2 sigma^2))
                    along a seeded random unit Bloch direction, u = 0.
  * ``modes``    -- density, velocity and spin as sums of Fourier modes with
                    integer wave vectors 1 <= |k| <= kmax; each field's
                    coefficients are N(0,1) draws rescaled so that its RMS over
                    the periodic box equals ``amp`` (Parseval), the velocity
                    rescaled so that |u| <= umax holds everywhere (triangle
                    inequality on the coefficients).
  * ``shear2d``  -- doubly periodic double shear layer: u_x = +-U0 tanh bands
                    of width ``delta`` cells, seeded transverse noise in u_y,
                    spin +z 0.1 n in one band and -z 0.1 n in the other.
  * ``random_populations`` -- arbitrary positive populations (f_i > |s_i|),
                    used for parity cases away from equilibrium.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed, stream):
    """Per-(seed, stream) key: one SplitMix64 output of the pair."""
    s = np.array([(int(seed) * 1000003 + int(stream)) & 0xFFFFFFFFFFFFFFFF], np.uint64)
    return _mix(s)[0]


def splitmix64(seed, stream, counters):
    """SplitMix64 outputs at the given counters (uint64 array)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + (c + np.uint64(1)) * _GOLDEN
        return _mix(z)


def uniform(seed, stream, n, offset=0):
    """n doubles in [0, 1) from counters offset .. offset+n-1."""
    c = np.arange(offset, offset + n, dtype=np.uint64)
    return (splitmix64(seed, stream, c) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, stream, n, offset=0):
    """n standard normals by Box-Muller from pairs of uniforms."""
    m = (n + 1) // 2
    u1 = uniform(seed, stream, m, 2 * offset)
    u2 = uniform(seed, stream + 7777, m, 2 * offset)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    th = 2.0 * np.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:n]


def unit_vector(seed, stream):
    """A uniformly distributed unit vector on S^2 (normalised Gaussian)."""
    g = normal(seed, stream, 3)
    return g / np.linalg.norm(g)


def _coords(dims):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)


def _dims3(d, dims):
    dims = tuple(int(v) for v in dims)
    if len(dims) == 2:
        dims = dims + (1,)
    if d == 2:
        dims = (dims[0], dims[1], 1)
    return dims


def blob2d(nx=64, ny=64, seed=1, sigma=8.0, dens_amp=0.05, spin_amp=0.1):
    """Density wave plus Gaussian spin blob, zero velocity (2D)."""
    x, y, _ = _coords((nx, ny, 1))
    n = 1.0 + dens_amp * np.sin(2.0 * np.pi * x / nx)
    cx, cy = nx / 2.0, ny / 2.0
    g = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * sigma ** 2))
    axis = unit_vector(seed, 11)
    rho4 = np.zeros((4, nx * ny))
    rho4[0] = n
    for k in range(3):
        rho4[1 + k] = spin_amp * n * g * axis[k]
    u = np.zeros((2, nx * ny))
    return dict(rho4=rho4, u=u, eps=None)


def _mode_list(d, kmax):
    """Integer wave vectors with 1 <= |k| <= kmax, one of each +-k pair."""
    r = range(-kmax, kmax + 1)
    ks = []
    for kz in (r if d == 3 else [0]):
        for ky in r:
            for kx in r:
                k = (kx, ky, kz)
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                if k > tuple(-v for v in k):  # keep the lexicographically smaller one
                    continue
                ks.append(k)
    return np.array(ks, dtype=np.float64)


class ModeField:
    """Real Fourier sum  sum_k A_k cos(2 pi k.x/L) + B_k sin(2 pi k.x/L)."""

    def __init__(self, d, dims, seed, stream, kmax):
        self.dims = _dims3(d, dims)
        self.k = _mode_list(d, kmax)
        m = len(self.k)
        g = normal(seed, stream, 2 * m)
        self.A = g[:m]
        self.B = g[m:]

    def rms(self):
        return float(np.sqrt(0.5 * np.sum(self.A ** 2 + self.B ** 2)))

    def bound(self):
        return float(np.sum(np.sqrt(self.A ** 2 + self.B ** 2)))

    def at(self, sites):
        """Field values at flat site indices (direct sum, float64)."""
        nx, ny, nz = self.dims
        s = np.asarray(sites, dtype=np.int64)
        x = (s % nx).astype(np.float64)
        y = ((s // nx) % ny).astype(np.float64)
        z = (s // (nx * ny)).astype(np.float64)
        out = np.zeros(s.shape, np.float64)
        for (kx, ky, kz), a, b in zip(self.k, self.A, self.B):
            ph = 2.0 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz)
            out += a * np.cos(ph) + b * np.sin(ph)
        return out

    def grid(self):
        """Field on the whole periodic grid, via a real inverse FFT."""
        nx, ny, nz = self.dims
        spec = np.zeros((nz, ny, nx), np.complex128)
        for (kx, ky, kz), a, b in zip(self.k, self.A, self.B):
            # a cos(ph) + b sin(ph) = Re[(a - i b) e^{i ph}]
            c = 0.5 * (a - 1j * b)
            i0, i1, i2 = int(kz) % nz, int(ky) % ny, int(kx) % nx
            spec[i0, i1, i2] += c
            spec[(-int(kz)) % nz, (-int(ky)) % ny, (-int(kx)) % nx] += np.conj(c)
        f = np.fft.ifftn(spec) * (nx * ny * nz)
        return np.ascontiguousarray(f.real).ravel()


def mode_spec(d, dims, seed=2, kmax=4, amp=0.02, umax=0.05):
    """The Fourier-mode workload as data: for each output row a tuple
    (ModeField, scale, offset), the row's values being offset + scale *
    field.  dict(rho4=[4 rows], u=[d rows], eps=None)."""
    dims = _dims3(d, dims)
    fn = ModeField(d, dims, seed, 100, kmax)
    fu = [ModeField(d, dims, seed, 200 + c, kmax) for c in range(d)]
    fr = [ModeField(d, dims, seed, 300 + c, kmax) for c in range(3)]
    ub = np.sqrt(sum(f.bound() ** 2 for f in fu))
    uscale = umax / ub
    rho4 = [(fn, amp / fn.rms(), 1.0)] + [(fr[c], amp / fr[c].rms(), 0.0) for c in range(3)]
    u = [(fu[c], uscale, 0.0) for c in range(d)]
    return dict(rho4=rho4, u=u, eps=None)


def modes(d, dims, seed=2, kmax=4, amp=0.02, umax=0.05, sites=None):
    """Fourier-mode density / velocity / spin fields (zero-mean perturbations).

    Returns dict(rho4 [4][M], u [d][M], eps=None) on the full grid, or at the
    given flat ``sites`` only (then M = len(sites))."""
    dims = _dims3(d, dims)
    spec = mode_spec(d, dims, seed, kmax, amp, umax)

    def ev(f):
        return f.grid() if sites is None else f.at(sites)

    M = int(np.prod(dims)) if sites is None else len(sites)
    rho4 = np.empty((4, M))
    for c, (f, scale, offset) in enumerate(spec["rho4"]):
        rho4[c] = offset + scale * ev(f)
    u = np.empty((d, M))
    for c, (f, scale, offset) in enumerate(spec["u"]):
        u[c] = offset + scale * ev(f)
    return dict(rho4=rho4, u=u, eps=None)


def shear2d(nx=4096, ny=4096, seed=3, U0=0.04, delta=80.0, noise=1e-3, spin=0.1):
    """Double shear layer with opposite spin polarisation in the two bands."""
    x, y, _ = _coords((nx, ny, 1))
    y1, y2 = ny / 4.0, 3.0 * ny / 4.0
    prof = np.where(y <= ny / 2.0, np.tanh((y - y1) / delta), np.tanh((y2 - y) / delta))
    N = nx * ny
    u = np.zeros((2, N))
    u[0] = U0 * prof
    u[1] = noise * normal(seed, 21, N)
    rho4 = np.zeros((4, N))
    rho4[0] = 1.0
    rho4[3] = spin * rho4[0] * prof
    return dict(rho4=rho4, u=u, eps=None)


def dichotomic3d(L=32, spin=0.1, umax=0.05, sharp=4.0):
    """Uniform density, Bloch vectors along z with a dichotomic outline
    r_z = spin tanh(sharp sin(2 pi x/L) sin(2 pi y/L)) and a velocity along x
    proportional to r_z (|u_x| <= umax): the shape of the paper's 3D
    convergence example (its exact outline is not given)."""
    x, y, _ = _coords((L, L, L))
    prof = np.tanh(sharp * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L))
    N = L ** 3
    rho4 = np.zeros((4, N))
    rho4[0] = 1.0
    rho4[3] = spin * prof
    u = np.zeros((3, N))
    u[0] = umax * prof
    return dict(rho4=rho4, u=u, eps=None)


def random_fields(d, dims, seed=4, umax=0.2, eps_range=(0.8, 2.2), spin_frac=0.6):
    """Random per-site (rho, u, eps): n in [0.5, 1.5], |S| < spin_frac * n."""
    dims = _dims3(d, dims)
    N = int(np.prod(dims))
    n = 0.5 + uniform(seed, 31, N)
    axis = normal(seed, 32, 3 * N).reshape(3, N)
    axis /= np.linalg.norm(axis, axis=0)
    mag = spin_frac * n * uniform(seed, 33, N)
    rho4 = np.vstack([n, mag * axis])
    u = umax * (2.0 * uniform(seed, 34, d * N).reshape(d, N) - 1.0) / np.sqrt(d)
    lo, hi = eps_range
    eps = lo + (hi - lo) * uniform(seed, 35, N)
    return dict(rho4=rho4, u=u, eps=eps)


def random_populations(d, dims, seed=5, fmin=0.02, fmax=0.2, spin_frac=0.8):
    """Positive populations away from equilibrium: f_i in [fmin, fmax],
    |s_i| < spin_frac * f_i.  Returns the canonical Pauli array [b][4][N]."""
    dims = _dims3(d, dims)
    N = int(np.prod(dims))
    b = 9 if d == 2 else 19
    f = fmin + (fmax - fmin) * uniform(seed, 41, b * N).reshape(b, N)
    ax = normal(seed, 42, 3 * b * N).reshape(b, 3, N)
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    mag = spin_frac * f * uniform(seed, 43, b * N).reshape(b, N)
    st = np.empty((b, 4, N))
    st[:, 0] = f
    st[:, 1:] = ax * mag[:, None, :]
    return st
