"""FP64 CPU oracle for the matrix-valued quantum lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and the two share no code.

The arithmetic lives in ``qlbm_oracle.c`` (plain C, double precision, every
population kept as a literal complex 2x2 matrix, each step following Sec. 3.3
of Mendl, "Matrix-valued Quantum Lattice Boltzmann Method").  This module
only compiles it with gcc and marshals numpy arrays through ctypes.

Array conventions (identical to the library's canonical C-ABI layout so that
results compare element by element):
  state   float64 [b][4][N]  Pauli components (f, s_x, s_y, s_z) of every W_i,
                             W = (f 1 + s.sigma)/2, site = x + nx*(y + ny*z)
  rho4    float64 [4][N]     (tr rho, tr rho sigma_x, tr rho sigma_y, tr rho sigma_z)
  u       float64 [d][N]     local velocity
  eps     float64 [N]        local internal energy
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qlbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)


def _same_arch(path):
    """True if the ELF file was built for this machine's architecture."""
    import platform
    want = {"x86_64": 62, "amd64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine().lower())
    try:
        with open(path, "rb") as f:
            h = f.read(20)
    except OSError:
        return False
    return h[:4] == b"\x7fELF" and int.from_bytes(h[18:20], "little") == want


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction, OpenMP over sites)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and _same_arch(_LIB)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_zeta.restype = _d
        lib.oracle_zeta.argtypes = [_d]
        lib.oracle_eps0.restype = _d
        lib.oracle_eps0.argtypes = [_i, _d]
        lib.oracle_constants.restype = _i
        lib.oracle_constants.argtypes = [_i, _d, _pd]
        lib.oracle_max_threads.restype = _i
        lib.oracle_max_threads.argtypes = [_i]
        lib.oracle_run.restype = _i
        lib.oracle_run.argtypes = [_i, _pi64, _d, _d, _d, _i64, _pd, _i]
        lib.oracle_run_matrix.restype = _i
        lib.oracle_run_matrix.argtypes = [_i, _pi64, _d, _d, _d, _i64, _pd, _i]
        lib.oracle_collide_site.restype = _i
        lib.oracle_collide_site.argtypes = [_i, _d, _d, _d, _pd, _pd]
        lib.oracle_equilibrium_site.restype = _i
        lib.oracle_equilibrium_site.argtypes = [_i, _d, _pd, _pd, _d, _pd]
        lib.oracle_init_equilibrium.restype = _i
        lib.oracle_init_equilibrium.argtypes = [_i, _pi64, _d, _pd, _pd, _pd, _pd]
        lib.oracle_moments.restype = _i
        lib.oracle_moments.argtypes = [_i, _pi64, _d, _pd, _pd, _pd, _pd]
        lib.oracle_conserved.restype = _i
        lib.oracle_conserved.argtypes = [_i, _pi64, _d, _pd, _pd]
        lib.oracle_eq_min_eigenvalues.restype = _i
        lib.oracle_eq_min_eigenvalues.argtypes = [_i, _pi64, _d, _pd, _pd]
        lib.oracle_adjoint_step.restype = _i
        lib.oracle_adjoint_step.argtypes = [_i, _pi64, _d, _d, _d, _pd, _pd, _pd, _pd, _i]
        lib.oracle_set_field.restype = None
        lib.oracle_set_field.argtypes = [_d, _d, _d, _d]
        lib.oracle_set_field_array.restype = _i
        lib.oracle_set_field_array.argtypes = [_d, _pd, _i64]
        lib.oracle_fd.restype = _d
        lib.oracle_fd.argtypes = [_d, _d]
        lib.oracle_fd_moments.restype = _i
        lib.oracle_fd_moments.argtypes = [_i, _d, _d, _d, _pd]
        lib.oracle_fd_params.restype = _i
        lib.oracle_fd_params.argtypes = [_i, _pd, _d, _pd]
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_pd)


def _dims(d, dims):
    dims = tuple(int(v) for v in dims)
    if d == 2 and len(dims) == 2:
        dims = dims + (1,)
    if len(dims) != 3:
        raise ValueError("dims must have 3 entries (nz = 1 for 2D)")
    return (ctypes.c_int64 * 3)(*dims), dims[0] * dims[1] * (dims[2] if d == 3 else 1)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError("oracle %s failed (rc=%d)" % (what, rc))


def nq(d):
    return 9 if d == 2 else 19


def zeta(s):
    return _load().oracle_zeta(float(s))


def eps0(d, beta0):
    return _load().oracle_eps0(int(d), float(beta0))


def constants(d, beta0):
    """Lattice constants of Sec. 3.1 and the appendix as a dict."""
    out = np.zeros(16 + 4 * 19, np.float64)
    k = _load().oracle_constants(int(d), float(beta0), _ptr(out))
    _check(k, "constants")
    names = ["a", "xi", "alpha_fac", "A1_0", "A1_1", "A2_0", "A2_1", "alpha3", "alpha4", "alpha5"]
    c = {n: float(out[j]) for j, n in enumerate(names)}
    b = int(out[10])
    c["b"] = b
    c["w"] = out[11:11 + b].copy()
    c["idx"] = out[11 + b:11 + 4 * b].reshape(b, 3).astype(np.int64)
    return c


def max_threads(nthreads=0):
    return _load().oracle_max_threads(int(nthreads))


def run(d, dims, tau, beta0, nsteps, state, dt=1.0, nthreads=0):
    """Advance a canonical Pauli state [b][4][N] by nsteps (returns a copy)."""
    cd, N = _dims(d, dims)
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(nq(d), 4, N).copy()
    _check(_load().oracle_run(d, cd, tau, beta0, dt, int(nsteps), _ptr(st), int(nthreads)), "run")
    return st


def run_matrix(d, dims, tau, beta0, nsteps, W, dt=1.0, nthreads=0):
    """Advance a complex matrix state W[N][b][2][2] (complex128) by nsteps."""
    cd, N = _dims(d, dims)
    Wc = np.ascontiguousarray(W, dtype=np.complex128).reshape(N, nq(d), 2, 2).copy()
    view = Wc.view(np.float64)
    _check(_load().oracle_run_matrix(d, cd, tau, beta0, dt, int(nsteps),
                                     view.ctypes.data_as(_pd), int(nthreads)), "run_matrix")
    return Wc


def collide_site(d, tau, beta0, pops, dt=1.0):
    """Collision (no streaming) of one site's populations given as [b][4]."""
    pin = np.ascontiguousarray(pops, dtype=np.float64).reshape(nq(d), 4)
    out = np.zeros_like(pin)
    _check(_load().oracle_collide_site(d, tau, beta0, dt, _ptr(pin), _ptr(out)), "collide_site")
    return out


def equilibrium_site(d, beta0, rho4, u, eps):
    """W_i^eq of Eq. WeqAlgo for one site, as [b][4] Pauli components."""
    r = np.ascontiguousarray(rho4, dtype=np.float64).reshape(4)
    uu = np.zeros(3, np.float64)
    uu[:d] = np.asarray(u, dtype=np.float64)[:d]
    out = np.zeros((nq(d), 4), np.float64)
    _check(_load().oracle_equilibrium_site(d, beta0, _ptr(r), _ptr(uu), float(eps), _ptr(out)),
           "equilibrium_site")
    return out


def init_equilibrium(d, dims, beta0, rho4, u, eps=None):
    cd, N = _dims(d, dims)
    r = np.ascontiguousarray(rho4, dtype=np.float64).reshape(4, N)
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(d, N)
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64).reshape(N)
    st = np.zeros((nq(d), 4, N), np.float64)
    _check(_load().oracle_init_equilibrium(d, cd, beta0, _ptr(r), _ptr(uu), _ptr(e), _ptr(st)),
           "init_equilibrium")
    return st


def moments(d, dims, beta0, state):
    cd, N = _dims(d, dims)
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(nq(d), 4, N)
    rho4 = np.zeros((4, N))
    u = np.zeros((d, N))
    eps = np.zeros(N)
    _check(_load().oracle_moments(d, cd, beta0, _ptr(st), _ptr(rho4), _ptr(u), _ptr(eps)),
           "moments")
    return rho4, u, eps


def conserved(d, dims, beta0, state):
    cd, N = _dims(d, dims)
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(nq(d), 4, N)
    out = np.zeros(8)
    _check(_load().oracle_conserved(d, cd, beta0, _ptr(st), _ptr(out)), "conserved")
    return out


def eq_min_eigenvalues(d, dims, beta0, state):
    """Smallest eigenvalue of every W_i^eq (Eq. WeqAlgo) built from the
    state's moments, [b][N] (Sec. 3.2 end: negative values are not clipped)."""
    cd, N = _dims(d, dims)
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(nq(d), 4, N)
    out = np.zeros((nq(d), N))
    _check(_load().oracle_eq_min_eigenvalues(d, cd, beta0, _ptr(st), _ptr(out)), "eq_min_eigenvalues")
    return out


def negative_eq(d, dims, beta0, state):
    """(count, mask): the number of (site, direction) pairs whose W_i^eq has a
    negative eigenvalue, and per site the bit mask of those directions."""
    lmin = eq_min_eigenvalues(d, dims, beta0, state)
    neg = lmin < 0.0
    mask = np.zeros(neg.shape[1], np.uint32)
    for q in range(neg.shape[0]):
        mask |= neg[q].astype(np.uint32) << np.uint32(q)
    return int(neg.sum()), mask


def adjoint_step(d, dims, tau, beta0, state, lam_next, dt=1.0, nthreads=0):
    """Cotangent of W^n from that of W^{n+1}; returns (lam_n, dJ/dtau part)."""
    cd, N = _dims(d, dims)
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(nq(d), 4, N)
    ln = np.ascontiguousarray(lam_next, dtype=np.float64).reshape(nq(d), 4, N)
    lam = np.zeros_like(ln)
    g = np.zeros(1)
    _check(_load().oracle_adjoint_step(d, cd, tau, beta0, dt, _ptr(st), _ptr(ln), _ptr(lam),
                                       _ptr(g), int(nthreads)), "adjoint_step")
    return lam, float(g[0])


def fd(k, x):
    """Complete Fermi-Dirac integral F_k(x) (Sec. 2.2)."""
    return _load().oracle_fd(float(k), float(x))


def fd_moments(d, beta, mu_up, mu_dn):
    """(n_up, n_dn, eps) of the FD distribution (Eqs. nFDstdOmega, energyFDstdOmega)."""
    out = np.zeros(3)
    _check(_load().oracle_fd_moments(int(d), float(beta), float(mu_up), float(mu_dn), _ptr(out)),
           "fd_moments")
    return out


def fd_params(d, rho4, eps):
    """(status, [beta, mu_up, mu_dn, a_x, a_y, a_z]) from rho (Pauli) and eps (Prop. 1)."""
    r = np.ascontiguousarray(rho4, dtype=np.float64).reshape(4)
    out = np.zeros(6)
    rc = _load().oracle_fd_params(int(d), _ptr(r), float(eps), _ptr(out))
    return rc, out


def set_field(mu, B):
    """Uniform external magnetic field for the following runs (mu = 0: off)."""
    _load().oracle_set_field(float(mu), float(B[0]), float(B[1]), float(B[2]))


def set_field_array(mu, B):
    """Per-site external magnetic field B [3][N] for the following runs on
    N-site lattices (None: off)."""
    if B is None:
        _check(_load().oracle_set_field_array(0.0, None, 0), "set_field_array")
        return
    b = np.ascontiguousarray(B, dtype=np.float64).reshape(3, -1)
    _check(_load().oracle_set_field_array(float(mu), _ptr(b), b.shape[1]), "set_field_array")
