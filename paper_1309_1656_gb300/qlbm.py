"""Python binding of the C ABI in ``include/qlbm.h`` (argument marshalling only).

Every function here forwards to the entry point of the same name in the
in-tree CUDA library ``_build/libqlbm.so``; all arithmetic of the lattice
Boltzmann step runs in that library's kernels.  Arrays may be numpy arrays
(host memory) or CUDA torch tensors (device memory of the handle's GPU);
both must be C-contiguous float64 in the layouts the header documents.

Importing this module fails loudly if the library has not been built: there
is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import _build

QLBM_OK = 0
QLBM_ERR_INVALID_ARG = -1
QLBM_ERR_UNSUPPORTED = -2
QLBM_ERR_OOM = -3
QLBM_ERR_CUDA = -4
QLBM_ERR_NONFINITE = -5
QLBM_ERR_NONPOSITIVE_DENSITY = -6
QLBM_ERR_STATE = -7

QLBM_D2Q9 = 2
QLBM_D3Q19 = 3
QLBM_FP64 = 0
QLBM_FP32 = 1
QLBM_FP16_DEV = 2
QLBM_DF64 = 3
QLBM_FP64_DF = 4
QLBM_HOST = 0
QLBM_DEVICE = 1
QLBM_EQ_DIRECT = 0
QLBM_EQ_FD_PARAMS = 1

PRECISIONS = {"fp64": QLBM_FP64, "fp32": QLBM_FP32, "fp16dev": QLBM_FP16_DEV, "df64": QLBM_DF64,
              "fp64df": QLBM_FP64_DF}

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError("libqlbm.so is not built (%s); run __graft_entry__.build() first" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_create = _sig("qlbm_create", _i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_i64), _d, _d, _d, _i, _vp])
_destroy = _sig("qlbm_destroy", None, [_vp])
_last_error = _sig("qlbm_last_error", ctypes.c_char_p, [_vp])
_info = _sig("qlbm_info", _i, [_vp, _vp, _i])
_init_eq = _sig("qlbm_init_equilibrium", _i, [_vp, _vp, _vp, _vp, _i])
_step = _sig("qlbm_step", _i, [_vp, _i64])
_time = _sig("qlbm_time", _i64, [_vp])
_sync = _sig("qlbm_sync", _i, [_vp])
_moments = _sig("qlbm_moments", _i, [_vp, _vp, _vp, _vp, _i])
_conserved = _sig("qlbm_conserved", _i, [_vp, _vp])
_get_state = _sig("qlbm_get_state", _i, [_vp, _vp, _i])
_set_state = _sig("qlbm_set_state", _i, [_vp, _vp, _i])
_step_adjoint = _sig("qlbm_step_adjoint", _i, [_vp, _vp, _vp, ctypes.POINTER(_d), _i])
_rollout = _sig("qlbm_rollout", _i, [_vp, _i64, _i64])
_rollout_adjoint = _sig("qlbm_rollout_adjoint", _i, [_vp, _vp, _vp, ctypes.POINTER(_d), _i])
_rollout_interval = _sig("qlbm_rollout_interval", _i64, [_vp])
_rollout_id = _sig("qlbm_rollout_id", _i64, [_vp])
_init_adjoint = _sig("qlbm_init_equilibrium_adjoint", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i])
_fd_params = _sig("qlbm_fd_params", _i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_i64), _i])
_fd_params_adjoint = _sig("qlbm_fd_params_adjoint", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _i])
_step_fd_output = _sig("qlbm_step_fd_output", _i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_i64), _i])
_init_fd = _sig("qlbm_init_fd_params", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _i])
_set_field = _sig("qlbm_set_magnetic_field", _i, [_vp, _d, ctypes.POINTER(_d)])
_set_field_array = _sig("qlbm_set_magnetic_field_array", _i, [_vp, _d, _vp, _i])
_set_eq_path = _sig("qlbm_set_equilibrium_path", _i, [_vp, _i])
_conserved_static = _sig("qlbm_conserved_static", _i, [_i, ctypes.POINTER(_i64), _d, _vp, _vp, _vp])
_negative_eq = _sig("qlbm_negative_eq_count", _i, [_vp, ctypes.POINTER(_i64), _vp, _i])
_checkpoint_bytes = _sig("qlbm_checkpoint_bytes", _i64, [_vp])
_save_checkpoint = _sig("qlbm_save_checkpoint", _i, [_vp, _vp, _i])
_load_checkpoint = _sig("qlbm_load_checkpoint", _i, [_vp, _vp, _i])
_fourier_field = _sig("qlbm_fourier_field", _i, [ctypes.POINTER(_i64), _i, _vp, _vp, _vp, _d, _d, _vp, _vp])

QLBM_FOURIER_MAX_MODES = 512
QLBM_FOURIER_MAX_K = 64
QLBM_STATIC_SCRATCH_BLOCKS = 1024
QLBM_STATIC_MAX_SITES = 2147483647


class QLBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("qlbm error %d: %s" % (code, msg))
        self.code = code


def _check(rc, h=None):
    if rc != QLBM_OK:
        msg = _last_error(h)
        raise QLBMError(rc, msg.decode() if msg else "")
    return rc


# Geometry of every live handle created through this binding: handle ->
# (d, b, N, CUDA device ordinal current at creation).  The wrappers check
# each array's size and device against it before the C call, so that a short
# array or a tensor on another GPU is refused here instead of being read or
# written out of bounds by the library.
_handles = {}


def _geom(h):
    g = _handles.get(h)
    if g is None:
        raise ValueError("unknown or destroyed qlbm handle")
    return g


def _ptr(a, n=None, dev=None, dtype=np.float64):
    """(pointer, ptr_kind) of a numpy array or CUDA tensor; None -> NULL.
    n: the least number of elements the call reads or writes; dev: the CUDA
    device ordinal a tensor must live on."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous %s" % np.dtype(dtype).name)
        if n is not None and a.size < n:
            raise ValueError("array of %d elements where %d are needed" % (a.size, n))
        return a.ctypes.data, QLBM_HOST
    # torch tensor
    if not getattr(a, "is_cuda", False):
        raise TypeError("expected a numpy array or a CUDA tensor")
    import torch
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    if a.dtype != tdt or not a.is_contiguous():
        raise TypeError("device tensors must be contiguous %s" % str(tdt))
    if n is not None and a.numel() < n:
        raise ValueError("tensor of %d elements where %d are needed" % (a.numel(), n))
    if dev is not None and a.device.index != dev:
        raise ValueError("tensor on cuda:%s, the handle lives on cuda:%d" % (a.device.index, dev))
    return a.data_ptr(), QLBM_DEVICE


def _ptr32(a, n=None, dev=None):
    """(pointer, ptr_kind) of a float32 numpy array or CUDA tensor."""
    return _ptr(a, n, dev, np.float32)


def _kind(*ptrs):
    kinds = {k for p, k in ptrs if p is not None}
    if not kinds:
        raise TypeError("at least one array argument is required")
    if len(kinds) != 1:
        raise TypeError("all array arguments must live on the same side (host or device)")
    return kinds.pop()


def qlbm_create(lattice, dims, tau, beta0, dt=1.0, precision=QLBM_FP64, stream=None):
    """Returns a handle (int); stream is a cudaStream_t value (int) or None."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    d = (ctypes.c_int64 * 3)(*[int(v) for v in (list(dims) + [1] * (3 - len(dims)))])
    h = _vp()
    _check(_create(ctypes.byref(h), int(lattice), d, float(tau), float(beta0), float(dt),
                   int(precision), _vp(stream) if stream else None))
    import torch
    dd = int(lattice)
    _handles[h.value] = (dd, 9 if dd == 2 else 19, d[0] * d[1] * d[2], torch.cuda.current_device())
    return h.value


def qlbm_destroy(h):
    _handles.pop(h, None)
    _destroy(h)


def qlbm_last_error(h=None):
    m = _last_error(h)
    return m.decode() if m else ""


def qlbm_info(h):
    out = np.zeros(16)
    _check(_info(h, out.ctypes.data, 16), h)
    keys = ["d", "b", "xi", "a", "w_rest", "w_axis", "w_diag", "c", "m", "alpha3", "alpha4",
            "alpha5", "tau", "beta0", "dt", "precision"]
    return dict(zip(keys, out.tolist()))


def qlbm_init_equilibrium(h, rho4, u, eps=None):
    d, b, N, dev = _geom(h)
    p = [_ptr(rho4, 4 * N, dev), _ptr(u, d * N, dev), _ptr(eps, N, dev)]
    _check(_init_eq(h, p[0][0], p[1][0], p[2][0], _kind(*p)), h)


def qlbm_step(h, nsteps):
    _check(_step(h, int(nsteps)), h)


def qlbm_time(h):
    return _time(h)


def qlbm_sync(h):
    _check(_sync(h), h)


def qlbm_moments(h, rho4=None, u=None, eps=None):
    d, b, N, dev = _geom(h)
    p = [_ptr(rho4, 4 * N, dev), _ptr(u, d * N, dev), _ptr(eps, N, dev)]
    _check(_moments(h, p[0][0], p[1][0], p[2][0], _kind(*p)), h)


def qlbm_conserved(h):
    out = np.zeros(8)
    _check(_conserved(h, out.ctypes.data), h)
    return out


def qlbm_get_state(h, buf):
    d, b, N, dev = _geom(h)
    p, k = _ptr(buf, b * 4 * N, dev)
    _check(_get_state(h, p, k), h)
    return buf


def qlbm_set_state(h, buf):
    d, b, N, dev = _geom(h)
    p, k = _ptr(buf, b * 4 * N, dev)
    _check(_set_state(h, p, k), h)


def qlbm_checkpoint_bytes(h):
    _geom(h)
    return _checkpoint_bytes(h)


def _raw(buf, nbytes, dev):
    """(pointer, ptr_kind) of a byte buffer: a numpy array or CUDA tensor of
    any dtype holding at least nbytes."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"] or buf.nbytes < nbytes:
            raise ValueError("checkpoint buffer must be C-contiguous with %d bytes" % nbytes)
        return buf.ctypes.data, QLBM_HOST
    if not getattr(buf, "is_cuda", False) or not buf.is_contiguous():
        raise TypeError("expected a numpy array or a contiguous CUDA tensor")
    if buf.numel() * buf.element_size() < nbytes or buf.device.index != dev:
        raise ValueError("checkpoint tensor too small or on another device")
    return buf.data_ptr(), QLBM_DEVICE


def qlbm_save_checkpoint(h, buf):
    """Bit-exact image of the populations (see qlbm_checkpoint_bytes)."""
    d, b, N, dev = _geom(h)
    p, k = _raw(buf, qlbm_checkpoint_bytes(h), dev)
    _check(_save_checkpoint(h, p, k), h)
    return buf


def qlbm_load_checkpoint(h, buf):
    d, b, N, dev = _geom(h)
    p, k = _raw(buf, qlbm_checkpoint_bytes(h), dev)
    _check(_load_checkpoint(h, p, k), h)


def qlbm_step_adjoint(h, lam_next, lam):
    """One reverse step at the current state; fills lam, returns dJ/dtau part."""
    d, b, N, dev = _geom(h)
    p = [_ptr(lam_next, b * 4 * N, dev), _ptr(lam, b * 4 * N, dev)]
    g = _d(0.0)
    _check(_step_adjoint(h, p[0][0], p[1][0], ctypes.byref(g), _kind(*p)), h)
    return g.value


def qlbm_rollout(h, nsteps, interval=0):
    _check(_rollout(h, int(nsteps), int(interval)), h)


def qlbm_rollout_interval(h):
    return _rollout_interval(h)


def qlbm_rollout_id(h):
    return _rollout_id(h)


def qlbm_rollout_adjoint(h, lam_T, lam_0):
    """Reverse sweep over the last rollout; fills lam_0, returns dJ/dtau."""
    d, b, N, dev = _geom(h)
    p = [_ptr(lam_T, b * 4 * N, dev), _ptr(lam_0, b * 4 * N, dev)]
    g = _d(0.0)
    _check(_rollout_adjoint(h, p[0][0], p[1][0], ctypes.byref(g), _kind(*p)), h)
    return g.value


def qlbm_init_equilibrium_adjoint(h, rho4, u, eps, lam0, g_rho4=None, g_u=None, g_eps=None):
    d, b, N, dev = _geom(h)
    p = [_ptr(rho4, 4 * N, dev), _ptr(u, d * N, dev), _ptr(eps, N, dev), _ptr(lam0, b * 4 * N, dev),
         _ptr(g_rho4, 4 * N, dev), _ptr(g_u, d * N, dev), _ptr(g_eps, N, dev)]
    _check(_init_adjoint(h, *[x[0] for x in p], _kind(*p)), h)


def qlbm_fd_params(h, beta=None, mu_up=None, mu_dn=None, axis=None):
    """Per-site Fermi-Dirac parameters into the given arrays; returns the
    number of sites without a solution."""
    d, b, N, dev = _geom(h)
    p = [_ptr(beta, N, dev), _ptr(mu_up, N, dev), _ptr(mu_dn, N, dev), _ptr(axis, 3 * N, dev)]
    nf = _i64(0)
    _check(_fd_params(h, *[x[0] for x in p], ctypes.byref(nf), _kind(*p)), h)
    return nf.value


def qlbm_step_fd_output(h, beta, mu_up, mu_dn, axis, count=True):
    """One step that also writes the float32 FD parameters of the state it
    started from; returns the number of unresolved sites (None if not
    counted, which keeps device calls asynchronous)."""
    d, b, N, dev = _geom(h)
    p = [_ptr32(beta, N, dev), _ptr32(mu_up, N, dev), _ptr32(mu_dn, N, dev), _ptr32(axis, 3 * N, dev)]
    nf = _i64(0)
    _check(_step_fd_output(h, *[x[0] for x in p], ctypes.byref(nf) if count else None, _kind(*p)), h)
    return nf.value if count else None


def qlbm_fd_params_adjoint(h, lam, g_beta=None, g_mu_up=None, g_mu_dn=None, g_axis=None):
    """Cotangent of the current state (into lam) from those of the FD parameters."""
    d, b, N, dev = _geom(h)
    p = [_ptr(g_beta, N, dev), _ptr(g_mu_up, N, dev), _ptr(g_mu_dn, N, dev), _ptr(g_axis, 3 * N, dev),
         _ptr(lam, b * 4 * N, dev)]
    _check(_fd_params_adjoint(h, *[x[0] for x in p], _kind(*p)), h)


def qlbm_init_fd_params(h, beta, mu_up, mu_dn, axis, u):
    d, b, N, dev = _geom(h)
    p = [_ptr(beta, N, dev), _ptr(mu_up, N, dev), _ptr(mu_dn, N, dev), _ptr(axis, 3 * N, dev),
         _ptr(u, d * N, dev)]
    _check(_init_fd(h, *[x[0] for x in p], _kind(*p)), h)


def qlbm_negative_eq_count(h, mask=None):
    """Number of (site, direction) pairs whose discrete equilibrium, formed
    from the current state, has a negative eigenvalue; mask (optional:
    uint32 numpy array or int32 CUDA tensor of N) receives the per-site bit
    masks of those directions."""
    d, b, N, dev = _geom(h)
    c = _i64(0)
    if mask is None:
        _check(_negative_eq(h, ctypes.byref(c), None, QLBM_HOST), h)
        return c.value
    if isinstance(mask, np.ndarray):
        if mask.dtype != np.uint32 or not mask.flags["C_CONTIGUOUS"] or mask.size < N:
            raise TypeError("mask must be a C-contiguous uint32 array of N")
        _check(_negative_eq(h, ctypes.byref(c), mask.ctypes.data, QLBM_HOST), h)
        return c.value
    import torch
    if not getattr(mask, "is_cuda", False) or mask.dtype != torch.int32 or not mask.is_contiguous():
        raise TypeError("device masks must be contiguous int32 CUDA tensors")
    if mask.numel() < N or mask.device.index != dev:
        raise ValueError("mask too short or on another device")
    _check(_negative_eq(h, ctypes.byref(c), mask.data_ptr(), QLBM_DEVICE), h)
    return c.value


def qlbm_set_magnetic_field(h, mu, B):
    b = (ctypes.c_double * 3)(*[float(v) for v in B])
    _check(_set_field(h, float(mu), b), h)


def qlbm_set_magnetic_field_array(h, mu, B):
    """Per-site magnetic field B [3][N] (numpy float64 or CUDA float64 tensor)."""
    d, b, N, dev = _geom(h)
    p, k = _ptr(B, 3 * N, dev)
    _check(_set_field_array(h, float(mu), p, k), h)


def qlbm_set_equilibrium_path(h, path):
    _check(_set_eq_path(h, int(path)), h)


def qlbm_conserved_static(lattice, dims, beta0, state, out, stream=None):
    """The eight global averages of qlbm_conserved for a caller-owned device
    state (canonical layout [b][4][N], float64) into a caller-owned device
    buffer of 8 float64, without allocating device memory.

    For callers that cannot allocate at the point of the call, e.g. code
    running under another component's memory manager that owns the device's
    memory, or latency-critical loops that cannot afford cudaMalloc/cudaFree.
    The scratch is a fixed array inside the library; calls that overlap on
    the GPU race on it.  Asynchronous on ``stream`` (a cudaStream_t value).
    """
    d = (ctypes.c_int64 * 3)(*[int(v) for v in (list(dims) + [1] * (3 - len(dims)))])
    import torch
    dev = torch.cuda.current_device()   # the library reduces on the current device
    # buffer sizes are checked for dims the library accepts; it rejects the rest itself
    valid = min(d[0], d[1], d[2]) >= 1 and (int(lattice) != 2 or d[2] == 1) and \
        d[0] * d[1] * d[2] <= QLBM_STATIC_MAX_SITES
    nsites = d[0] * d[1] * d[2] if valid else 0
    sp, sk = _ptr(state, (9 if int(lattice) == 2 else 19) * 4 * nsites, dev)
    op, ok = _ptr(out, 8, dev)
    if sk != QLBM_DEVICE or ok != QLBM_DEVICE:
        raise TypeError("state and out must be CUDA tensors")
    _check(_conserved_static(int(lattice), d, float(beta0), sp, op, _vp(stream) if stream else None))


def qlbm_fourier_field(dims, k, A, B, scale, offset, out, stream=None):
    """out (CUDA float64 tensor of nx*ny*nz) = offset + scale * sum_m
    A_m cos(2 pi k_m.x/L) + B_m sin(2 pi k_m.x/L) at every site, evaluated by
    the library on the device.  k: int [nmodes][3]; A, B: float64 [nmodes]
    (host arrays).  Asynchronous on ``stream``."""
    d = (ctypes.c_int64 * 3)(*[int(v) for v in (list(dims) + [1] * (3 - len(dims)))])
    kk = np.ascontiguousarray(np.asarray(k).reshape(-1, 3), dtype=np.int32)
    a = np.ascontiguousarray(A, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(B, dtype=np.float64).reshape(-1)
    if not (len(kk) == len(a) == len(b)):
        raise ValueError("k, A and B must describe the same number of modes")
    import torch
    op, ok = _ptr(out, d[0] * d[1] * d[2], torch.cuda.current_device())
    if ok != QLBM_DEVICE:
        raise TypeError("out must be a CUDA tensor")
    _check(_fourier_field(d, len(kk), kk.ctypes.data, a.ctypes.data, b.ctypes.data, float(scale),
                          float(offset), op, _vp(stream) if stream else None))


def fields_on_device(spec, dims, stream=None):
    """Device tensors dict(rho4 [4][N], u [d][N], eps=None) of a Fourier-mode
    workload description (``fields.mode_spec``), each row evaluated by
    qlbm_fourier_field."""
    import torch
    dims = tuple(int(v) for v in (list(dims) + [1] * (3 - len(dims))))
    N = dims[0] * dims[1] * dims[2]
    out = {}
    for key in ("rho4", "u"):
        rows = spec[key]
        t = torch.empty((len(rows), N), dtype=torch.float64, device="cuda")
        for c, (f, scale, offset) in enumerate(rows):
            qlbm_fourier_field(dims, f.k.astype(np.int32), f.A, f.B, scale, offset, t[c], stream)
        out[key] = t
    out["eps"] = None
    return out


class Lattice:
    """Owning wrapper of a handle with numpy conveniences (host round trips)."""

    def __init__(self, lattice, dims, tau, beta0=1.0, dt=1.0, precision="fp64", stream=None):
        if lattice in ("D2Q9", "d2q9"):
            lattice = QLBM_D2Q9
        elif lattice in ("D3Q19", "d3q19"):
            lattice = QLBM_D3Q19
        self.d = int(lattice)
        self.b = 9 if self.d == 2 else 19
        self.dims = tuple(int(v) for v in (list(dims) + [1] * (3 - len(dims))))
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.tau, self.beta0, self.dt = float(tau), float(beta0), float(dt)
        self.h = qlbm_create(lattice, self.dims, tau, beta0, dt, precision, stream)

    def close(self):
        if self.h:
            qlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        return qlbm_info(self.h)

    def init_equilibrium(self, rho4, u, eps=None):
        qlbm_init_equilibrium(self.h, rho4, u, eps)

    def step(self, n=1):
        qlbm_step(self.h, n)

    def time(self):
        return qlbm_time(self.h)

    def sync(self):
        qlbm_sync(self.h)

    def moments(self):
        rho4 = np.zeros((4, self.N))
        u = np.zeros((self.d, self.N))
        eps = np.zeros(self.N)
        qlbm_moments(self.h, rho4, u, eps)
        return rho4, u, eps

    def conserved(self):
        return qlbm_conserved(self.h)

    def get_state(self):
        buf = np.zeros((self.b, 4, self.N))
        qlbm_get_state(self.h, buf)
        return buf

    def set_state(self, state):
        qlbm_set_state(self.h, np.ascontiguousarray(state, dtype=np.float64))

    def step_adjoint(self, lam_next):
        lam = np.zeros((self.b, 4, self.N))
        g = qlbm_step_adjoint(self.h, np.ascontiguousarray(lam_next, dtype=np.float64), lam)
        return lam, g

    def fd_params(self):
        beta = np.zeros(self.N)
        mu_up = np.zeros(self.N)
        mu_dn = np.zeros(self.N)
        axis = np.zeros((3, self.N))
        nfail = qlbm_fd_params(self.h, beta, mu_up, mu_dn, axis)
        return beta, mu_up, mu_dn, axis, nfail

    def step_fd_output(self):
        """One step; returns the float32 FD parameters (beta, mu_up, mu_dn,
        axis, nfail) of the state it started from."""
        beta = np.zeros(self.N, np.float32)
        mu_up = np.zeros(self.N, np.float32)
        mu_dn = np.zeros(self.N, np.float32)
        axis = np.zeros((3, self.N), np.float32)
        nfail = qlbm_step_fd_output(self.h, beta, mu_up, mu_dn, axis)
        return beta, mu_up, mu_dn, axis, nfail

    def save_checkpoint(self):
        """Bit-exact checkpoint image (numpy uint8)."""
        buf = np.zeros(qlbm_checkpoint_bytes(self.h), np.uint8)
        return qlbm_save_checkpoint(self.h, buf)

    def load_checkpoint(self, buf):
        qlbm_load_checkpoint(self.h, np.ascontiguousarray(buf))

    def negative_eq(self):
        """(count, mask uint32 [N]) of the negative-eigenvalue diagnostic."""
        mask = np.zeros(self.N, np.uint32)
        return qlbm_negative_eq_count(self.h, mask), mask

    def set_magnetic_field(self, mu, B):
        qlbm_set_magnetic_field(self.h, mu, B)

    def set_magnetic_field_array(self, mu, B):
        qlbm_set_magnetic_field_array(self.h, mu, np.ascontiguousarray(B, dtype=np.float64)
                                      if isinstance(B, np.ndarray) else B)

    def set_equilibrium_path(self, path):
        qlbm_set_equilibrium_path(self.h, path)

    def rollout(self, nsteps, interval=0):
        qlbm_rollout(self.h, nsteps, interval)

    def rollout_adjoint(self, lam_T):
        lam = np.zeros((self.b, 4, self.N))
        g = qlbm_rollout_adjoint(self.h, np.ascontiguousarray(lam_T, dtype=np.float64), lam)
        return lam, g
