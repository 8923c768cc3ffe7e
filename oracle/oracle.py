"""ctypes wrapper around the C oracle (``bzoracle.c``).

TEST INFRASTRUCTURE ONLY (see ``bzoracle.h``).  Every array crosses the
boundary as contiguous float64 numpy memory; complex mode arrays are numpy
complex128 of shape ``(M,)*d`` with mode index ``k_i + h`` along axis i.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "bzoracle.c")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


class _Grid(ctypes.Structure):
    _fields_ = [("dim", _i), ("N", _i), ("h", _i), ("M", _i), ("nv", _i64), ("nm", _i64),
                ("L", _d), ("dv", _d), ("s", _d)]


class _Kernel(ctypes.Structure):
    _fields_ = [("g", _Grid), ("gamma", _d), ("b0", _d), ("nq", _i), ("arows", _i),
                ("amax2", _i), ("F", ctypes.POINTER(_d)), ("ndirs", _i),
                ("alpha", ctypes.POINTER(_d)), ("alphap", ctypes.POINTER(_d)), ("penalty", _d)]


def build(force=False):
    """Compile liboracle.so next to its source (plain gcc, OpenMP, no -march)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bzoracle.h"))):
            return _SO
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    P = ctypes.POINTER
    lib.orc_grid_init.argtypes = [P(_Grid), _i, _i, _d]
    lib.orc_gauss_legendre.argtypes = [_i, _p, _p]
    lib.orc_radial_Bhat.argtypes = [_i, _d, _d, _i, _d, _d]
    lib.orc_radial_Bhat.restype = _d
    lib.orc_kernel_init.argtypes = [P(_Kernel), P(_Grid), _d, _d, _i]
    lib.orc_kernel_free.argtypes = [P(_Kernel)]
    lib.orc_fast_kernel_init.argtypes = [P(_Kernel), P(_Grid), _d, _i]
    lib.orc_Bhat.argtypes = [P(_Kernel), _p, _p]
    lib.orc_Bhat.restype = _d
    lib.orc_beta.argtypes = [P(_Kernel), _p, _p]
    lib.orc_beta.restype = _d
    lib.orc_beta_table.argtypes = [P(_Kernel), _p]
    lib.orc_beta_pairs.argtypes = [P(_Kernel), _i64, _p, _p, _p]
    lib.orc_dft_forward.argtypes = [P(_Grid), _p, _p]
    lib.orc_mode_sum.argtypes = [P(_Kernel), _p, _p]
    lib.orc_dft_inverse.argtypes = [P(_Grid), _p, _d, _p]
    lib.orc_conserve.argtypes = [P(_Grid), _p]
    lib.orc_collide.argtypes = [P(_Kernel), _p, _p, _i64, _i]
    lib.orc_moments.argtypes = [P(_Grid), _p, _p]
    lib.orc_maxwellian.argtypes = [P(_Grid), _p, _p]
    lib.orc_imex_step.argtypes = [P(_Kernel), _i, _i, _d, _d, _p, _p, _p, _i64, _i]
    lib.orc_imex_step_stages.argtypes = [P(_Kernel), _i, _i, _d, _d, _p, _p, _p, _i64, _i,
                                         _p, _p, _p]
    lib.orc_num_threads.restype = _i
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads():
    return load().orc_num_threads()


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    load().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def radial_bhat(dim, gamma, b0, nq, a, b):
    return load().orc_radial_Bhat(dim, gamma, b0, nq, float(a), float(b))


SCHEMES = {"ars222": 0, "bpr343": 1, "euler": 2}
MODELS = {"boltzmann": 0, "bgk": 1}
STAGES = {"ars222": 3, "bpr343": 5, "euler": 2}


class Kernel:
    """Velocity grid plus kernel modes B(|q|) = b0 |q|^gamma (b0 <= 0: default).

    ndirs > 0 selects the fast spectral (Carleman) form of the kernel modes
    with that many collision directions (2-D, gamma = 0 only); see
    ``FastKernel``."""

    def __init__(self, dim, N, L, gamma, b0=0.0, nq=0, ndirs=0):
        lib = load()
        self._g = _Grid()
        if lib.orc_grid_init(ctypes.byref(self._g), dim, N, float(L)) != 0:
            raise ValueError("bad grid (dim=%r N=%r L=%r)" % (dim, N, L))
        self._k = _Kernel()
        if ndirs:
            if gamma != 0.0 or dim != 2:
                raise ValueError("the fast (Carleman) form is built for 2-D Maxwell molecules")
            if lib.orc_fast_kernel_init(ctypes.byref(self._k), ctypes.byref(self._g), float(b0),
                                        int(ndirs)) != 0:
                raise ValueError("bad fast-method parameters (ndirs=%r)" % (ndirs,))
        elif lib.orc_kernel_init(ctypes.byref(self._k), ctypes.byref(self._g), float(gamma),
                                 float(b0), int(nq)) != 0:
            raise MemoryError("oracle kernel table allocation failed")
        self.ndirs = int(ndirs)
        g = self._g
        self.dim, self.N, self.h, self.M = g.dim, g.N, g.h, g.M
        self.nv, self.nm = g.nv, g.nm
        self.L, self.dv, self.s = g.L, g.dv, g.s
        self.gamma, self.b0, self.nq = self._k.gamma, self._k.b0, self._k.nq

    def __del__(self):
        try:
            load().orc_kernel_free(ctypes.byref(self._k))
        except Exception:
            pass

    # grid helpers -------------------------------------------------------
    def velocities(self):
        """1-D velocity nodes v_j = -L + j dv."""
        return -self.L + self.dv * np.arange(self.N)

    def modes(self):
        return np.arange(-self.h, self.h + 1)

    # kernel modes -------------------------------------------------------
    def bhat(self, l, m):
        l = np.ascontiguousarray(l, dtype=np.int32)
        m = np.ascontiguousarray(m, dtype=np.int32)
        return load().orc_Bhat(ctypes.byref(self._k), _ptr(l), _ptr(m))

    def beta(self, l, m):
        l = np.ascontiguousarray(l, dtype=np.int32)
        m = np.ascontiguousarray(m, dtype=np.int32)
        return load().orc_beta(ctypes.byref(self._k), _ptr(l), _ptr(m))

    def beta_table(self):
        t = np.zeros((self.nm, self.nm))
        load().orc_beta_table(ctypes.byref(self._k), _ptr(t))
        return t

    def beta_pairs(self, li, mi):
        """beta-hat(l, m) for arrays of flat mode indices (row-major, k_i + h)."""
        li = np.ascontiguousarray(li, dtype=np.int64)
        mi = np.ascontiguousarray(mi, dtype=np.int64)
        out = np.zeros(li.shape[0])
        load().orc_beta_pairs(ctypes.byref(self._k), li.shape[0], _ptr(li), _ptr(mi), _ptr(out))
        return out

    # transforms ---------------------------------------------------------
    def dft_forward(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.nv)
        out = np.zeros(2 * self.nm)
        load().orc_dft_forward(ctypes.byref(self._g), _ptr(f), _ptr(out))
        return (out[0::2] + 1j * out[1::2]).reshape((self.M,) * self.dim)

    def mode_sum(self, fhat):
        fh = np.ascontiguousarray(np.asarray(fhat, dtype=np.complex128).reshape(self.nm))
        inter = np.zeros(2 * self.nm)
        inter[0::2] = fh.real
        inter[1::2] = fh.imag
        out = np.zeros(2 * self.nm)
        load().orc_mode_sum(ctypes.byref(self._k), _ptr(inter), _ptr(out))
        return (out[0::2] + 1j * out[1::2]).reshape((self.M,) * self.dim)

    def dft_inverse(self, qhat, scale=None):
        if scale is None:
            scale = self.s ** (self.dim + self.gamma)
        qh = np.asarray(qhat, dtype=np.complex128).reshape(self.nm)
        inter = np.zeros(2 * self.nm)
        inter[0::2] = qh.real
        inter[1::2] = qh.imag
        out = np.zeros(self.nv)
        load().orc_dft_inverse(ctypes.byref(self._g), _ptr(inter), float(scale), _ptr(out))
        return out.reshape((self.N,) * self.dim)

    def conserve(self, Q):
        q = np.array(Q, dtype=np.float64).reshape(self.nv).copy()
        load().orc_conserve(ctypes.byref(self._g), _ptr(q))
        return q.reshape(np.shape(Q))

    # whole operator -----------------------------------------------------
    def collide(self, f, conserve=False):
        """Q(f) for f of shape (ncells, N^d) (or (N,)*d for one cell)."""
        f = np.asarray(f, dtype=np.float64)
        shape = f.shape
        f2 = np.ascontiguousarray(f.reshape(-1, self.nv))
        Q = np.zeros_like(f2)
        if load().orc_collide(ctypes.byref(self._k), _ptr(f2), _ptr(Q), f2.shape[0],
                              int(bool(conserve))) != 0:
            raise MemoryError("oracle collide failed")
        return Q.reshape(shape)

    def moments(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.nv)
        U = np.zeros(self.dim + 2)
        load().orc_moments(ctypes.byref(self._g), _ptr(f), _ptr(U))
        return U

    def maxwellian(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(self.nv)
        load().orc_maxwellian(ctypes.byref(self._g), _ptr(U), _ptr(out))
        return out.reshape((self.N,) * self.dim)

    def imex_step(self, f_n, dt, eps, scheme="ars222", model="boltzmann", Lres=None,
                  conserve=False, stages=False, penalty=1.0):
        """One penalised IMEX step.  f_n: (ncells, N^d).  Lres: (stages, ncells, N^d)
        or None.  With stages=True also returns (F, G, P) per stage.  penalty:
        c of the Boltzmann model's penalty rate nu = c rho."""
        self._k.penalty = float(penalty)
        f = np.ascontiguousarray(np.asarray(f_n, dtype=np.float64).reshape(-1, self.nv))
        nc = f.shape[0]
        ns = STAGES[scheme]
        out = np.zeros_like(f)
        Lp = None
        if Lres is not None:
            Lres = np.ascontiguousarray(np.asarray(Lres, dtype=np.float64).reshape(ns, nc, self.nv))
            Lp = _ptr(Lres)
        lib = load()
        if stages:
            F = np.zeros((ns, nc, self.nv))
            G = np.zeros_like(F)
            P = np.zeros_like(F)
            rc = lib.orc_imex_step_stages(ctypes.byref(self._k), SCHEMES[scheme], MODELS[model],
                                          float(dt), float(eps), _ptr(f), Lp, _ptr(out), nc,
                                          int(bool(conserve)), _ptr(F), _ptr(G), _ptr(P))
            if rc != 0:
                raise RuntimeError("oracle imex failed")
            return out, F, G, P
        rc = lib.orc_imex_step(ctypes.byref(self._k), SCHEMES[scheme], MODELS[model], float(dt),
                               float(eps), _ptr(f), Lp, _ptr(out), nc, int(bool(conserve)))
        if rc != 0:
            raise RuntimeError("oracle imex failed")
        return out


def FastKernel(N, L, ndirs, b0=0.0):
    """Kernel modes of the fast spectral method (Sec. 3.3, eq. ode / eq. FKM) for
    2-D Maxwell molecules with ``ndirs`` collision directions."""
    return Kernel(2, N, L, 0.0, b0=b0, ndirs=ndirs)
