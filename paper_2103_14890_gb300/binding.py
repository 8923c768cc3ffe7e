"""Thin ctypes binding of libbzcoll.so (C ABI in include/bzcoll.h).

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (contiguous, float64 for
``"fp64"``, float32 for ``"fp32"``); streams default to torch's
current stream.  There is no CPU fallback: if the library is missing or
cannot be loaded, every call raises.
"""
import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "libbzcoll.so")
HEADER = os.path.join(ROOT, "include", "bzcoll.h")

OK, EINVAL, ENOMEM, ECUDA, ENOTSUP, ETIMEOUT, ENONFINITE = 0, -1, -2, -3, -4, -5, -6
PRECISION = {"fp64": 0, "fp32": 1, "fp32x2": 2}
CONSERVE, CHECK_INPUT = 1, 2
SCHEME = {"ars222": 0, "bpr343": 1, "euler": 2}
STAGES = {"ars222": 3, "bpr343": 5, "euler": 2}
MODEL = {"boltzmann": 0, "bgk": 1}

_lock = threading.Lock()
_lib = None


class BzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bzcoll error %d: %s" % (code, msg))
        self.code = code


def header_functions():
    """Names of the functions declared in include/bzcoll.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"defined"})


def load(path=None):
    """Load the library (raises if it is absent: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise BzError(ECUDA, "libbzcoll.so not built (%s); run __graft_entry__.build()" % p)
        lib = ctypes.CDLL(p)
        c_i, c_d, c_p, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "init_velocity_grid": ([c_i, c_i, c_d, pp], c_i),
            "build_kernel_modes": ([c_p, c_d, c_d, c_i, pp], c_i),
            "collide_batch": ([c_p, c_i, c_i, c_p, c_p, c_i64, c_p], c_i),
            "imex_stage_local": ([c_p, c_i, c_i, c_i, c_d, c_d, c_p, c_p, c_p, c_p, c_p, c_i64, c_i, c_i, c_p], c_i),
            "imex_step": ([c_p, c_i, c_i, c_d, c_d, c_p, c_p, c_p, c_i64, c_i, c_i, c_p], c_i),
            "bz_check": ([c_p], c_i),
            "bz_last_error": ([], ctypes.c_char_p),
            "bz_modes_info": ([c_p, ctypes.POINTER(c_i64)], c_i),
            "bz_modes_beta": ([c_p, c_p], c_i),
            "bz_modes_set_penalty": ([c_p, c_d], c_i),
            "bz_grid_destroy": ([c_p], None),
            "bz_modes_destroy": ([c_p], None),
            "bz_profile": ([c_i], c_i),
            "collide_batch_noalloc": ([c_p, c_i, c_i, c_p, c_p, c_i64, c_p], c_i),
            "collide_batch_host": ([c_p, c_i, c_i, c_p, c_p, c_i64, c_p], c_i),
            "group_collide": ([c_p, c_i, c_i, c_i, c_p], c_i),
            "bz_profile_read": ([c_p, c_i, c_p, c_p, c_i], c_i),
            "build_fast_modes": ([c_p, c_d, c_i, pp], c_i),
            "bz_fast_info": ([c_p, ctypes.POINTER(c_i64)], c_i),
            "build_fv_mesh": ([c_i, c_p, c_i64, c_p, c_p, c_i, pp], c_i),
            "build_fv_mesh_periodic": ([c_i, c_p, c_i64, c_p, c_p, c_i, c_d, c_d, pp], c_i),
            "transport_residual": ([c_p, c_p, c_i, c_p, c_p, c_p], c_i),
            "imex_step_fv": ([c_p, c_p, c_i, c_i, c_d, c_d, c_p, c_p, c_i, c_i, c_p], c_i),
            "bz_mesh_info": ([c_p, ctypes.POINTER(c_i64)], c_i),
            "bz_mesh_destroy": ([c_p], None),
            "fv_mesh_set_walls": ([c_p, c_i64, c_p, c_p], c_i),
            "bz_inject_alloc_failure": ([c_i64], c_i),
            "bz_alloc_stats": ([c_p, c_p], c_i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc):
    if rc != OK:
        raise BzError(rc, load().bz_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t, dtype, what):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return ctypes.c_void_p(t.data_ptr())


def _dtype(precision):
    import torch
    return torch.float64 if precision == "fp64" else torch.float32


class Grid:
    """Velocity grid (init_velocity_grid): d, N points per dimension, [-L, L]^d."""

    def __init__(self, dim, N, L):
        h = ctypes.c_void_p()
        _check(load().init_velocity_grid(int(dim), int(N), float(L), ctypes.byref(h)))
        self._h = h
        self.dim, self.N, self.L = dim, N, L
        self.nv = N ** dim

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.bz_grid_destroy(self._h)
            self._h = None


class Modes:
    """Kernel modes (build_kernel_modes) of B = b0 |q|^gamma on a grid."""

    def __init__(self, grid, gamma, b0=0.0, quad_nodes=0, _handle=None):
        h = ctypes.c_void_p()
        if _handle is None:
            _check(load().build_kernel_modes(grid._h, float(gamma), float(b0), int(quad_nodes), ctypes.byref(h)))
        else:
            h = _handle
        self._h = h
        self.grid = grid              # keep the grid alive
        self.gamma = gamma
        self.penalty = 1.0
        fi = (ctypes.c_int64 * 4)()
        _check(load().bz_fast_info(h, fi))
        self.method, self.ndirs, self.pad, self.fast_cells = list(fi)
        info = (ctypes.c_int64 * 8)()
        _check(load().bz_modes_info(h, info))
        self.dim, self.N, self.h, self.nv, self.nhalf, self.nq, self.pairs_sym, self.modesum_variant = list(info)
        self.fast32 = self.modesum_variant > 0   # register-blocked FP32 mode-sum kernel in use

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.bz_modes_destroy(self._h)
            self._h = None

    def set_penalty(self, c):
        """Penalty rate nu = c rho of the Boltzmann model in the IMEX stages
        (bz_modes_set_penalty)."""
        _check(load().bz_modes_set_penalty(self._h, float(c)))
        self.penalty = float(c)

    def beta_table(self):
        import numpy as np
        nm = (2 * self.h + 1) ** self.dim
        out = np.zeros((nm, nm))
        _check(load().bz_modes_beta(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out


class FastModes(Modes):
    """Kernel modes of the fast spectral (Carleman) form (build_fast_modes):
    2-D Maxwell molecules, ``ndirs`` collision directions.  Accepted by every
    call that takes a Modes object."""

    def __init__(self, grid, ndirs, b0=0.0):
        h = ctypes.c_void_p()
        _check(load().build_fast_modes(grid._h, float(b0), int(ndirs), ctypes.byref(h)))
        super().__init__(grid, 0.0, _handle=h)


class Mesh:
    """Finite-volume mesh of the transport step (build_fv_mesh): vertices xy
    (n_vtx, 2) and cells, either an (n_cells, k) integer array or a list of
    vertex lists; order 1 (first order), 2 (CWENO of degree 1) or 3 (CWENO
    of degree 2, two Gauss points per face); periodic
    (Lx, Ly) makes it periodic (build_fv_mesh_periodic, 0 for a direction
    without periodicity)."""

    def __init__(self, xy, cells, order=2, periodic=None):
        import numpy as np
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        cells = [list(map(int, c)) for c in cells]
        ptr = np.zeros(len(cells) + 1, dtype=np.int64)
        ptr[1:] = np.cumsum([len(c) for c in cells])
        vtx = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int64) for c in cells]))
        h = ctypes.c_void_p()
        args = (int(len(xy)), xy.ctypes.data_as(ctypes.c_void_p), int(len(cells)),
                ptr.ctypes.data_as(ctypes.c_void_p), vtx.ctypes.data_as(ctypes.c_void_p), int(order))
        if periodic is None:
            _check(load().build_fv_mesh(*args, ctypes.byref(h)))
        else:
            _check(load().build_fv_mesh_periodic(*args, float(periodic[0]), float(periodic[1]), ctypes.byref(h)))
        self._h = h
        info = (ctypes.c_int64 * 5)()
        _check(load().bz_mesh_info(h, info))
        self.n_cells, self.n_faces_interior, self.n_faces_boundary, self.max_faces, self.order = list(info)

    def set_walls(self, edges, params):
        """Walls with full accommodation on boundary edges (vertex pairs, shape
        (n, 2)); params (n, 3) = (theta_w, u_w1, u_w2) per edge; an empty list
        removes every wall."""
        import numpy as np
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 2))
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1, 3))
        if len(e) != len(p):
            raise ValueError("one parameter triple per edge")
        _check(load().fv_mesh_set_walls(self._h, int(len(e)), e.ctypes.data_as(ctypes.c_void_p),
                                        p.ctypes.data_as(ctypes.c_void_p)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.bz_mesh_destroy(self._h)
            self._h = None


def transport_residual(mesh, grid, f, L=None, precision="fp32", stream=None):
    """<L(f^w)>_x for f of shape (n_cells, N^2) on the device."""
    import torch
    dt = _dtype(precision)
    if L is None:
        L = torch.empty_like(f)
    if f.numel() != mesh.n_cells * grid.nv or L.numel() != f.numel():
        raise ValueError("f and L must have n_cells * N^2 elements")
    _check(load().transport_residual(mesh._h, grid._h, PRECISION[precision], _dptr(f, dt, "f"), _dptr(L, dt, "L"),
                                     _stream(stream)))
    return L


def imex_step_fv(modes, mesh, f_n, dt, eps, f_out=None, scheme="ars222", model="boltzmann", precision="fp32",
                 conserve=False, check_input=False, stream=None):
    """One IMEX step of the finite-volume scheme (transport + collisions) on the mesh."""
    import torch
    ty = _dtype(precision)
    if f_out is None:
        f_out = torch.empty_like(f_n)
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    _check(load().imex_step_fv(modes._h, mesh._h, SCHEME[scheme], MODEL[model], float(dt), float(eps),
                               _dptr(f_n, ty, "f_n"), _dptr(f_out, ty, "f_out"), PRECISION[precision], flags,
                               _stream(stream)))
    return f_out


def collide_batch(modes, f, Q=None, precision="fp32", conserve=False, check_input=False, stream=None):
    """Q(f) for f of shape (n_cells, N^d) on the device."""
    import torch
    dt = _dtype(precision)
    if Q is None:
        Q = torch.empty_like(f)
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    n = f.shape[0] if f.dim() > 1 else 1
    if f.numel() != n * modes.nv:
        raise ValueError("f must have n_cells * N^d elements")
    _check(load().collide_batch(modes._h, PRECISION[precision], flags, _dptr(f, dt, "f"), _dptr(Q, dt, "Q"),
                                n, _stream(stream)))
    return Q


def collide_batch_noalloc(modes, f, Q=None, precision="fp32", conserve=False, stream=None):
    """Q(f) through the allocation-free entry point (bounded batch, see the header)."""
    import torch
    dt = _dtype(precision)
    if Q is None:
        Q = torch.empty_like(f)
    n = f.shape[0] if f.dim() > 1 else 1
    if f.numel() != n * modes.nv:
        raise ValueError("f must have n_cells * N^d elements")
    _check(load().collide_batch_noalloc(modes._h, PRECISION[precision], CONSERVE if conserve else 0,
                                        _dptr(f, dt, "f"), _dptr(Q, dt, "Q"), n, _stream(stream)))
    return Q


def _hptr(a, dtype_name, what):
    """Host pointer of a contiguous CPU torch tensor or numpy array."""
    import numpy as np
    try:
        import torch
    except ImportError:        # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise TypeError("%s must be a host (CPU) tensor" % what)
        if str(a.dtype) != "torch." + dtype_name:
            raise TypeError("%s must be %s, got %s" % (what, dtype_name, a.dtype))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % what)
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype_name):
            raise TypeError("%s must be %s, got %s" % (what, dtype_name, a.dtype))
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be C-contiguous" % what)
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("%s must be a CPU torch tensor or a numpy array" % what)


def collide_batch_host(modes, f, Q=None, precision="fp32", conserve=False, check_input=False, stream=None):
    """Q(f) for HOST f of shape (n_cells, N^d) (CPU torch tensor, pinned for
    overlap, or numpy array); Q is returned in the same kind of container and
    is complete once the stream has completed."""
    import numpy as np
    name = "float64" if precision == "fp64" else "float32"
    if Q is None:
        Q = np.empty_like(f) if isinstance(f, np.ndarray) else f.new_empty(f.shape).pin_memory() \
            if f.is_pinned() else f.new_empty(f.shape)
    n = f.shape[0] if len(f.shape) > 1 else 1
    if int(np.prod(f.shape)) != n * modes.nv or int(np.prod(Q.shape)) != n * modes.nv:
        raise ValueError("f and Q must have n_cells * N^d elements")
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    _check(load().collide_batch_host(modes._h, PRECISION[precision], flags, _hptr(f, name, "f"),
                                     _hptr(Q, name, "Q"), n, _stream(stream)))
    return Q


class GroupItem(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_void_p), ("f", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("n_cells", ctypes.c_int64)]


def group_collide(entries, precision="fp32", conserve=False, check_input=False, stream=None):
    """entries: list of (modes, f, Q) with device tensors; one call for all."""
    dt = _dtype(precision)
    arr = (GroupItem * len(entries))()
    for i, (m, f, Q) in enumerate(entries):
        n = f.shape[0] if f.dim() > 1 else 1
        if f.numel() != n * m.nv or Q.numel() != f.numel():
            raise ValueError("item %d: f and Q must have n_cells * N^d elements" % i)
        arr[i].modes = m._h
        arr[i].f = _dptr(f, dt, "f")
        arr[i].Q = _dptr(Q, dt, "Q")
        arr[i].n_cells = n
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    _check(load().group_collide(ctypes.cast(arr, ctypes.c_void_p), len(entries), PRECISION[precision], flags,
                                _stream(stream)))


def imex_stage_local(modes, stage, f_n, F, G, P, dt, eps, scheme="ars222", model="boltzmann",
                     L_res=None, precision="fp32", conserve=False, check_input=False, stream=None):
    """Stage `stage` (1-based); F, G, P of shape (stages, n_cells, N^d)."""
    ty = _dtype(precision)
    n = f_n.shape[0]
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    _check(load().imex_stage_local(modes._h, SCHEME[scheme], int(stage), MODEL[model], float(dt), float(eps),
                                   _dptr(f_n, ty, "f_n"), _dptr(F, ty, "F"), _dptr(G, ty, "G"), _dptr(P, ty, "P"),
                                   _dptr(L_res, ty, "L_res"), n, PRECISION[precision], flags, _stream(stream)))


def imex_step(modes, f_n, dt, eps, f_out=None, scheme="ars222", model="boltzmann", L_res=None,
              precision="fp32", conserve=False, check_input=False, stream=None):
    """One IMEX step f_n -> f_out (shape (n_cells, N^d))."""
    import torch
    ty = _dtype(precision)
    if f_out is None:
        f_out = torch.empty_like(f_n)
    flags = (CONSERVE if conserve else 0) | (CHECK_INPUT if check_input else 0)
    _check(load().imex_step(modes._h, SCHEME[scheme], MODEL[model], float(dt), float(eps),
                            _dptr(f_n, ty, "f_n"), _dptr(f_out, ty, "f_out"), _dptr(L_res, ty, "L_res"),
                            f_n.shape[0], PRECISION[precision], flags, _stream(stream)))
    return f_out


def check(stream=None):
    """Synchronise and raise on a latched device-side error."""
    _check(load().bz_check(_stream(stream)))


def profile(enable):
    """Turn per-kernel CUDA-event timing inside the library on or off (clears it)."""
    _check(load().bz_profile(1 if enable else 0))


def inject_alloc_failure(after):
    """Test hook: the library's next `after` device allocations succeed and the
    one after them fails with BZ_ENOMEM (host side); None or < 0 turns it off."""
    _check(load().bz_inject_alloc_failure(-1 if after is None else int(after)))


def alloc_stats():
    """(device blocks the library holds outside its pools, bytes in use in its
    stream-ordered pools)."""
    live = ctypes.c_int64()
    used = ctypes.c_uint64()
    _check(load().bz_alloc_stats(ctypes.byref(live), ctypes.byref(used)))
    return int(live.value), int(used.value)


def profile_read(max_kernels=32):
    """{kernel name: (launches, total ms)} of the launches timed since profile(True)."""
    names = ctypes.create_string_buffer(64 * max_kernels)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_int64 * max_kernels)()
    n = load().bz_profile_read(names, 64 * max_kernels, ms, cnt, max_kernels)
    if n < 0:
        _check(n)
    out = {}
    for i in range(n):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(cnt[i]), float(ms[i]))
    return out
