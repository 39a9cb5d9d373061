"""Python binding of libcl_lattice.so (include/cl_lattice.h).

Argument marshalling only: every step of the lattice method runs in the CUDA
library.  There is no CPU fallback; if the library is missing this module
raises at load time.  PyTorch is used only to hand over CUDA streams and
device buffers (torch tensors as sources/destinations of fields).
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

# --- status codes and enums (mirror include/cl_lattice.h) ---
CL_OK, CL_ERR_ARG, CL_ERR_CUDA, CL_ERR_OOM, CL_ERR_UNSTABLE_DT, CL_ERR_NONFINITE, CL_ERR_TIMEOUT, \
    CL_ERR_STATE, CL_ERR_IO = range(9)
CL_MODEL_SCALAR, CL_MODEL_U1, CL_MODEL_SU2 = 0, 1, 2
CL_INT_LF, CL_INT_VV2, CL_INT_VV4, CL_INT_VV6, CL_INT_VV8, CL_INT_VV10, CL_INT_RK4, CL_INT_GL2, CL_INT_GL3, \
    CL_INT_GL4, CL_INT_GL5 = range(11)
CL_FP64, CL_FP32 = 0, 1
CL_BG_FRIEDMANN, CL_BG_FLUID = 0, 1
CL_POT_HIGGS, CL_POT_MONOMIAL = 0, 1
INTEGRATORS = {"lf": CL_INT_LF, "vv2": CL_INT_VV2, "vv4": CL_INT_VV4, "vv6": CL_INT_VV6, "vv8": CL_INT_VV8,
               "vv10": CL_INT_VV10, "rk4": CL_INT_RK4, "gl2": CL_INT_GL2, "gl3": CL_INT_GL3, "gl4": CL_INT_GL4,
               "gl5": CL_INT_GL5}


def FIELD(i):
    return i


def MOMENTUM(i):
    return 4 + i


def LINK(i):
    return 8 + i


def SU2_LINK(i, c):
    return 16 + 4 * i + c


def SU2_EMOMENTUM(i, a):
    return 28 + 3 * i + a


def EMOMENTUM(i):
    return 12 + i


SINGLET, SINGLET_MOMENTUM = 37, 38


class cl_model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_fields", C.c_int32), ("pexp", C.c_int32), ("background", C.c_int32),
                ("alpha", C.c_double), ("fstar_over_mp", C.c_double), ("omega_over_fstar", C.c_double),
                ("lam", C.c_double), ("q", C.c_double), ("vev2", C.c_double), ("gauge_e", C.c_double),
                ("fluid_w", C.c_double), ("hubble0", C.c_double), ("potential", C.c_int32), ("noncompact", C.c_int32),
                ("gauge_e_u1", C.c_double)]


class cl_grid(C.Structure):
    _fields_ = [("N", C.c_int32), ("integrator", C.c_int32), ("precision", C.c_int32), ("force_dt", C.c_int32),
                ("kIR", C.c_double), ("dt", C.c_double)]


class cl_init(C.Structure):
    _fields_ = [("phi0", C.c_double * 4), ("dphi0", C.c_double * 4), ("seed", C.c_uint64),
                ("spectrum", C.c_int32), ("reserved", C.c_int32), ("fluct_scale", C.c_double), ("a0", C.c_double)]


class cl_means(C.Structure):
    _fields_ = [("t", C.c_double), ("a", C.c_double), ("b", C.c_double), ("step", C.c_int64),
                ("mean", C.c_double * 4), ("mean2", C.c_double * 4), ("var", C.c_double * 4),
                ("mean_pi", C.c_double * 4), ("EK", C.c_double * 4), ("EG", C.c_double * 4),
                ("EV", C.c_double * 4), ("rho", C.c_double), ("w", C.c_double),
                ("hubble_violation", C.c_double), ("gauss_violation", C.c_double), ("reserved", C.c_double * 4)]


class cl_train_cfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("weight_decay", C.c_float), ("standardize", C.c_int32),
                ("lr_end", C.c_float), ("shuffle", C.c_int32)]


SYMBOLS = ["cl_status_str", "cl_last_error", "lattice_init", "lattice_evolve", "lattice_measure_means",
           "lattice_spectrum_bins", "lattice_measure_spectrum", "lattice_measure_gauge_spectrum", "lattice_get_field", "lattice_set_field",
           "lattice_get_stored", "lattice_set_stored",
           "lattice_set_background", "lattice_save", "lattice_restore", "lattice_destroy",
           "lattice_energies_noalloc", "ensemble_init", "ensemble_evolve", "ensemble_observe",
           "ensemble_member", "ensemble_destroy", "ensemble_get_tile", "ensemble_set_tile",
           "ensemble_autotune", "lattice_observe", "surrogate_create", "surrogate_param_count",
           "surrogate_get_params", "surrogate_set_params", "surrogate_loss_grad", "surrogate_train",
           "surrogate_predict", "surrogate_destroy"]
CL_OBS_SIZE = 34

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libcl_lattice.so (building it in-tree if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libcl_lattice.so is not built; run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path)
    vp, d, i32, i64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
    pd, pf = C.POINTER(C.c_double), C.POINTER(C.c_float)
    sig = {
        "cl_status_str": ([C.c_int], C.c_char_p),
        "cl_last_error": ([vp], C.c_char_p),
        "lattice_init": ([C.POINTER(cl_model), C.POINTER(cl_grid), C.POINTER(cl_init), vp, C.POINTER(vp)], C.c_int),
        "lattice_evolve": ([vp, i64], C.c_int),
        "lattice_measure_means": ([vp, C.POINTER(cl_means)], C.c_int),
        "lattice_spectrum_bins": ([vp], i32),
        "lattice_measure_spectrum": ([vp, i32, i32, pd, pd, C.POINTER(C.c_int64)], C.c_int),
        "lattice_measure_gauge_spectrum": ([vp, i32, i32, pd, pd, C.POINTER(C.c_int64)], C.c_int),
        "lattice_get_field": ([vp, i32, vp, i32], C.c_int),
        "lattice_set_field": ([vp, i32, vp, i32], C.c_int),
        "lattice_get_stored": ([vp, i32, vp, pd, i32], C.c_int),
        "lattice_set_stored": ([vp, i32, vp, d, i32], C.c_int),
        "lattice_set_background": ([vp, d, d, d], C.c_int),
        "lattice_save": ([vp, C.c_char_p], C.c_int),
        "lattice_restore": ([vp, C.c_char_p], C.c_int),
        "lattice_destroy": ([vp], C.c_int),
        "lattice_energies_noalloc": ([C.POINTER(cl_model), i32, d, d, vp, vp, vp, vp], C.c_int),
        "ensemble_init": ([i32, C.POINTER(cl_model), pd, C.POINTER(C.c_int32), C.POINTER(C.c_uint64),
                           C.POINTER(cl_grid), C.POINTER(cl_init), vp, C.POINTER(vp)], C.c_int),
        "ensemble_evolve": ([vp, i64], C.c_int),
        "ensemble_observe": ([vp, C.c_double, C.POINTER(C.c_float), pd], C.c_int),
        "ensemble_member": ([vp, i32, C.POINTER(vp)], C.c_int),
        "ensemble_destroy": ([vp], C.c_int),
        "ensemble_get_tile": ([vp, C.POINTER(C.c_int32)], C.c_int),
        "ensemble_set_tile": ([vp, C.POINTER(C.c_int32)], C.c_int),
        "ensemble_autotune": ([vp, i32, C.POINTER(C.c_int32), pd, C.POINTER(C.c_int32)], C.c_int),
        "lattice_observe": ([vp, d, pf, pd], C.c_int),
        "surrogate_create": ([i32, i32, i32, i32, C.c_uint64, vp, C.POINTER(vp)], C.c_int),
        "surrogate_param_count": ([vp], i64),
        "surrogate_get_params": ([vp, pd], C.c_int),
        "surrogate_set_params": ([vp, pd], C.c_int),
        "surrogate_loss_grad": ([vp, pf, pf, i64, pd, pd], C.c_int),
        "surrogate_train": ([vp, pf, pf, i64, C.POINTER(cl_train_cfg), pf], C.c_int),
        "surrogate_predict": ([vp, pf, i64, pf], C.c_int),
        "surrogate_destroy": ([vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class LatticeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (load().cl_status_str(status).decode(), msg))
        self.status = status


def _check(status, handle=None):
    if status != CL_OK:
        raise LatticeError(status, load().cl_last_error(handle).decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dev_ptr(t, n=None):
    """(pointer, on_device) of a contiguous float64 buffer: numpy array or torch
    tensor, of exactly n elements when n is given.  Raises ValueError otherwise,
    so that a short buffer never reaches a copy of n elements."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags.c_contiguous or (n is not None and t.size != n):
            raise ValueError("expected a contiguous float64 array of %s elements, got %s %s" % (n, t.dtype, t.shape))
        return C.c_void_p(t.ctypes.data), 0
    import torch  # only for device buffers
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous() or \
            (n is not None and t.numel() != n):
        raise ValueError("expected a contiguous float64 array or tensor of %s elements" % n)
    return C.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0


def make_model(kind=CL_MODEL_SCALAR, n_fields=1, pexp=2, alpha=0.0, fstar_over_mp=0.0, omega_over_fstar=1.0,
               lam=1.0, q=0.0, vev2=1.0, gauge_e=1.0, background=CL_BG_FRIEDMANN, fluid_w=0.0, hubble0=0.0,
               potential=CL_POT_HIGGS, gauge_e_u1=0.0, noncompact=0):
    return cl_model(kind, n_fields, pexp, background, alpha, fstar_over_mp, omega_over_fstar, lam, q, vev2, gauge_e,
                    fluid_w, hubble0, potential, noncompact, gauge_e_u1)


def make_grid(N, kIR, dt, integrator=CL_INT_VV2, precision=CL_FP64, force_dt=False):
    if isinstance(integrator, str):
        integrator = INTEGRATORS[integrator]
    return cl_grid(N, integrator, precision, 1 if force_dt else 0, kIR, dt)


def make_init(phi0=(0, 0, 0, 0), dphi0=(0, 0, 0, 0), seed=0, spectrum=1, fluct_scale=1.0, a0=1.0):
    p = (C.c_double * 4)(*(list(phi0) + [0.0] * (4 - len(phi0))))
    dp = (C.c_double * 4)(*(list(dphi0) + [0.0] * (4 - len(dphi0))))
    return cl_init(p, dp, seed, spectrum, 0, fluct_scale, a0)


def energies_noalloc(model, N, kIR, a, phi, pi, out, stream=None):
    """lattice_energies_noalloc on caller-owned device tensors (float64, CUDA):
    phi, pi of n_fields x N^3, out of 10 doubles; allocates nothing on the device.
    Raises ValueError for tensors of the wrong dtype, layout, device or size."""
    import torch  # only for device buffers
    need = {"phi": model.n_fields * int(N) ** 3, "pi": model.n_fields * int(N) ** 3, "out": 10}
    dev0 = None
    for name, t in (("phi", phi), ("pi", pi), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA float64 tensor" % name)
        if t.numel() < need[name]:
            raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), need[name]))
        if dev0 is None:
            dev0 = t.device
        elif t.device != dev0:
            raise ValueError("phi, pi and out must be on one device")
    _check(load().lattice_energies_noalloc(C.byref(model), int(N), float(kIR), float(a), _dev_ptr(phi)[0],
                                           _dev_ptr(pi)[0], _dev_ptr(out)[0], _stream_ptr(stream)))


class Lattice:
    """Owner of one cl_lattice handle (see include/cl_lattice.h for semantics)."""

    def __init__(self, model, grid, init, stream=None):
        lib = load()
        h = C.c_void_p()
        _check(lib.lattice_init(C.byref(model), C.byref(grid), C.byref(init), _stream_ptr(stream), C.byref(h)))
        self.h = h
        self.model, self.grid, self.init = model, grid, init
        self.N = grid.N

    def close(self):
        if getattr(self, "h", None):
            load().lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def evolve(self, nsteps):
        _check(load().lattice_evolve(self.h, int(nsteps)), self.h)

    def measure_means(self):
        m = cl_means()
        _check(load().lattice_measure_means(self.h, C.byref(m)), self.h)
        out = {}
        for name, _ in cl_means._fields_:
            v = getattr(m, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    def spectrum(self, field=0, what=0):
        nb = load().lattice_spectrum_bins(self.h)
        k = np.zeros(nb)
        D = np.zeros(nb)
        c = np.zeros(nb, dtype=np.int64)
        _check(load().lattice_measure_spectrum(self.h, field, what, k.ctypes.data_as(C.POINTER(C.c_double)),
                                               D.ctypes.data_as(C.POINTER(C.c_double)),
                                               c.ctypes.data_as(C.POINTER(C.c_int64))), self.h)
        return k, D, c

    def gauge_spectrum(self, sector=0, what=0):
        """Spectrum of the electric (what 0) or magnetic (what 1) field of the
        U(1) (sector 0) or SU(2) (sector 1) gauge field."""
        nb = load().lattice_spectrum_bins(self.h)
        k = np.zeros(nb)
        D = np.zeros(nb)
        c = np.zeros(nb, dtype=np.int64)
        _check(load().lattice_measure_gauge_spectrum(self.h, sector, what, k.ctypes.data_as(C.POINTER(C.c_double)),
                                                     D.ctypes.data_as(C.POINTER(C.c_double)),
                                                     c.ctypes.data_as(C.POINTER(C.c_int64))), self.h)
        return k, D, c

    def observe(self, kmax=0.0):
        """The CL_OBS_SIZE observables (see lattice_observe) and the program time."""
        out = np.zeros(CL_OBS_SIZE, dtype=np.float32)
        t = C.c_double(0.0)
        _check(load().lattice_observe(self.h, float(kmax), out.ctypes.data_as(C.POINTER(C.c_float)), C.byref(t)),
               self.h)
        return out, t.value

    def get_field(self, which, out=None):
        N = self.N
        if out is None:
            out = np.zeros((N, N, N))
        p, dev = _dev_ptr(out, N ** 3)
        _check(load().lattice_get_field(self.h, which, p, dev), self.h)
        return out

    def set_field(self, which, src):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.float64)
        p, dev = _dev_ptr(src, self.N ** 3)
        _check(load().lattice_set_field(self.h, which, p, dev), self.h)

    def _stored_ptr(self, t):
        """(pointer, on_device) of a buffer in the handle's precision."""
        want = np.float32 if self.grid.precision == CL_FP32 else np.float64
        if isinstance(t, np.ndarray):
            if t.dtype != want or not t.flags.c_contiguous or t.size != self.N ** 3:
                raise ValueError("expected a contiguous %s array of N^3 elements" % np.dtype(want).name)
            return C.c_void_p(t.ctypes.data), 0
        import torch  # only for device or pinned buffers
        tw = torch.float32 if want == np.float32 else torch.float64
        if t.dtype != tw or not t.is_contiguous() or t.numel() != self.N ** 3:
            raise ValueError("expected a contiguous %s tensor of N^3 elements" % tw)
        return C.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0

    def get_stored(self, which, out=None):
        """The stored array (handle precision) and its FP64 mean: field = mean + array."""
        if out is None:
            out = np.zeros((self.N,) * 3, dtype=np.float32 if self.grid.precision == CL_FP32 else np.float64)
        p, dev = self._stored_ptr(out)
        mean = C.c_double(0.0)
        _check(load().lattice_get_stored(self.h, which, p, C.byref(mean), dev), self.h)
        return out, mean.value

    def set_stored(self, which, src, mean):
        p, dev = self._stored_ptr(src)
        _check(load().lattice_set_stored(self.h, which, p, float(mean), dev), self.h)

    def set_background(self, a, b=math.nan, t=0.0):
        _check(load().lattice_set_background(self.h, a, b, t), self.h)

    def save(self, path):
        _check(load().lattice_save(self.h, path.encode()), self.h)

    def restore(self, path):
        _check(load().lattice_restore(self.h, path.encode()), self.h)


class _Member(Lattice):
    """Borrowed handle of an ensemble member (owned by the ensemble)."""

    def __init__(self, h, N, grid):
        self.h = h
        self.N = N
        self.grid = grid

    def close(self):
        self.h = None


class Ensemble:
    """Owner of one cl_ensemble (see include/cl_lattice.h)."""

    def __init__(self, model, q, Ns, seeds, grid, init, stream=None):
        lib = load()
        n = len(q)
        qa = np.ascontiguousarray(q, dtype=np.float64)
        Na = np.ascontiguousarray(Ns, dtype=np.int32)
        sa = np.ascontiguousarray(seeds, dtype=np.uint64)
        h = C.c_void_p()
        _check(lib.ensemble_init(n, C.byref(model), qa.ctypes.data_as(C.POINTER(C.c_double)),
                                 Na.ctypes.data_as(C.POINTER(C.c_int32)), sa.ctypes.data_as(C.POINTER(C.c_uint64)),
                                 C.byref(grid), C.byref(init), _stream_ptr(stream), C.byref(h)))
        self.h = h
        self.n = n
        self.Ns = list(Na)
        self.grid = grid

    def evolve(self, nsteps):
        _check(load().ensemble_evolve(self.h, int(nsteps)))

    def observe(self, kmax=0.0):
        out = np.zeros((self.n, CL_OBS_SIZE), dtype=np.float32)
        t = C.c_double(0.0)
        _check(load().ensemble_observe(self.h, float(kmax), out.ctypes.data_as(C.POINTER(C.c_float)), C.byref(t)))
        return out, t.value

    def tile(self):
        t = (C.c_int32 * 4)()
        _check(load().ensemble_get_tile(self.h, t))
        return tuple(t)

    def set_tile(self, tile):
        t = (C.c_int32 * 4)(*[int(v) for v in tile])
        _check(load().ensemble_set_tile(self.h, t))

    def autotune(self, max_report=16):
        """Runs the tile autotuner; returns [(tile, ms per pass), ...] for the shapes tried."""
        tiles = (C.c_int32 * (4 * max_report))()
        ms = (C.c_double * max_report)()
        n = C.c_int32(0)
        _check(load().ensemble_autotune(self.h, int(max_report), tiles, ms, C.byref(n)))
        return [(tuple(tiles[4 * i:4 * i + 4]), ms[i]) for i in range(min(n.value, max_report))]

    def member(self, i):
        h = C.c_void_p()
        _check(load().ensemble_member(self.h, int(i), C.byref(h)))
        return _Member(h, self.Ns[i], self.grid)

    def close(self):
        if getattr(self, "h", None):
            load().ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f32(x, cols):
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError("expected an (n, %d) array, got shape %s" % (cols, a.shape))
    return a


class Surrogate:
    """Owner of one cl_surrogate: BF16 tensor-core MLP (see include/cl_lattice.h)."""

    def __init__(self, n_in, n_out, width=256, depth=3, seed=0, stream=None):
        lib = load()
        h = C.c_void_p()
        _check(lib.surrogate_create(int(n_in), int(n_out), int(width), int(depth), int(seed), _stream_ptr(stream),
                                    C.byref(h)))
        self.h = h
        self.n_in, self.n_out, self.width, self.depth = int(n_in), int(n_out), int(width), int(depth)
        self.dims = [self.n_in] + [self.width] * self.depth + [self.n_out]

    def param_count(self):
        return int(load().surrogate_param_count(self.h))

    def get_params(self):
        out = np.zeros(self.param_count(), dtype=np.float64)
        _check(load().surrogate_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float64)
        if t.size != self.param_count():
            raise ValueError("expected %d parameters" % self.param_count())
        _check(load().surrogate_set_params(self.h, t.ctypes.data_as(C.POINTER(C.c_double))))

    def loss_grad(self, X, T):
        X, T = _f32(X, self.n_in), _f32(T, self.n_out)
        loss = C.c_double(0.0)
        g = np.zeros(self.param_count(), dtype=np.float64)
        pf = C.POINTER(C.c_float)
        _check(load().surrogate_loss_grad(self.h, X.ctypes.data_as(pf), T.ctypes.data_as(pf), X.shape[0],
                                          C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_double))))
        return loss.value, g

    def train(self, X, Y, epochs, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
              standardize=True, lr_end=-1.0, shuffle=False):
        """Adam on (X, Y); lr_end >= 0 anneals the step size (cosine) to lr_end.
        Returns the per-epoch mean squared error."""
        X, Y = _f32(X, self.n_in), _f32(Y, self.n_out)
        cfg = cl_train_cfg(int(epochs), int(batch), lr, beta1, beta2, eps, weight_decay, int(bool(standardize)),
                           float(lr_end), int(bool(shuffle)))
        hist = np.zeros(int(epochs), dtype=np.float32)
        pf = C.POINTER(C.c_float)
        _check(load().surrogate_train(self.h, X.ctypes.data_as(pf), Y.ctypes.data_as(pf), X.shape[0], C.byref(cfg),
                                      hist.ctypes.data_as(pf)))
        return hist

    def predict(self, X):
        X = _f32(X, self.n_in)
        Y = np.zeros((X.shape[0], self.n_out), dtype=np.float32)
        pf = C.POINTER(C.c_float)
        _check(load().surrogate_predict(self.h, X.ctypes.data_as(pf), X.shape[0], Y.ctypes.data_as(pf)))
        return Y

    def close(self):
        if getattr(self, "h", None):
            load().surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
