"""ctypes binding of libfftlb.so (C ABI in include/fftlb.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers are passed as integer addresses (for example
``tensor.data_ptr()`` of a CUDA tensor) with ``on_device=True``; host
buffers as float64 C-contiguous numpy arrays.  Importing this module loads
the library and raises if it has not been built (``build.build()``).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfftlb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libfftlb.so is not built: run paper_1011_3582_gb300.build.build() "
                      "(or __graft_entry__.build()) first")
_lib = ct.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_UNSTABLE, ERR_TIMEOUT, ERR_STATE = range(7)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_OOM", "ERR_CUDA", "ERR_UNSTABLE", "ERR_TIMEOUT", "ERR_STATE"]

EXPORTED = ["fftlb_create", "fftlb_set_fields", "fftlb_step", "fftlb_fields", "fftlb_get_f",
            "fftlb_set_f", "fftlb_invariants", "fftlb_gradient", "fftlb_save", "fftlb_load",
            "fftlb_destroy", "fftlb_last_error", "fftlb_launches_per_step", "fftlb_profile",
            "fftlb_profile_read", "fftlb_kernel_name", "fftlb_gradient_static", "fftlb_autotune",
            "fftlb_tuning", "fftlb_debug_wait_test", "fftlb_batch_create", "fftlb_batch_set_fields", "fftlb_batch_step",
            "fftlb_batch_fields", "fftlb_batch_get_f", "fftlb_batch_invariants", "fftlb_batch_tuning",
            "fftlb_batch_launches_per_step", "fftlb_batch_destroy", "fftlb_batch_last_error",
            "fftlb_cnn_create", "fftlb_cnn_destroy", "fftlb_cnn_last_error", "fftlb_cnn_set_params",
            "fftlb_cnn_get_params", "fftlb_cnn_forward", "fftlb_cnn_gradient", "fftlb_cnn_train_step",
            "fftlb_cnn_encode", "fftlb_cnn_warm_start", "fftlb_cnn_launches"]

CNN_NPARAMS = 32 * 9 * 3 + 32 + 32 * 9 * 32 + 32 + 32 * 9 * 32 + 32 + 2 * 9 * 32 + 2


class fftlb_params(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int),
                ("dx", ct.c_double), ("dt", ct.c_double), ("tau", ct.c_double),
                ("a", ct.c_double), ("b", ct.c_double), ("K", ct.c_double), ("H", ct.c_double),
                ("q", ct.c_double), ("zeta", ct.c_double),
                ("window", ct.c_int), ("integrator", ct.c_int), ("precision", ct.c_int),
                ("check_every", ct.c_int)]


class fftlb_velset(ct.Structure):
    _fields_ = [("nspeeds", ct.c_int), ("speeds", ct.POINTER(ct.c_double)), ("ndirs", ct.c_int)]


_h = ct.c_void_p
_p = ct.c_void_p
_lib.fftlb_create.argtypes = [ct.POINTER(_h), ct.POINTER(fftlb_params), ct.POINTER(fftlb_velset), _p]
_lib.fftlb_set_fields.argtypes = [_h, _p, _p, _p, _p, ct.c_int]
_lib.fftlb_step.argtypes = [_h, ct.c_long, ct.POINTER(ct.c_long)]
_lib.fftlb_fields.argtypes = [_h, _p, _p, _p, _p, ct.c_int]
_lib.fftlb_get_f.argtypes = [_h, _p, ct.c_int]
_lib.fftlb_set_f.argtypes = [_h, _p, ct.c_int]
_lib.fftlb_invariants.argtypes = [_h, ct.POINTER(ct.c_double)]
_lib.fftlb_gradient.argtypes = [_h, _p, _p, ct.c_int]
_lib.fftlb_save.argtypes = [_h, ct.c_char_p]
_lib.fftlb_load.argtypes = [_h, ct.c_char_p]
_lib.fftlb_destroy.argtypes = [_h]
_lib.fftlb_last_error.argtypes = [_h]
_lib.fftlb_last_error.restype = ct.c_char_p
_lib.fftlb_launches_per_step.argtypes = [_h]
_lib.fftlb_launches_per_step.restype = ct.c_int
_lib.fftlb_profile.argtypes = [_h, ct.c_int]
_lib.fftlb_profile_read.argtypes = [_h, ct.POINTER(ct.c_double), ct.POINTER(ct.c_long),
                                    ct.POINTER(ct.c_double), ct.c_int]
_lib.fftlb_gradient_static.argtypes = [_p, _p, ct.c_int, ct.c_int, ct.c_double, ct.c_int, _p]
_lib.fftlb_autotune.argtypes = [_h, ct.POINTER(ct.c_double)]
_lib.fftlb_tuning.argtypes = [_h, ct.POINTER(ct.c_int), ct.c_int]
_lib.fftlb_debug_wait_test.argtypes = [_h, ct.c_longlong]
_lib.fftlb_batch_create.argtypes = [ct.POINTER(_h), ct.c_int, ct.POINTER(fftlb_params), ct.POINTER(fftlb_velset),
                                    ct.c_int, _p]
_lib.fftlb_batch_set_fields.argtypes = [_h, ct.c_int, _p, _p, _p, _p, ct.c_int]
_lib.fftlb_batch_step.argtypes = [_h, ct.c_long]
_lib.fftlb_batch_fields.argtypes = [_h, ct.c_int, _p, _p, _p, _p, ct.c_int]
_lib.fftlb_batch_get_f.argtypes = [_h, ct.c_int, _p, ct.c_int]
_lib.fftlb_batch_invariants.argtypes = [_h, ct.c_int, ct.POINTER(ct.c_double)]
_lib.fftlb_batch_tuning.argtypes = [_h, ct.c_int, ct.POINTER(ct.c_int)]
_lib.fftlb_batch_launches_per_step.argtypes = [_h]
_lib.fftlb_batch_launches_per_step.restype = ct.c_long
_lib.fftlb_batch_destroy.argtypes = [_h]
_lib.fftlb_batch_last_error.argtypes = [_h]
_lib.fftlb_batch_last_error.restype = ct.c_char_p
_lib.fftlb_kernel_name.argtypes = [ct.c_int]
_lib.fftlb_kernel_name.restype = ct.c_char_p
for _n in EXPORTED:
    if _n not in ("fftlb_last_error", "fftlb_launches_per_step", "fftlb_kernel_name",
                  "fftlb_batch_launches_per_step", "fftlb_batch_last_error"):
        getattr(_lib, _n).restype = ct.c_int


class FFTLBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


def _addr(x, on_device, count=None):
    """Address of a buffer handed to the C calls.  Host buffers: C-contiguous
    float64 numpy arrays; device buffers: torch tensors (float64, contiguous,
    on a CUDA device) or raw integer addresses.  count: required number of
    float64 elements (checked for arrays and tensors)."""
    if x is None:
        return None
    if on_device:
        if isinstance(x, int):
            return x
        if not (x.is_cuda and x.dtype == torch_float64() and x.is_contiguous()):
            raise TypeError("device buffers must be contiguous float64 CUDA tensors")
        if count is not None and x.numel() != count:
            raise ValueError(f"device buffer has {x.numel()} elements, expected {count}")
        return int(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise TypeError("host buffers must be C-contiguous float64 numpy arrays")
    if count is not None and x.size != count:
        raise ValueError(f"host buffer has {x.size} elements, expected {count}")
    return x.ctypes.data


def torch_float64():
    import torch
    return torch.float64


# precision flag: fp32 with split-BF16 tensor-core first radix-16 passes
BF16SPLIT = 256


def params(nx, ny, dx=1.0 / 256, dt=1e-5, tau=1e-2, a=9.0 / 8.0, b=1.0 / 3.0, K=1e-5, H=0.0,
           q=-0.004, zeta=0.0, window=4, integrator=3, precision=64, check_every=0):
    """fftlb_params with the paper's defaults (Sec. 3)."""
    return fftlb_params(nx, ny, dx, dt, tau, a, b, K, H, q, zeta, window, integrator, precision,
                        check_every)


class Handle:
    """Owning wrapper of an fftlb_t.  Method names follow the C calls."""

    def __init__(self, p: fftlb_params, speeds=None, stream=0):
        self._h = _h()
        vs = None
        if speeds is not None:
            arr = (ct.c_double * 4)(*speeds)
            self._speeds = arr
            vs = ct.byref(fftlb_velset(4, ct.cast(arr, ct.POINTER(ct.c_double)), 8))
        self.params = p
        st = _lib.fftlb_create(ct.byref(self._h), ct.byref(p), vs, ct.c_void_p(int(stream)))
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_last_error(None).decode())

    def _check(self, st):
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.params.ny, self.params.nx)

    @property
    def sites(self):
        return self.params.nx * self.params.ny

    def set_fields(self, rho, ux, uy, T, on_device=False):
        a = [_addr(v, on_device, self.sites) for v in (rho, ux, uy, T)]
        self._check(_lib.fftlb_set_fields(self._h, *a, int(on_device)))

    def step(self, nsteps=1):
        done = ct.c_long(0)
        st = _lib.fftlb_step(self._h, int(nsteps), ct.byref(done))
        if st != OK:
            err = FFTLBError(st, _lib.fftlb_last_error(self._h).decode())
            err.steps_done = done.value
            raise err
        return done.value

    def fields(self, rho=None, ux=None, uy=None, T=None, on_device=False):
        if not on_device and rho is None and ux is None and uy is None and T is None:
            rho, ux, uy, T = (np.empty(self.shape) for _ in range(4))
        a = [_addr(v, on_device, self.sites) for v in (rho, ux, uy, T)]
        self._check(_lib.fftlb_fields(self._h, *a, int(on_device)))
        return rho, ux, uy, T

    def get_f(self, out=None, on_device=False):
        if out is None:
            out = np.empty((33,) + self.shape)
        self._check(_lib.fftlb_get_f(self._h, _addr(out, on_device, 33 * self.sites), int(on_device)))
        return out

    def set_f(self, f, on_device=False):
        self._check(_lib.fftlb_set_f(self._h, _addr(f, on_device, 33 * self.sites), int(on_device)))

    def invariants(self):
        out = (ct.c_double * 6)()
        self._check(_lib.fftlb_invariants(self._h, out))
        return dict(mass=out[0], px=out[1], py=out[2], eT=out[3], umax=out[4], time=out[5])

    def gradient(self, g, out, nfields):
        """g, out: device addresses (fp64 [nfields][ny][nx] and [2 nfields][ny][nx])."""
        n = self.sites * int(nfields)
        self._check(_lib.fftlb_gradient(self._h, _addr(g, True, n), _addr(out, True, 2 * n), int(nfields)))

    def save(self, path):
        self._check(_lib.fftlb_save(self._h, path.encode()))

    def load(self, path):
        self._check(_lib.fftlb_load(self._h, path.encode()))

    def launches_per_step(self):
        return _lib.fftlb_launches_per_step(self._h)

    def profile(self, enable=True):
        self._check(_lib.fftlb_profile(self._h, int(enable)))

    def profile_read(self):
        """{kernel name: (total ms, launches, algorithmic bytes per launch)}."""
        ms = (ct.c_double * 6)()
        n = (ct.c_long * 6)()
        by = (ct.c_double * 6)()
        self._check(_lib.fftlb_profile_read(self._h, ms, n, by, 6))
        return {_lib.fftlb_kernel_name(k).decode(): (ms[k], n[k], by[k]) for k in range(6)}

    def autotune(self):
        """fftlb_autotune: returns the best stage time in ms."""
        ms = ct.c_double(0)
        self._check(_lib.fftlb_autotune(self._h, ct.byref(ms)))
        return ms.value

    def tuning(self, values=None):
        t = (ct.c_int * 5)(*(values or [0] * 5))
        self._check(_lib.fftlb_tuning(self._h, t, 0 if values is None else 1))
        return list(t)

    def debug_wait_test(self, ns):
        """fftlb_debug_wait_test: every later stage starts with a kernel whose
        bounded wait nothing completes (limit ns; 0 = off)."""
        self._check(_lib.fftlb_debug_wait_test(self._h, int(ns)))

    def close(self):
        if self._h:
            _lib.fftlb_destroy(self._h)
            self._h = _h()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class fftlb_cnn_norm(ct.Structure):
    _fields_ = [("rho_c", ct.c_double), ("T_c", ct.c_double), ("s_rho", ct.c_double), ("s_T", ct.c_double)]


_lib.fftlb_cnn_create.argtypes = [ct.POINTER(_h), ct.c_int, ct.c_int, _p]
_lib.fftlb_cnn_destroy.argtypes = [_h]
_lib.fftlb_cnn_last_error.argtypes = [_h]
_lib.fftlb_cnn_last_error.restype = ct.c_char_p
_lib.fftlb_cnn_set_params.argtypes = [_h, _p, ct.c_int]
_lib.fftlb_cnn_get_params.argtypes = [_h, _p]
_lib.fftlb_cnn_forward.argtypes = [_h, _p, _p, ct.c_int]
_lib.fftlb_cnn_gradient.argtypes = [_h, _p, _p, _p, ct.POINTER(ct.c_double), ct.c_int]
_lib.fftlb_cnn_train_step.argtypes = [_h, _p, _p, ct.c_float, ct.POINTER(ct.c_double), ct.c_int]
_lib.fftlb_cnn_encode.argtypes = [_h, _h, ct.c_double, ct.POINTER(fftlb_cnn_norm), _p]
_lib.fftlb_cnn_warm_start.argtypes = [_h, _h, ct.c_double, ct.POINTER(fftlb_cnn_norm)]
_lib.fftlb_cnn_launches.argtypes = [_h]
_lib.fftlb_cnn_launches.restype = ct.c_long


def _faddr(x, on_device, count):
    """Address of a float32 buffer (numpy on the host, torch on the device)."""
    if on_device:
        if isinstance(x, int):
            return x
        import torch
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise TypeError("device buffers must be contiguous float32 CUDA tensors")
        if x.numel() != count:
            raise ValueError(f"device buffer has {x.numel()} elements, expected {count}")
        return int(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.dtype == np.float32 and x.flags.c_contiguous):
        raise TypeError("host buffers must be C-contiguous float32 numpy arrays")
    if x.size != count:
        raise ValueError(f"host buffer has {x.size} elements, expected {count}")
    return x.ctypes.data


class CNN:
    """Owning wrapper of an fftlb_cnn_t (the learned warm start)."""

    def __init__(self, H, W, stream=0):
        self._h = _h()
        self.H, self.W = int(H), int(W)
        st = _lib.fftlb_cnn_create(ct.byref(self._h), self.H, self.W, ct.c_void_p(int(stream)))
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_last_error(None).decode())

    def _check(self, st):
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_cnn_last_error(self._h).decode())

    @property
    def P(self):
        return self.H * self.W

    def set_params(self, params, reset_optimizer=True):
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != CNN_NPARAMS:
            raise ValueError(f"expected {CNN_NPARAMS} parameters")
        self._check(_lib.fftlb_cnn_set_params(self._h, a.ctypes.data, int(bool(reset_optimizer))))

    def get_params(self):
        a = np.empty(CNN_NPARAMS, np.float32)
        self._check(_lib.fftlb_cnn_get_params(self._h, a.ctypes.data))
        return a

    def forward(self, X, Y=None, on_device=False):
        if Y is None and not on_device:
            Y = np.empty((2, self.H, self.W), np.float32)
        self._check(_lib.fftlb_cnn_forward(self._h, _faddr(X, on_device, 3 * self.P),
                                           _faddr(Y, on_device, 2 * self.P), int(on_device)))
        return Y

    def gradient(self, X, Xt, on_device=False):
        g = np.empty(CNN_NPARAMS, np.float32)
        loss = ct.c_double(0)
        self._check(_lib.fftlb_cnn_gradient(self._h, _faddr(X, on_device, 3 * self.P),
                                            _faddr(Xt, on_device, 2 * self.P), g.ctypes.data, ct.byref(loss),
                                            int(on_device)))
        return loss.value, g

    def train_step(self, X, Xt, lr, on_device=False, want_loss=True):
        loss = ct.c_double(0)
        self._check(_lib.fftlb_cnn_train_step(self._h, _faddr(X, on_device, 3 * self.P),
                                              _faddr(Xt, on_device, 2 * self.P), float(lr),
                                              ct.byref(loss) if want_loss else None, int(on_device)))
        return loss.value if want_loss else None

    def encode(self, handle, T_run, norm, X_dev):
        self._check(_lib.fftlb_cnn_encode(self._h, handle._h, float(T_run), ct.byref(norm),
                                          _faddr(X_dev, True, 3 * self.P)))

    def warm_start(self, handle, T_run, norm):
        self._check(_lib.fftlb_cnn_warm_start(self._h, handle._h, float(T_run), ct.byref(norm)))

    def launches(self):
        return _lib.fftlb_cnn_launches(self._h)

    def close(self):
        if self._h:
            _lib.fftlb_cnn_destroy(self._h)
            self._h = _h()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def pack_params(params):
    """Flatten [(W_l [out, 3, 3, in], b_l [out]), ...] into the fp32 vector
    of the C ABI (W_1, b_1, W_2, b_2, ...)."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64).ravel()])
                           for W, b in params]).astype(np.float32)


def unpack_params(vec, layers=((3, 32), (32, 32), (32, 32), (32, 2))):
    out, o = [], 0
    for ci, co in layers:
        W = np.asarray(vec[o:o + co * 9 * ci], np.float64).reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = np.asarray(vec[o:o + co], np.float64)
        o += co
        out.append((W, b))
    return out


class Batch:
    """Owning wrapper of an fftlb_batch_t (batched sweep of independent runs)."""

    def __init__(self, params_list, speeds=None, autotune=True, stream=0):
        self._h = _h()
        n = len(params_list)
        arr = (fftlb_params * n)(*params_list)
        vs = None
        if speeds is not None:
            sp = (ct.c_double * 4)(*speeds)
            self._speeds = sp
            vs = ct.byref(fftlb_velset(4, ct.cast(sp, ct.POINTER(ct.c_double)), 8))
        self.params = list(params_list)
        st = _lib.fftlb_batch_create(ct.byref(self._h), n, arr, vs, int(bool(autotune)), ct.c_void_p(int(stream)))
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_last_error(None).decode())

    def _check(self, st):
        if st != OK:
            raise FFTLBError(st, _lib.fftlb_batch_last_error(self._h).decode())

    def __len__(self):
        return len(self.params)

    def shape(self, run):
        p = self.params[run]
        return (p.ny, p.nx)

    def set_fields(self, run, rho, ux, uy, T, on_device=False):
        ny, nx = self.shape(run)
        a = [_addr(v, on_device, nx * ny) for v in (rho, ux, uy, T)]
        self._check(_lib.fftlb_batch_set_fields(self._h, int(run), *a, int(on_device)))

    def step(self, nsteps=1):
        self._check(_lib.fftlb_batch_step(self._h, int(nsteps)))

    def fields(self, run):
        out = [np.empty(self.shape(run)) for _ in range(4)]
        self._check(_lib.fftlb_batch_fields(self._h, int(run), *[_addr(v, False) for v in out], 0))
        return out

    def get_f(self, run):
        out = np.empty((33,) + self.shape(run))
        self._check(_lib.fftlb_batch_get_f(self._h, int(run), _addr(out, False), 0))
        return out

    def invariants(self, run):
        out = (ct.c_double * 6)()
        self._check(_lib.fftlb_batch_invariants(self._h, int(run), out))
        return dict(mass=out[0], px=out[1], py=out[2], eT=out[3], umax=out[4], time=out[5])

    def tuning(self, run):
        t = (ct.c_int * 5)()
        self._check(_lib.fftlb_batch_tuning(self._h, int(run), t))
        return list(t)

    def launches_per_step(self):
        return _lib.fftlb_batch_launches_per_step(self._h)

    def close(self):
        if self._h:
            _lib.fftlb_batch_destroy(self._h)
            self._h = _h()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def gradient_static(g, out, nx, ny, dx=1.0 / 256, window=4, stream=0):
    """fftlb_gradient_static: D_x, D_y of one fp64 device field without any
    device allocation (g, out: device addresses of [ny][nx] and [2][ny][nx])."""
    st = _lib.fftlb_gradient_static(_addr(g, True, nx * ny), _addr(out, True, 2 * nx * ny), int(nx), int(ny), float(dx),
                                    int(window), ct.c_void_p(int(stream)))
    if st != OK:
        raise FFTLBError(st, _lib.fftlb_last_error(None).decode())


def lib():
    return _lib
