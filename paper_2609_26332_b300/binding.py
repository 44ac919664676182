"""ctypes binding of the C ABI in ``include/surflbm.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``libsurflbm.so``; this module only
converts numpy arrays / torch streams to pointers and status codes to exceptions.
Importing it loads the library and raises if it is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsurflbm.so")

SLBM_OK, SLBM_EINVAL, SLBM_ENOMEM, SLBM_ECUDA, SLBM_EUNSTABLE, SLBM_ESTATE = range(6)
FP32, FP16DEV, BF16DEV = 0, 1, 2
NONLINEAR, LINEAR = 0, 1
PAPER, TARGET = 0, 1
_PREC = {"fp32": FP32, "fp16": FP16DEV, "bf16": BF16DEV}


class SlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"surflbm status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau_f", ctypes.c_double), ("tau_f_gas", ctypes.c_double),
        ("tau_g", ctypes.c_double), ("tau_h", ctypes.c_double),
        ("mrt_f", ctypes.c_double * 4), ("mrt_g", ctypes.c_double * 4), ("mrt_h", ctypes.c_double * 4),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double), ("Ex", ctypes.c_double), ("Pi", ctypes.c_double),
        ("M_phi", ctypes.c_double), ("M_psi", ctypes.c_double),
        ("eta_phi", ctypes.c_double), ("eta_psi", ctypes.c_double),
        ("lambda_s", ctypes.c_double), ("psi_b", ctypes.c_double), ("phi_b", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double), ("Gx", ctypes.c_double), ("Gy", ctypes.c_double),
        ("constraint", ctypes.c_int), ("multiplier", ctypes.c_int), ("precision", ctypes.c_int),
        ("psi_on", ctypes.c_int),
    ]


class Totals(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_longlong), ("Q_phi", ctypes.c_double), ("H", ctypes.c_double),
        ("phi_total", ctypes.c_double), ("psi_total", ctypes.c_double), ("lambda_phi", ctypes.c_double),
        ("mubar_psi", ctypes.c_double), ("kinetic", ctypes.c_double), ("S1", ctypes.c_double),
        ("S2", ctypes.c_double), ("clamp_count", ctypes.c_longlong), ("range_count", ctypes.c_longlong),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_26332_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    L.slbm_default_params.argtypes = [ctypes.POINTER(Params), i, i]
    L.slbm_default_params.restype = None
    L.slbm_create_domain.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    L.slbm_set_walls.argtypes = [vp, i, d, d, d, d]
    L.slbm_init_fields.argtypes = [vp, dp, dp]
    L.slbm_step.argtypes = [vp, ll]
    L.slbm_read_fields.argtypes = [vp, dp, dp, dp, dp, dp]
    L.slbm_read_totals.argtypes = [vp, ctypes.POINTER(Totals)]
    L.slbm_read_fields_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(Totals)]
    L.slbm_read_fields_noalloc.restype = ctypes.c_int
    L.slbm_device_bytes.argtypes = [vp]
    L.slbm_device_bytes.restype = ctypes.c_size_t
    L.slbm_destroy.argtypes = [vp]
    L.slbm_destroy.restype = None
    L.slbm_last_error.argtypes = [vp]
    L.slbm_last_error.restype = ctypes.c_char_p
    L.slbm_version.restype = ctypes.c_char_p
    for name in ("slbm_create_domain", "slbm_set_walls", "slbm_init_fields", "slbm_step",
                 "slbm_read_fields", "slbm_read_totals"):
        getattr(L, name).restype = ctypes.c_int
    return L


lib = _load()


def default_params(nx, ny, **kw):
    """slbm_default_params plus keyword overrides (precision may be 'fp32'/'fp16'/'bf16')."""
    p = Params()
    lib.slbm_default_params(ctypes.byref(p), int(nx), int(ny))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = _PREC[v]
        if k in ("mrt_f", "mrt_g", "mrt_h"):
            arr = getattr(p, k)
            for j, x in enumerate(v):
                arr[j] = float(x)
            continue
        if not hasattr(p, k):
            raise AttributeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _stream_handle(stream):
    if stream is None:
        return None
    h = getattr(stream, "cuda_stream", stream)
    return ctypes.c_void_p(int(h))


class Domain:
    """One simulation domain living on the current CUDA device."""

    def __init__(self, params, stream=None):
        self._h = ctypes.c_void_p()
        self.nx, self.ny = params.nx, params.ny
        st = lib.slbm_create_domain(ctypes.byref(params), _stream_handle(stream), ctypes.byref(self._h))
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_last_error(None).decode())
        self.params = params

    def _check(self, st):
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_last_error(self._h).decode())

    def set_wall(self, wall, theta0_deg=90.0, beta_sg=0.0, beta_sl=0.0, u_x=0.0):
        self._check(lib.slbm_set_walls(self._h, int(wall), float(theta0_deg), float(beta_sg), float(beta_sl),
                                       float(u_x)))

    def init_fields(self, phi, psi=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if phi.shape != (self.ny, self.nx):
            raise ValueError("phi must have shape (ny, nx)")
        if psi is not None:
            psi = np.ascontiguousarray(psi, dtype=np.float64)
            if psi.shape != (self.ny, self.nx):
                raise ValueError("psi must have shape (ny, nx)")
        self._check(lib.slbm_init_fields(self._h, _dptr(phi), _dptr(psi)))

    def step(self, n=1):
        self._check(lib.slbm_step(self._h, int(n)))

    def read_fields(self, which=("phi", "psi", "ux", "uy", "p")):
        out = {k: np.empty((self.ny, self.nx), dtype=np.float64) for k in which}
        ptrs = [_dptr(out.get(k)) for k in ("phi", "psi", "ux", "uy", "p")]
        self._check(lib.slbm_read_fields(self._h, *ptrs))
        return out

    def read_totals(self, check=True):
        t = Totals()
        st = lib.slbm_read_totals(self._h, ctypes.byref(t))
        if check:
            self._check(st)
        return {name: getattr(t, name) for name, _ in Totals._fields_}

    def read_fields_noalloc(self, phi=None, psi=None, ux=None, uy=None, p=None, totals=True):
        """Fields written into caller-owned DEVICE buffers (e.g. torch CUDA tensors of
        float64 with nx*ny elements, or raw device addresses); the library allocates
        nothing.  Returns the totals dict when ``totals`` is true (synchronises)."""
        def ptr(x):
            if x is None:
                return None
            if hasattr(x, "data_ptr"):
                if x.numel() != self.nx * self.ny or x.element_size() != 8 or not x.is_contiguous():
                    raise ValueError("device buffers must be contiguous float64 with nx*ny elements")
                return ctypes.c_void_p(x.data_ptr())
            return ctypes.c_void_p(int(x))
        t = Totals() if totals else None
        self._check(lib.slbm_read_fields_noalloc(self._h, ptr(phi), ptr(psi), ptr(ux), ptr(uy), ptr(p),
                                                 ctypes.byref(t) if t is not None else None))
        return {name: getattr(t, name) for name, _ in Totals._fields_} if t is not None else None

    @property
    def device_bytes(self):
        return int(lib.slbm_device_bytes(self._h))

    def close(self):
        if self._h:
            lib.slbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def version():
    return lib.slbm_version().decode()
