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
PAPER, TARGET, EXACT = 0, 1, 2
CPASYNC, TMA = 0, 1
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
        ("psi_on", ctypes.c_int), ("wall_saturation", ctypes.c_int), ("staging", ctypes.c_int),
    ]


class WallSpec(ctypes.Structure):
    _fields_ = [("theta0_deg", ctypes.c_double), ("beta_sg", ctypes.c_double), ("beta_sl", ctypes.c_double),
                ("u_x", ctypes.c_double)]


class MMS(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("amplitude", "u", "M", "beta", "kappa", "kT", "W", "dx", "dt")]


class Totals(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_longlong), ("Q_phi", ctypes.c_double), ("H", ctypes.c_double),
        ("phi_total", ctypes.c_double), ("psi_total", ctypes.c_double), ("lambda_phi", ctypes.c_double),
        ("mubar_psi", ctypes.c_double), ("kinetic", ctypes.c_double), ("S1", ctypes.c_double),
        ("S2", ctypes.c_double), ("clamp_count", ctypes.c_longlong), ("range_count", ctypes.c_longlong),
        ("free_energy", ctypes.c_double), ("residual", ctypes.c_double),
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
    L.slbm_device_allocations.argtypes = []
    L.slbm_device_allocations.restype = ctypes.c_ulonglong
    L.slbm_workspace_bytes.argtypes = [ctypes.POINTER(Params)]
    L.slbm_workspace_bytes.restype = ctypes.c_size_t
    L.slbm_create_domain_ext.argtypes = [ctypes.POINTER(Params), vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.slbm_set_mms.argtypes = [vp, ctypes.POINTER(MMS)]
    L.slbm_save.argtypes = [vp, ctypes.c_char_p]
    L.slbm_load.argtypes = [vp, ctypes.c_char_p]
    L.slbm_destroy.argtypes = [vp]
    L.slbm_destroy.restype = None
    L.slbm_last_error.argtypes = [vp]
    L.slbm_last_error.restype = ctypes.c_char_p
    L.slbm_version.restype = ctypes.c_char_p
    for name in ("slbm_create_domain", "slbm_set_walls", "slbm_init_fields", "slbm_step",
                 "slbm_read_fields", "slbm_read_totals", "slbm_create_domain_ext", "slbm_save", "slbm_load",
                 "slbm_set_mms"):
        getattr(L, name).restype = ctypes.c_int
    # three-dimensional extension
    L.slbm3d_create_domain.argtypes = [ctypes.POINTER(Params), i, vp, ctypes.POINTER(vp)]
    L.slbm3d_set_walls.argtypes = [vp, i, d, d, d, d]
    L.slbm3d_init_fields.argtypes = [vp, dp, dp]
    L.slbm3d_step.argtypes = [vp, ll]
    L.slbm3d_read_fields.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    L.slbm3d_read_totals.argtypes = [vp, ctypes.POINTER(Totals)]
    L.slbm3d_device_bytes.argtypes = [vp]
    L.slbm3d_device_bytes.restype = ctypes.c_size_t
    L.slbm3d_destroy.argtypes = [vp]
    L.slbm3d_destroy.restype = None
    L.slbm3d_last_error.argtypes = [vp]
    L.slbm3d_last_error.restype = ctypes.c_char_p
    for name in ("slbm3d_create_domain", "slbm3d_set_walls", "slbm3d_init_fields", "slbm3d_step",
                 "slbm3d_read_fields", "slbm3d_read_totals"):
        getattr(L, name).restype = ctypes.c_int
    # batches
    L.slbm_create_batch.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(WallSpec), i, vp, ctypes.POINTER(vp)]
    L.slbm_batch_init_fields.argtypes = [vp, i, dp, dp]
    L.slbm_batch_set_tiling.argtypes = [vp, i, i, i]
    L.slbm_batch_set_strip_width.argtypes = [vp, i]
    L.slbm_batch_get_tiling.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.slbm_batch_autotune.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.slbm_batch_step.argtypes = [vp, ll]
    L.slbm_batch_run_to_equilibrium.argtypes = [vp, d, ll, i, ctypes.POINTER(ll)]
    L.slbm_batch_step_instance.argtypes = [vp, i, ll]
    L.slbm_batch_read_fields.argtypes = [vp, i, dp, dp, dp, dp, dp]
    L.slbm_batch_read_totals.argtypes = [vp, i, ctypes.POINTER(Totals)]
    for name in ("slbm_create_batch", "slbm_batch_init_fields", "slbm_batch_set_tiling", "slbm_batch_autotune",
                 "slbm_batch_set_strip_width", "slbm_batch_get_tiling",
                 "slbm_batch_step", "slbm_batch_run_to_equilibrium", "slbm_batch_step_instance",
                 "slbm_batch_read_fields", "slbm_batch_read_totals"):
        getattr(L, name).restype = ctypes.c_int
    L.slbm_batch_active.argtypes = [vp, ctypes.POINTER(i)]
    L.slbm_batch_active.restype = i
    L.slbm_batch_device_bytes.argtypes = [vp]
    L.slbm_batch_device_bytes.restype = ctypes.c_size_t
    L.slbm_batch_last_error.argtypes = [vp]
    L.slbm_batch_last_error.restype = ctypes.c_char_p
    L.slbm_batch_destroy.argtypes = [vp]
    L.slbm_batch_destroy.restype = None
    L.slbm_init_fields_device.argtypes = [vp, vp, vp]
    L.slbm_batch_init_fields_device.argtypes = [vp, i, vp, vp]
    # warm-start network and its conv primitives (include/surflbm_ws.h)
    fp = ctypes.POINTER(ctypes.c_float)
    L.slbm_conv3x3_forward.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp]
    L.slbm_conv3x3_flip_weights.argtypes = [vp, vp, i, i, vp]
    L.slbm_conv3x3_input_grad.argtypes = [vp, vp, vp, vp, i, i, i, i, i, vp]
    L.slbm_conv3x3_weight_grad.argtypes = [vp, vp, vp, i, i, i, i, i, vp]
    L.slbm_conv_error.argtypes = [ctypes.POINTER(i)]
    L.slbm_ws_create.argtypes = [i, i, i, ctypes.c_ulonglong, vp, ctypes.POINTER(vp)]
    L.slbm_ws_param_count.argtypes = [vp]
    L.slbm_ws_param_count.restype = ll
    L.slbm_ws_get_params.argtypes = [vp, fp]
    L.slbm_ws_set_params.argtypes = [vp, fp]
    L.slbm_ws_forward.argtypes = [vp, vp, i, vp]
    L.slbm_ws_loss_grad.argtypes = [vp, vp, vp, vp, i, dp, fp]
    L.slbm_ws_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.slbm_ws_train_step.argtypes = [vp, vp, vp, vp, i, ctypes.c_float, dp]
    L.slbm_ws_batch_targets.argtypes = [vp, vp, i, d, vp]
    L.slbm_ws_warm_start.argtypes = [vp, vp, ctypes.POINTER(i), fp, i, ctypes.POINTER(i)]
    L.slbm_ws_device_bytes.argtypes = [vp]
    L.slbm_ws_device_bytes.restype = ctypes.c_size_t
    L.slbm_ws_last_error.argtypes = [vp]
    L.slbm_ws_last_error.restype = ctypes.c_char_p
    L.slbm_ws_destroy.argtypes = [vp]
    L.slbm_ws_destroy.restype = None
    for name in ("slbm_init_fields_device", "slbm_batch_init_fields_device", "slbm_conv3x3_forward",
                 "slbm_conv3x3_flip_weights", "slbm_conv3x3_input_grad", "slbm_conv3x3_weight_grad",
                 "slbm_conv_error", "slbm_ws_create", "slbm_ws_get_params", "slbm_ws_set_params",
                 "slbm_ws_forward", "slbm_ws_loss_grad", "slbm_ws_adam", "slbm_ws_train_step",
                 "slbm_ws_batch_targets", "slbm_ws_warm_start"):
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


def workspace_bytes(params):
    """slbm_workspace_bytes: device bytes a domain with these parameters needs (current device)."""
    return int(lib.slbm_workspace_bytes(ctypes.byref(params)))


class Domain:
    """One simulation domain living on the current CUDA device.

    workspace: optional caller-owned device memory (a CUDA tensor, or an (address, bytes)
    pair) that all of the domain's device buffers are carved from (slbm_create_domain_ext);
    the caller keeps it alive for the domain's lifetime."""

    def __init__(self, params, stream=None, workspace=None):
        self._h = ctypes.c_void_p()
        self.nx, self.ny = params.nx, params.ny
        if workspace is None:
            st = lib.slbm_create_domain(ctypes.byref(params), _stream_handle(stream), ctypes.byref(self._h))
        else:
            if hasattr(workspace, "data_ptr"):
                addr, nbytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
            else:
                addr, nbytes = workspace
            st = lib.slbm_create_domain_ext(ctypes.byref(params), ctypes.c_void_p(int(addr)), ctypes.c_size_t(nbytes),
                                            _stream_handle(stream), ctypes.byref(self._h))
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_last_error(None).decode())
        self.params = params
        self._workspace = workspace

    def set_mms(self, **kw):
        """slbm_set_mms with the test's physical parameters (None switches it off)."""
        if not kw:
            self._check(lib.slbm_set_mms(self._h, None))
            return
        m = MMS(**kw)
        self._check(lib.slbm_set_mms(self._h, ctypes.byref(m)))

    def save(self, path):
        self._check(lib.slbm_save(self._h, os.fsencode(path)))

    def load(self, path):
        self._check(lib.slbm_load(self._h, os.fsencode(path)))

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


def device_allocations():
    """slbm_device_allocations: device allocations the library has made in this process."""
    return int(lib.slbm_device_allocations())


class Domain3D:
    """A three-dimensional domain (D3Q19, include/surflbm3d.h) on the current CUDA device:
    nx x ny x nz nodes, x and z periodic, walls below y = 0 and above y = ny - 1; fields are
    numpy arrays of shape (nz, ny, nx)."""

    def __init__(self, params, nz, stream=None):
        self._h = ctypes.c_void_p()
        self.nx, self.ny, self.nz = params.nx, params.ny, int(nz)
        st = lib.slbm3d_create_domain(ctypes.byref(params), int(nz), _stream_handle(stream), ctypes.byref(self._h))
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm3d_last_error(None).decode())
        self.params = params

    def _check(self, st):
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm3d_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def set_wall(self, wall, theta0_deg=90.0, beta_sg=0.0, beta_sl=0.0, u_x=0.0):
        self._check(lib.slbm3d_set_walls(self._h, int(wall), float(theta0_deg), float(beta_sg), float(beta_sl),
                                         float(u_x)))

    def init_fields(self, phi, psi=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if phi.shape != self.shape:
            raise ValueError("phi must have shape (nz, ny, nx)")
        if psi is not None:
            psi = np.ascontiguousarray(psi, dtype=np.float64)
            if psi.shape != self.shape:
                raise ValueError("psi must have shape (nz, ny, nx)")
        self._check(lib.slbm3d_init_fields(self._h, _dptr(phi), _dptr(psi)))

    def step(self, n=1):
        self._check(lib.slbm3d_step(self._h, int(n)))

    def read_fields(self, which=("phi", "psi", "ux", "uy", "uz", "p")):
        out = {k: np.empty(self.shape, dtype=np.float64) for k in which}
        ptrs = [_dptr(out.get(k)) for k in ("phi", "psi", "ux", "uy", "uz", "p")]
        self._check(lib.slbm3d_read_fields(self._h, *ptrs))
        return out

    def read_totals(self, check=True):
        t = Totals()
        st = lib.slbm3d_read_totals(self._h, ctypes.byref(t))
        if check:
            self._check(st)
        return {name: getattr(t, name) for name, _ in Totals._fields_}

    @property
    def device_bytes(self):
        return int(lib.slbm3d_device_bytes(self._h))

    def close(self):
        if self._h:
            lib.slbm3d_destroy(self._h)
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


class Batch:
    """Many domains stepped together by the batch tile-queue kernel (see slbm_create_batch)."""

    def __init__(self, params_list, walls=None, stream=None):
        n = len(params_list)
        self.count = n
        self.dims = [(p.ny, p.nx) for p in params_list]
        P = (Params * n)(*params_list)
        W = None
        if walls is not None:
            flat = []
            for (bottom, top) in walls:
                flat += [WallSpec(*bottom), WallSpec(*top)]
            W = (WallSpec * (2 * n))(*flat)
        self._h = ctypes.c_void_p()
        st = lib.slbm_create_batch(P, W, n, _stream_handle(stream), ctypes.byref(self._h))
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_batch_last_error(None).decode())

    def _check(self, st):
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_batch_last_error(self._h).decode())

    def init_fields(self, idx, phi, psi=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if phi.shape != self.dims[idx]:
            raise ValueError("phi must have shape (ny, nx) of the instance")
        psi = None if psi is None else np.ascontiguousarray(psi, dtype=np.float64)
        self._check(lib.slbm_batch_init_fields(self._h, int(idx), _dptr(phi), _dptr(psi)))

    def set_tiling(self, band_rows=64, ctas_per_sm=2, graph_steps=32):
        self._check(lib.slbm_batch_set_tiling(self._h, int(band_rows), int(ctas_per_sm), int(graph_steps)))

    def set_strip_width(self, width):
        self._check(lib.slbm_batch_set_strip_width(self._h, int(width)))

    def tiling(self):
        """(strip width, band rows, resident CTAs per SM) of the tile queue."""
        w, br, cs = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib.slbm_batch_get_tiling(self._h, ctypes.byref(w), ctypes.byref(br), ctypes.byref(cs)))
        return w.value, br.value, cs.value

    def autotune(self, cache_path=None):
        br, cs = ctypes.c_int(), ctypes.c_int()
        self._check(lib.slbm_batch_autotune(self._h, cache_path.encode() if cache_path else None,
                                            ctypes.byref(br), ctypes.byref(cs)))
        return br.value, cs.value

    def step(self, n=1):
        self._check(lib.slbm_batch_step(self._h, int(n)))

    def step_instance(self, idx, n=1):
        self._check(lib.slbm_batch_step_instance(self._h, int(idx), int(n)))

    def run_to_equilibrium(self, tol, max_steps, check_every=100):
        out = (ctypes.c_longlong * self.count)()
        self._check(lib.slbm_batch_run_to_equilibrium(self._h, float(tol), int(max_steps), int(check_every), out))
        return np.array(out[:], dtype=np.int64)

    def read_fields(self, idx, which=("phi", "psi", "ux", "uy", "p")):
        ny, nx = self.dims[idx]
        out = {k: np.empty((ny, nx), dtype=np.float64) for k in which}
        ptrs = [_dptr(out.get(k)) for k in ("phi", "psi", "ux", "uy", "p")]
        self._check(lib.slbm_batch_read_fields(self._h, int(idx), *ptrs))
        return out

    def read_totals(self, idx, check=True):
        t = Totals()
        st = lib.slbm_batch_read_totals(self._h, int(idx), ctypes.byref(t))
        if check:
            self._check(st)
        return {name: getattr(t, name) for name, _ in Totals._fields_}

    def active(self):
        flags = (ctypes.c_int * self.count)()
        lib.slbm_batch_active(self._h, flags)
        return np.array(flags[:], dtype=bool)

    def close(self):
        if self._h:
            lib.slbm_batch_destroy(self._h)
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


# ---------------------------------------------------------------- warm start
def _ptr(t):
    """Device pointer of a torch tensor (or an int / None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _prim(st, what):
    if st != SLBM_OK:
        raise SlbmError(st, what)


def conv3x3_forward(x, w, bias, y, relu=True, stream=None):
    """y = act(conv3x3(x, w) + bias) on the tensor cores; x [B,H,W,Cin], w [Cout,3,3,Cin],
    y [B,H,W,Cout] BF16 CUDA tensors, bias FP32 [Cout] or None."""
    B, H, W, Cin = x.shape
    _prim(lib.slbm_conv3x3_forward(_ptr(x), _ptr(w), _ptr(bias), _ptr(y), B, H, W, Cin, w.shape[0], int(relu),
                                   _stream_handle(stream)), "conv3x3_forward")


def conv3x3_flip_weights(w, wt, stream=None):
    Cout, _, _, Cin = w.shape
    _prim(lib.slbm_conv3x3_flip_weights(_ptr(w), _ptr(wt), Cin, Cout, _stream_handle(stream)), "flip_weights")


def conv3x3_input_grad(dy, wt, mask, dx, stream=None):
    """dx = (conv^T dy) * [mask > 0]; wt [Cin,3,3,Cout] from conv3x3_flip_weights."""
    B, H, W, Cout = dy.shape
    _prim(lib.slbm_conv3x3_input_grad(_ptr(dy), _ptr(wt), _ptr(mask), _ptr(dx), B, H, W, wt.shape[0], Cout,
                                      _stream_handle(stream)), "conv3x3_input_grad")


def conv3x3_weight_grad(x, dy, dw, stream=None):
    """dw [Cout,3,3,Cin] (FP32) += d sum(dy * conv(x, w)) / dw."""
    B, H, W, Cin = x.shape
    _prim(lib.slbm_conv3x3_weight_grad(_ptr(x), _ptr(dy), _ptr(dw), B, H, W, Cin, dy.shape[3],
                                       _stream_handle(stream)), "conv3x3_weight_grad")


def conv_error():
    """Synchronises; returns and clears the primitives' tensor-core timeout flag."""
    f = ctypes.c_int()
    _prim(lib.slbm_conv_error(ctypes.byref(f)), "conv_error")
    return f.value


class WarmStartNet:
    """The warm-start encoder-decoder (see include/surflbm_ws.h)."""

    def __init__(self, ny, nx, max_batch, seed=1, stream=None):
        self.ny, self.nx, self.max_batch = ny, nx, max_batch
        self._h = ctypes.c_void_p()
        st = lib.slbm_ws_create(int(ny), int(nx), int(max_batch), int(seed), _stream_handle(stream),
                                ctypes.byref(self._h))
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_ws_last_error(None).decode())
        self.nparam = lib.slbm_ws_param_count(self._h)

    def _check(self, st):
        if st != SLBM_OK:
            raise SlbmError(st, lib.slbm_ws_last_error(self._h).decode())

    def get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(lib.slbm_ws_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.nparam:
            raise ValueError("parameter count mismatch")
        self._check(lib.slbm_ws_set_params(self._h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def forward(self, cond, out):
        """cond: CUDA float32 [B, 5]; out: CUDA float32 [B, 2, ny, nx]."""
        self._check(lib.slbm_ws_forward(self._h, _ptr(cond), int(cond.shape[0]), _ptr(out)))

    def loss_grad(self, cond, targets, idx=None, batch=None, want_grad=True):
        """Loss (and host FP32 gradient) of rows idx (CUDA int32) or 0..batch-1."""
        B = int(idx.shape[0]) if idx is not None else int(batch if batch is not None else cond.shape[0])
        loss = ctypes.c_double()
        g = np.empty(self.nparam, dtype=np.float32) if want_grad else None
        self._check(lib.slbm_ws_loss_grad(self._h, _ptr(cond), _ptr(targets), _ptr(idx), B, ctypes.byref(loss),
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None))
        return loss.value, g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(lib.slbm_ws_adam(self._h, lr, beta1, beta2, eps))

    def train_step(self, cond, targets, idx, lr):
        loss = ctypes.c_double()
        self._check(lib.slbm_ws_train_step(self._h, _ptr(cond), _ptr(targets), _ptr(idx), int(idx.shape[0]),
                                           float(lr), ctypes.byref(loss)))
        return loss.value

    def batch_targets(self, batch, idx, psi0, out):
        """out (CUDA float32 [2, ny, nx]) = (phi, ln(psi/psi0)) of batch instance idx."""
        self._check(lib.slbm_ws_batch_targets(self._h, batch._h, int(idx), float(psi0), _ptr(out)))

    def warm_start(self, batch, which, cond):
        """Replace the cold starts of batch instances `which` by projected predictions;
        returns the accepted flags."""
        which = np.ascontiguousarray(which, dtype=np.int32)
        cond = np.ascontiguousarray(cond, dtype=np.float32)
        acc = np.zeros(len(which), dtype=np.int32)
        self._check(lib.slbm_ws_warm_start(self._h, batch._h, which.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                           cond.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(which),
                                           acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return acc.astype(bool)

    def device_bytes(self):
        return lib.slbm_ws_device_bytes(self._h)

    def close(self):
        if self._h:
            lib.slbm_ws_destroy(self._h)
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
