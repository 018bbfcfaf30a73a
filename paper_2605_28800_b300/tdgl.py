"""Python binding of libtdgl (include/tdgl.h): argument marshalling only.

Every computation runs in the CUDA kernels of libtdgl.so; this module converts numpy arrays or
torch CUDA tensors to pointers and raises on error codes.  There is no CPU fallback: importing
works without a GPU, but creating a Context needs the built library and a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdgl.so")

OK, EINVAL, ENOMEM, ECUDA, EDIVERGED, ENOTCONVERGED, ESTATE, ETOOBIG, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8
RELAX_CONVERGED, RELAX_AT_CAP, RELAX_DIVERGED, RELAX_TIMEOUT = 0, 1, 2, 3   # tdgl_batch_relax_state
HOST, DEVICE = 0, 1
TERM_LANDAU, TERM_GRAD, TERM_ELEC, TERM_EXT, TERM_ALL = 1, 2, 4, 8, 15
K_STEP, K_YFWD, K_ZCONV, K_YINV, K_XFWD, K_OTHER, K_UNET = range(7)
KERNEL_NAMES = {K_STEP: "k_rows<STEP>", K_YFWD: "k_yfwd", K_ZCONV: "k_zconv", K_YINV: "k_yinv",
                K_XFWD: "k_rows<XFWD>", K_OTHER: "other", K_UNET: "unet"}
MAX_MATERIALS, MAX_DIM = 16, 1024
EULER, HEUN, RK45, AB3M2 = 0, 1, 2, 3
ZPASS_VARIANTS = 4
ROW_CANDIDATES = 4

_CODES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EDIVERGED: "EDIVERGED",
          ENOTCONVERGED: "ENOTCONVERGED", ESTATE: "ESTATE", ETOOBIG: "ETOOBIG"}
STATIC_SCRATCH_BYTES = 16 << 20


class TdglError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class Material(ctypes.Structure):
    _fields_ = [("a1_form", ctypes.c_int)] + [(n, ctypes.c_double) for n in (
        "a0", "T0", "coth_A", "coth_Ts", "coth_T1", "a11_0", "a11_T", "a11_Tref", "a12",
        "a111_0", "a111_T", "a111_Tref", "a112", "a123", "G11", "G12", "G44", "G44p", "r_s")]


class Energies(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("land", "grad", "elec", "ext", "total")]


_lib = None
_VP, _D, _I, _U, _L = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_long

_SIGS = {
    "tdgl_ctx_create": (_I, [ctypes.POINTER(_VP), _I, _VP]),
    "tdgl_ctx_destroy": (None, [_VP]),
    "tdgl_last_error": (ctypes.c_char_p, [_VP]),
    "tdgl_launch_count": (_L, [_VP]),
    "tdgl_sim_create": (_I, [_VP, _I, _I, _I, _D, _D, _D, ctypes.POINTER(_VP)]),
    "tdgl_sim_destroy": (None, [_VP]),
    "tdgl_material_define": (_I, [_VP, _I, ctypes.POINTER(Material)]),
    "tdgl_set_material_map": (_I, [_VP, _VP, _I]),
    "tdgl_set_layers": (_I, [_VP, _I, _VP, _VP, _VP]),
    "tdgl_set_eps_b": (_I, [_VP, _D]),
    "tdgl_set_terms": (_I, [_VP, _U]),
    "tdgl_set_temperature": (_I, [_VP, _D]),
    "tdgl_set_field": (_I, [_VP, _D, _D, _D]),
    "tdgl_set_field_ac": (_I, [_VP, _D, _D, _D, _D, _D]),
    "tdgl_set_integrator": (_I, [_VP, _I]),
    "tdgl_set_adaptive": (_I, [_VP, _D, _D, _D]),
    "tdgl_get_dt": (_I, [_VP, ctypes.POINTER(_D)]),
    "tdgl_zpass_variant": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "tdgl_row_tile": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "tdgl_set_row_tile": (_I, [_VP, _I]),
    "tdgl_fft_pad": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "tdgl_set_fft_pad": (_I, [_VP, _I, _I, _I]),
    "tdgl_fp32_fma_peak": (_I, [_VP, ctypes.POINTER(_D)]),
    "tdgl_wait_probe": (_I, [_VP, _L]),
    "tdgl_set_zpass_variant": (_I, [_VP, _I, _I]),
    "tdgl_set_time": (_I, [_VP, _D]),
    "tdgl_get_time": (_I, [_VP, ctypes.POINTER(_D)]),
    "tdgl_set_scales": (_I, [_VP, _D, _D]),
    "tdgl_get_scales": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "tdgl_set_P": (_I, [_VP, _VP, _I]),
    "tdgl_get_P": (_I, [_VP, _VP, _I]),
    "tdgl_set_P_async": (_I, [_VP, _VP]),
    "tdgl_get_P_async": (_I, [_VP, _VP]),
    "tdgl_step_async": (_I, [_VP, _I, _D]),
    "tdgl_sync": (_I, [_VP]),
    "tdgl_init_random": (_I, [_VP, ctypes.c_uint64, _D]),
    "tdgl_get_field": (_I, [_VP, _U, _VP, _I]),
    "tdgl_step": (_I, [_VP, _I, _D]),
    "tdgl_last_max_dP": (_I, [_VP, ctypes.POINTER(_D)]),
    "tdgl_relax": (_I, [_VP, _D, _D, _L, _I, ctypes.POINTER(_L)]),
    "tdgl_energy": (_I, [_VP, ctypes.POINTER(Energies)]),
    "tdgl_batch_create": (_I, [_VP, _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "tdgl_batch_destroy": (None, [_VP]),
    "tdgl_batch_step": (_I, [_VP, _I, ctypes.POINTER(_D)]),
    "tdgl_batch_relax": (_I, [_VP, ctypes.POINTER(_D), _D, _L, _I, ctypes.POINTER(_L)]),
    "tdgl_batch_relax_state": (_I, [_VP, ctypes.POINTER(_D), _D, _L, _I, ctypes.POINTER(_L), ctypes.POINTER(_I)]),
    "tdgl_elec_field_static": (_I, [_I, _I, _I, _D, _D, _D, _D, _VP, _VP, _VP, _VP]),
    "tdgl_unet_create": (_I, [_VP, _I, _I, _I, _VP, _I, _I, _I, _I, ctypes.c_uint64, ctypes.POINTER(_VP)]),
    "tdgl_unet_destroy": (None, [_VP]),
    "tdgl_unet_param_count": (_L, [_VP]),
    "tdgl_unet_set_params": (_I, [_VP, _VP]),
    "tdgl_unet_get_params": (_I, [_VP, _VP]),
    "tdgl_unet_forward": (_I, [_VP, _VP, _VP, _I, _I]),
    "tdgl_unet_loss_grad": (_I, [_VP, _VP, _VP, _I, ctypes.POINTER(_D), _VP, _I]),
    "tdgl_unet_train_step": (_I, [_VP, _VP, _VP, _I, _D, ctypes.POINTER(_D), _I]),
    "tdgl_conv3d": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _I, _I]),
    "tdgl_conv3d_backward": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _I]),
    "tdgl_profile": (_I, [_VP, _I]),
    "tdgl_profile_read": (_I, [_VP, _I, ctypes.POINTER(_D), ctypes.POINTER(_L)]),
}

EXPORTED = tuple(_SIGS)


def library(path: str = LIB_PATH):
    """Load libtdgl.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"{path} not built; run paper_2605_28800_b300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch tensor (host or CUDA)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), DEVICE if a.is_cuda else HOST
    raise TypeError(f"unsupported buffer type {type(a)}")


def material_struct(rec: dict) -> Material:
    m = Material()
    for name, _ in Material._fields_:
        setattr(m, name, rec.get(name, 1.0 if name == "r_s" else 0))
    return m


class Context:
    def __init__(self, device: int = 0, stream=None):
        self.lib = library()
        h = _VP()
        s = None if stream is None else _VP(int(stream))
        rc = self.lib.tdgl_ctx_create(ctypes.byref(h), device, s)
        if rc != OK:
            raise TdglError(rc, f"tdgl_ctx_create(device={device}) failed")
        self.h = h
        self._children = weakref.WeakSet()

    def _adopt(self, obj):
        self._children.add(obj)

    def last_error(self) -> str:
        """message of the last failed call on this context"""
        return self.lib.tdgl_last_error(self.h).decode()

    def check(self, rc):
        if rc != OK:
            raise TdglError(rc, self.lib.tdgl_last_error(self.h).decode())
        return rc

    def zpass_variant(self, length):
        """(variant, microseconds per launch of each variant, 0 where the length has none) chosen by
        the z-pass autotuner; -1 = not yet tuned"""
        v, us = _I(), (_D * ZPASS_VARIANTS)()
        self.check(self.lib.tdgl_zpass_variant(self.h, int(length), ctypes.byref(v), us))
        return v.value, tuple(us)

    def fp32_fma_peak(self) -> float:
        """measured FP32 fused multiply-add throughput of the device, TFLOP/s"""
        v = _D()
        self.check(self.lib.tdgl_fp32_fma_peak(self.h, ctypes.byref(v)))
        return v.value

    def wait_probe(self, polls: int) -> int:
        """run one bounded mbarrier wait that nothing satisfies (nothing pending) for at most polls
        polls; returns the library's status code (ETIMEOUT expected) without raising"""
        return int(self.lib.tdgl_wait_probe(self.h, int(polls)))

    def set_zpass_variant(self, length, variant):
        self.check(self.lib.tdgl_set_zpass_variant(self.h, int(length), int(variant)))

    @property
    def launch_count(self) -> int:
        return int(self.lib.tdgl_launch_count(self.h))

    def profile(self, enable: bool = True):
        self.check(self.lib.tdgl_profile(self.h, int(enable)))

    def profile_read(self, kind: int):
        ms, n = _D(), _L()
        self.check(self.lib.tdgl_profile_read(self.h, kind, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        """Destroy the context; its batches and sims are closed first (their handles die with it)."""
        if getattr(self, "h", None):
            kids = list(self._children)
            for k in kids:
                if isinstance(k, Batch):
                    k.close()
            for k in kids:
                k.close()
            self.lib.tdgl_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """One finite sample: grid (nx, ny, nz) of (dx, dy, dz)-metre cells."""

    def __init__(self, ctx: Context, shape, cell):
        self.ctx, self.lib = ctx, ctx.lib
        self.shape = tuple(int(v) for v in shape)
        nx, ny, nz = self.shape
        h = _VP()
        ctx.check(self.lib.tdgl_sim_create(ctx.h, nx, ny, nz, *map(float, cell), ctypes.byref(h)))
        self.h = h
        self.ncell = nx * ny * nz
        ctx._adopt(self)

    def _c(self, rc):
        return self.ctx.check(rc)

    def define_material(self, mid: int, rec: dict):
        m = material_struct(rec)
        self._c(self.lib.tdgl_material_define(self.h, mid, ctypes.byref(m)))

    def set_material_map(self, ids):
        if isinstance(ids, np.ndarray):
            ids = np.ascontiguousarray(ids, dtype=np.uint8)
        p, where = _ptr(ids)
        self._c(self.lib.tdgl_set_material_map(self.h, p, where))

    def set_layers(self, layers):
        z0 = np.array([l[0] for l in layers], np.int32)
        z1 = np.array([l[1] for l in layers], np.int32)
        ids = np.array([l[2] for l in layers], np.int32)
        self._c(self.lib.tdgl_set_layers(self.h, len(layers), z0.ctypes.data, z1.ctypes.data, ids.ctypes.data))

    def set_eps_b(self, v): self._c(self.lib.tdgl_set_eps_b(self.h, float(v)))
    def set_terms(self, mask): self._c(self.lib.tdgl_set_terms(self.h, int(mask)))
    def set_temperature(self, T): self._c(self.lib.tdgl_set_temperature(self.h, float(T)))
    def set_field(self, E): self._c(self.lib.tdgl_set_field(self.h, *map(float, E)))
    def set_scales(self, P0, alpha_ref): self._c(self.lib.tdgl_set_scales(self.h, float(P0), float(alpha_ref)))

    def set_field_ac(self, A, freq_hz, phase=0.0):
        self._c(self.lib.tdgl_set_field_ac(self.h, *map(float, A), float(freq_hz), float(phase)))

    def set_time(self, t): self._c(self.lib.tdgl_set_time(self.h, float(t)))

    def set_integrator(self, method): self._c(self.lib.tdgl_set_integrator(self.h, int(method)))

    def set_adaptive(self, err_tol, dt_min=0.0, dt_max=0.0):
        """RK45 step-size control (err_tol = 0: fixed steps); see tdgl_set_adaptive."""
        self._c(self.lib.tdgl_set_adaptive(self.h, float(err_tol), float(dt_min), float(dt_max)))

    def dt_next(self):
        v = _D()
        self._c(self.lib.tdgl_get_dt(self.h, ctypes.byref(v)))
        return v.value

    def time(self):
        v = _D()
        self._c(self.lib.tdgl_get_time(self.h, ctypes.byref(v)))
        return v.value

    def scales(self):
        a, b = _D(), _D()
        self._c(self.lib.tdgl_get_scales(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_P(self, P):
        if isinstance(P, np.ndarray):
            P = np.ascontiguousarray(P, dtype=np.float32)
        if (P.numel() if hasattr(P, "numel") else P.size) != 3 * self.ncell:
            raise ValueError("P must have 3*nx*ny*nz elements")
        p, where = _ptr(P)
        self._c(self.lib.tdgl_set_P(self.h, p, where))

    def get_P(self, out=None):
        nx, ny, nz = self.shape
        if out is None:
            out = np.empty((3, nz, ny, nx), np.float32)
        p, where = _ptr(out)
        self._c(self.lib.tdgl_get_P(self.h, p, where))
        return out

    def _host_ptr(self, a):
        p, where = _ptr(a)
        if where != HOST:
            raise ValueError("the asynchronous I/O calls take host buffers")
        if (a.numel() if hasattr(a, "numel") else a.size) != 3 * self.ncell:
            raise ValueError("P must have 3*nx*ny*nz elements")
        if (a.dtype != np.float32) if isinstance(a, np.ndarray) else (str(a.dtype) != "torch.float32"):
            raise ValueError("P must be float32")
        return p

    def set_P_async(self, P):
        """Queue the upload of P (host, float32, page-locked to overlap); P must not change until sync()."""
        self._c(self.lib.tdgl_set_P_async(self.h, self._host_ptr(P)))

    def step_async(self, n: int, dt: float):
        """Queue n steps without reading their status (sync() reports it)."""
        self._c(self.lib.tdgl_step_async(self.h, int(n), float(dt)))

    def get_P_async(self, out):
        """Queue the download of the current P into out (host, float32); read it after sync()."""
        self._c(self.lib.tdgl_get_P_async(self.h, self._host_ptr(out)))

    def sync(self):
        """Wait for the queued uploads, steps and downloads; raises on divergence or a timeout."""
        self._c(self.lib.tdgl_sync(self.h))

    def init_random(self, seed: int, amp: float):
        self._c(self.lib.tdgl_init_random(self.h, ctypes.c_uint64(seed), float(amp)))

    def get_field(self, mask=TERM_ALL, out=None):
        nx, ny, nz = self.shape
        if out is None:
            out = np.empty((3, nz, ny, nx), np.float32)
        p, where = _ptr(out)
        self._c(self.lib.tdgl_get_field(self.h, int(mask), p, where))
        return out

    def step(self, n: int, dt: float):
        self._c(self.lib.tdgl_step(self.h, int(n), float(dt)))

    def row_tile(self):
        """(rows per block chosen by the row-tile autotuner, 0 = not tuned, and the list of
        (candidate, microseconds per launch) it timed)"""
        r, c, us = _I(), (_I * ROW_CANDIDATES)(), (_D * ROW_CANDIDATES)()
        self._c(self.lib.tdgl_row_tile(self.h, ctypes.byref(r), c, us))
        return r.value, [(int(a), float(b)) for a, b in zip(c, us) if a > 0]

    def fft_pad(self):
        """(Mx, My, Mz): the padded transform lengths of the electrostatic convolution."""
        a, b, c = _I(), _I(), _I()
        self._c(self.lib.tdgl_fft_pad(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_fft_pad(self, Mx=0, My=0, Mz=0):
        """Set the padded lengths (0 = the default for that axis)."""
        self._c(self.lib.tdgl_set_fft_pad(self.h, int(Mx), int(My), int(Mz)))

    def set_row_tile(self, rows: int):
        """Force rows per block of the step kernel (0: back to the autotuner)."""
        self._c(self.lib.tdgl_set_row_tile(self.h, int(rows)))

    def last_max_dP(self) -> float:
        v = _D()
        self._c(self.lib.tdgl_last_max_dP(self.h, ctypes.byref(v)))
        return v.value

    def relax(self, dt, tol, max_steps, check_every=16, raise_on_cap=True):
        n = _L()
        rc = self.lib.tdgl_relax(self.h, float(dt), float(tol), int(max_steps), int(check_every), ctypes.byref(n))
        if rc == ENOTCONVERGED and not raise_on_cap:
            return n.value, False
        self._c(rc)
        return n.value, True

    def energy(self) -> dict:
        e = Energies()
        self._c(self.lib.tdgl_energy(self.h, ctypes.byref(e)))
        return {k: getattr(e, k) for k, _ in Energies._fields_}

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None):      # a destroyed context already freed its sims
                self.lib.tdgl_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent sims of one context stepped with one launch per kernel."""

    def __init__(self, ctx: Context, sims):
        self.ctx, self.lib, self.sims = ctx, ctx.lib, list(sims)
        arr = (_VP * len(self.sims))(*[s.h for s in self.sims])
        h = _VP()
        ctx.check(self.lib.tdgl_batch_create(ctx.h, len(self.sims), arr, ctypes.byref(h)))
        self.h = h
        ctx._adopt(self)

    def _dts(self, dt):
        dts = [float(dt)] * len(self.sims) if np.isscalar(dt) else [float(v) for v in dt]
        return (_D * len(self.sims))(*dts)

    def step(self, n, dt):
        self.ctx.check(self.lib.tdgl_batch_step(self.h, int(n), self._dts(dt)))

    def relax(self, dt, tol, max_steps, check_every=16, raise_on_cap=True):
        steps = (_L * len(self.sims))()
        rc = self.lib.tdgl_batch_relax(self.h, self._dts(dt), float(tol), int(max_steps), int(check_every), steps)
        if not (rc == ENOTCONVERGED and not raise_on_cap):
            self.ctx.check(rc)
        return [int(v) for v in steps], rc == OK

    def relax_state(self, dt, tol, max_steps, check_every=16):
        """relax that reports how each sim ended: (steps taken, states), a state per sim one of
        RELAX_CONVERGED, RELAX_AT_CAP, RELAX_DIVERGED, RELAX_TIMEOUT.  Raises only for errors that
        are not a sim's own outcome."""
        steps = (_L * len(self.sims))()
        state = (_I * len(self.sims))()
        rc = self.lib.tdgl_batch_relax_state(self.h, self._dts(dt), float(tol), int(max_steps), int(check_every),
                                             steps, state)
        if rc not in (OK, ENOTCONVERGED, EDIVERGED, ETIMEOUT):
            self.ctx.check(rc)
        return [int(v) for v in steps], [int(v) for v in state]

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None):
                self.lib.tdgl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def elec_field_static(P, E, cell, eps_b, mat=None, stream=0):
    """Open-boundary field E_el of P without any device allocation (tdgl_elec_field_static).

    For callers that cannot allocate device memory (inside stream capture, host-owned memory
    pools, real-time loops).  P and E are contiguous CUDA tensors of shape (3, nz, ny, nx)
    (float32, C/m^2 in, V/m out); mat an optional uint8 CUDA tensor (nz, ny, nx).  Work is
    enqueued on `stream` (a cudaStream_t as int; 0 = legacy default stream).  Every call shares
    one fixed static scratch array: calls that overlap on the GPU race.
    """
    lib = library()
    _, nz, ny, nx = P.shape
    for t in (P, E) + (() if mat is None else (mat,)):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("P, E and mat must be contiguous CUDA tensors")
    rc = lib.tdgl_elec_field_static(nx, ny, nz, float(cell[0]), float(cell[1]), float(cell[2]), float(eps_b),
                                    P.data_ptr(), None if mat is None else mat.data_ptr(), E.data_ptr(),
                                    None if not stream else _VP(int(stream)))
    if rc != OK:
        raise TdglError(rc, "tdgl_elec_field_static failed")


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} values, got {a.size}")
    return a


class UNet:
    """The learned warm start (tdgl_unet_*): a 3D U-Net trained and run on the tensor cores.

    Tensors are (batch, channels, nz, ny, nx) float32: numpy arrays (host) or contiguous CUDA
    torch tensors (device; inputs and outputs must then all be on the device).  Parameters are one
    flat float32 vector in the layer order of the library (see include/tdgl.h).
    """

    def __init__(self, ctx: Context, shape, cin, cout, chans=(16, 32, 64, 128), max_batch=4, seed=0):
        self.ctx, self.lib = ctx, ctx.lib
        self.nx, self.ny, self.nz = (int(v) for v in shape)
        self.cin, self.cout, self.levels = int(cin), int(cout), len(chans)
        ch = (ctypes.c_int * len(chans))(*chans)
        h = _VP()
        ctx.check(self.lib.tdgl_unet_create(ctx.h, self.cin, self.cout, self.levels, ch, self.nx, self.ny, self.nz,
                                            int(max_batch), int(seed), ctypes.byref(h)))
        self.h = h
        ctx._adopt(self)

    @property
    def nvox(self):
        return self.nx * self.ny * self.nz

    def param_count(self):
        return int(self.lib.tdgl_unet_param_count(self.h))

    def set_params(self, p):
        p = _f32(p, (self.param_count(),))
        self.ctx.check(self.lib.tdgl_unet_set_params(self.h, p.ctypes.data))

    def get_params(self):
        p = np.empty(self.param_count(), dtype=np.float32)
        self.ctx.check(self.lib.tdgl_unet_get_params(self.h, p.ctypes.data))
        return p

    def _io(self, x, c):
        if isinstance(x, np.ndarray):
            x = _f32(x)
            if x.size % (c * self.nvox):
                raise ValueError("tensor size is not a multiple of channels x cells")
            return x, x.ctypes.data, HOST, x.size // (c * self.nvox)
        ptr, where = _ptr(x)
        return x, ptr, where, x.numel() // (c * self.nvox)

    def forward(self, x):
        x, px, where, B = self._io(x, self.cin)
        if where == HOST:
            y = np.empty((B, self.cout, self.nz, self.ny, self.nx), dtype=np.float32)
            py = y.ctypes.data
        else:
            import torch
            y = torch.empty((B, self.cout, self.nz, self.ny, self.nx), dtype=torch.float32, device=x.device)
            py = y.data_ptr()
        self.ctx.check(self.lib.tdgl_unet_forward(self.h, px, py, B, where))
        return y

    def loss_grad(self, x, t):
        x, px, where, B = self._io(x, self.cin)
        t, pt, _, _ = self._io(t, self.cout)
        g = np.empty(self.param_count(), dtype=np.float32)
        loss = _D()
        self.ctx.check(self.lib.tdgl_unet_loss_grad(self.h, px, pt, B, ctypes.byref(loss), g.ctypes.data, where))
        return loss.value, g

    def train_step(self, x, t, lr):
        x, px, where, B = self._io(x, self.cin)
        t, pt, _, _ = self._io(t, self.cout)
        loss = _D()
        self.ctx.check(self.lib.tdgl_unet_train_step(self.h, px, pt, B, float(lr), ctypes.byref(loss), where))
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            if getattr(self.ctx, "h", None):
                self.lib.tdgl_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def conv3d(ctx: Context, x, w, b, relu=False):
    """One tensor-core convolution (tdgl_conv3d): x (B, ci, nz, ny, nx), w (co, ci, k, k, k), b (co,)."""
    x, w, b = _f32(x), _f32(w), _f32(b)
    B, ci, nz, ny, nx = x.shape
    co, k = w.shape[0], w.shape[-1]
    y = np.empty((B, co, nz, ny, nx), dtype=np.float32)
    ctx.check(ctx.lib.tdgl_conv3d(ctx.h, x.ctypes.data, w.ctypes.data, b.ctypes.data, y.ctypes.data, B, ci, co, k, nx,
                                  ny, nz, int(relu)))
    return y


def conv3d_backward(ctx: Context, x, w, dy):
    """Gradients (dx, dw, db) of one convolution for upstream gradient dy (tdgl_conv3d_backward)."""
    x, w, dy = _f32(x), _f32(w), _f32(dy)
    B, ci, nz, ny, nx = x.shape
    co, k = w.shape[0], w.shape[-1]
    dx = np.empty_like(x)
    dw = np.empty_like(w)
    db = np.empty(co, dtype=np.float32)
    ctx.check(ctx.lib.tdgl_conv3d_backward(ctx.h, x.ctypes.data, w.ctypes.data, dy.ctypes.data, dx.ctypes.data,
                                           dw.ctypes.data, db.ctypes.data, B, ci, co, k, nx, ny, nz))
    return dx, dw, db
