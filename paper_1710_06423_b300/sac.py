"""ctypes binding of ``libsac.so`` (include/sac.h): argument marshalling only.

Every step of the MHD path runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  There is no CPU fallback: if the library is missing the import
of the solver fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsac.so")

SAC_OK, SAC_ERR_ARG, SAC_ERR_STATE, SAC_ERR_CUDA, SAC_ERR_OOM, SAC_ERR_NONFINITE, SAC_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
SAC_ERR_TOO_LARGE = -7
BC_PERIODIC, BC_FIXED, BC_OUTFLOW = 0, 1, 2
TILE_32x32, TILE_64x16, TILE_32x16 = 0, 1, 2
TILE_KERNEL_GHOSTS = 3   # + shape: the stage kernel writes the ghost frame itself (single runs)
TILE_NAMES = {TILE_32x32: "32x32", TILE_64x16: "64x16", TILE_32x16: "32x16"}
TILE_NAMES.update({TILE_KERNEL_GHOSTS + t: f"{n}, in-kernel ghosts" for t, n in list(TILE_NAMES.items())})
FP64, FP32 = 0, 1
NF, NB = 6, 4

#: every function the C header declares, in header order
EXPORTS = (
    "sac_default_params", "sac_init", "sac_free", "sac_last_error", "sac_status_string",
    "sac_set_state", "sac_get_state", "sac_set_state_dev", "sac_get_state_dev",
    "sac_step", "sac_steps", "sac_run_to", "sac_set_fixed_dt", "sac_dt", "sac_time", "sac_cmax", "sac_sums", "sac_divb",
    "sac_profile_stages", "sac_sync", "sac_set_tile", "sac_get_tile", "sac_tune",
    "sac_set_cell_size", "sac_stage", "sac_halo_size", "sac_halo_pack", "sac_halo_unpack", "sac_get_cmax_bits", "sac_set_cmax_bits",
    "sac_debug_drop_copies",
    "sac_batch_init", "sac_batch_free", "sac_batch_last_error", "sac_batch_set_state",
    "sac_batch_get_state", "sac_batch_steps", "sac_batch_sync", "sac_batch_time", "sac_batch_tune",
    "sac_batch_set_config", "sac_batch_set_tile", "sac_batch_get_config",
    "sac_cnn_param_count", "sac_cnn_init", "sac_cnn_free", "sac_cnn_last_error", "sac_cnn_set_tensor_path",
    "sac_cnn_set_limiter", "sac_cnn_sync", "sac_cnn_set_params",
    "sac_cnn_get_params", "sac_cnn_set_scales", "sac_cnn_forward", "sac_cnn_grads", "sac_cnn_train_step",
    "sac_cnn_apply", "sac_cnn_perturb", "sac_block_average",
    "sac_step_noalloc",
    "sac3_default_params", "sac3_init", "sac3_free", "sac3_last_error", "sac3_set_state", "sac3_get_state",
    "sac3_step", "sac3_steps", "sac3_run_to", "sac3_time", "sac3_sums", "sac3_divb", "sac3_debug_drop_copies",
)


class SacError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} [{code}]")
        self.code = code


class SacParams(ctypes.Structure):
    """Mirror of ``sac_params``."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("courant", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("hyperdiffusion", ctypes.c_int),
        ("c2", ctypes.c_double * 6),
        ("c_shk", ctypes.c_double),
        ("has_background", ctypes.c_int),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("gravity", ctypes.c_double * 2),
        ("hd_single_face", ctypes.c_int),
    ]


class Sac3Params(ctypes.Structure):
    """Mirror of ``sac3_params`` (include/sac.h)."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("z0", ctypes.c_double), ("z1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("courant", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("hyperdiffusion", ctypes.c_int),
        ("c2", ctypes.c_double * 8),
        ("c_shk", ctypes.c_double),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


_lib = None


def load() -> ctypes.CDLL:
    """Load libsac.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1710_06423_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, i, d, L = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_long
    P = ctypes.POINTER(SacParams)
    P3 = ctypes.POINTER(Sac3Params)
    sig = {
        "sac_default_params": (None, [P]),
        "sac_init": (i, [P, ctypes.POINTER(vp)]),
        "sac_free": (None, [vp]),
        "sac_last_error": (ctypes.c_char_p, [vp]),
        "sac_status_string": (ctypes.c_char_p, [i]),
        "sac_set_state": (i, [vp, dp, dp, d]),
        "sac_get_state": (i, [vp, dp, dp]),
        "sac_set_state_dev": (i, [vp, vp, vp, d]),
        "sac_get_state_dev": (i, [vp, vp, dp]),
        "sac_step": (i, [vp, d, dp]),
        "sac_steps": (i, [vp, L]),
        "sac_run_to": (i, [vp, d, L, ctypes.POINTER(L)]),
        "sac_set_fixed_dt": (i, [vp, d]),
        "sac_dt": (i, [vp, dp]),
        "sac_time": (i, [vp, dp, ctypes.POINTER(L)]),
        "sac_cmax": (i, [vp, dp, dp]),
        "sac_sums": (i, [vp, dp]),
        "sac_divb": (i, [vp, dp, dp, ctypes.POINTER(ctypes.c_longlong)]),
        "sac_profile_stages": (i, [vp, i, dp]),
        "sac_sync": (i, [vp]),
        "sac_set_tile": (i, [vp, i]),
        "sac_get_tile": (i, [vp, ctypes.POINTER(i)]),
        "sac_tune": (i, [vp, i, ctypes.POINTER(i), dp]),
        "sac_set_cell_size": (i, [vp, d, d]),
        "sac_stage": (i, [vp, i]),
        "sac_halo_size": (i, [vp, i, ctypes.POINTER(ctypes.c_longlong)]),
        "sac_halo_pack": (i, [vp, i, vp]),
        "sac_halo_unpack": (i, [vp, i, vp]),
        "sac_get_cmax_bits": (i, [vp, vp]),
        "sac_set_cmax_bits": (i, [vp, vp]),
        "sac_debug_drop_copies": (i, [vp, i]),
        "sac_batch_init": (i, [P, i, ctypes.POINTER(vp)]),
        "sac_batch_free": (None, [vp]),
        "sac_batch_last_error": (ctypes.c_char_p, [vp]),
        "sac_batch_set_state": (i, [vp, i, dp, dp, d]),
        "sac_batch_get_state": (i, [vp, i, dp, dp]),
        "sac_batch_steps": (i, [vp, L]),
        "sac_batch_sync": (i, [vp]),
        "sac_batch_time": (i, [vp, i, dp, ctypes.POINTER(L)]),
        "sac_batch_tune": (i, [vp, i, ctypes.POINTER(ctypes.c_int), dp]),
        "sac_batch_set_config": (i, [vp, i, i, i]),
        "sac_batch_set_tile": (i, [vp, i]),
        "sac_batch_get_config": (i, [vp, ctypes.POINTER(ctypes.c_int)]),
        "sac_cnn_param_count": (L, []),
        "sac_cnn_init": (i, [i, i, i, vp, ctypes.POINTER(vp)]),
        "sac_cnn_free": (None, [vp]),
        "sac_cnn_last_error": (ctypes.c_char_p, [vp]),
        "sac_cnn_set_tensor_path": (i, [vp, i]),
        "sac_cnn_set_limiter": (i, [vp, d, i]),
        "sac_cnn_sync": (i, [vp]),
        "sac_cnn_set_params": (i, [vp, ctypes.POINTER(ctypes.c_float), L]),
        "sac_cnn_get_params": (i, [vp, ctypes.POINTER(ctypes.c_float), L]),
        "sac_cnn_set_scales": (i, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "sac_cnn_forward": (i, [vp, vp, d, d, d, vp]),
        "sac_cnn_grads": (i, [vp, vp, vp, d, d, d, ctypes.POINTER(ctypes.c_float), dp]),
        "sac_cnn_train_step": (i, [vp, vp, vp, d, d, d, d, dp]),
        "sac_cnn_apply": (i, [vp, vp]),
        "sac_cnn_perturb": (i, [vp, vp, vp, ctypes.POINTER(ctypes.c_float), ctypes.c_ulonglong]),
        "sac_block_average": (i, [vp, i, i, i, i, vp, vp]),
        "sac_step_noalloc": (i, [P, vp, vp, d, dp]),
        "sac3_default_params": (None, [P3]),
        "sac3_init": (i, [P3, ctypes.POINTER(vp)]),
        "sac3_free": (None, [vp]),
        "sac3_last_error": (ctypes.c_char_p, [vp]),
        "sac3_set_state": (i, [vp, dp, d]),
        "sac3_get_state": (i, [vp, dp, dp]),
        "sac3_step": (i, [vp, d, dp]),
        "sac3_steps": (i, [vp, L]),
        "sac3_run_to": (i, [vp, d, L, ctypes.POINTER(L)]),
        "sac3_time": (d, [vp]),
        "sac3_sums": (i, [vp, dp]),
        "sac3_divb": (i, [vp, dp, dp]),
        "sac3_debug_drop_copies": (i, [vp, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_params() -> SacParams:
    p = SacParams()
    load().sac_default_params(ctypes.byref(p))
    return p


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_F32, _F64, _I64 = ("torch.float32",), ("torch.float64",), ("torch.int64", "torch.uint64")


def _dev_ptr(t, name: str, numel: int, dtypes, device: int) -> ctypes.c_void_p:
    """Device address of tensor ``t`` for a C call that receives only a bare
    pointer.  The library cannot see how large the buffer is, so a tensor that
    is too small, strided, of another dtype or on another device would be read
    or written past its end on the GPU: refuse it here, before the call."""
    if t.numel() != numel:
        raise ValueError(f"{name} holds {t.numel()} elements, {numel} needed")
    if str(t.dtype) not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}, not {' or '.join(dtypes)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda or t.device.index != device:
        raise ValueError(f"{name} must live on cuda:{device}, not {t.device}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One run on one GPU: ``Solver(nx=..., ny=..., precision=FP32, ...)``.

    Keyword arguments are ``sac_params`` fields; ``stream`` may be a
    ``torch.cuda.Stream`` or a raw handle (default: torch's current stream).
    """

    def __init__(self, **kw):
        lib = load()
        p = default_params()
        stream = kw.pop("stream", "current")
        for k, v in kw.items():
            if k in ("c2", "gravity"):
                fld = getattr(p, k)
                for j, x in enumerate(v):
                    fld[j] = x
            else:
                setattr(p, k, v)
        if stream == "current":
            import torch
            stream = torch.cuda.current_stream(p.device)
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        p.stream = stream or None
        self.params = p
        self._ctx = ctypes.c_void_p()
        rc = lib.sac_init(ctypes.byref(p), ctypes.byref(self._ctx))
        if rc != SAC_OK:
            raise SacError(rc, f"sac_init failed: {lib.sac_status_string(rc).decode()}")
        self.nx, self.ny = p.nx, p.ny
        self.fp32 = p.precision == FP32

    # -- helpers --------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != SAC_OK:
            lib = load()
            raise SacError(rc, f"{what}: {lib.sac_status_string(rc).decode()}: "
                               f"{lib.sac_last_error(self._ctx).decode()}")

    def close(self):
        if self._ctx:
            load().sac_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C ABI ----------------------------------------------------------------
    def set_state(self, w, bg=None, t: float = 0.0):
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (NF, self.ny, self.nx):
            raise ValueError(f"state shape {w.shape} != {(NF, self.ny, self.nx)}")
        if bg is not None:
            bg = np.ascontiguousarray(bg, dtype=np.float64)
            if bg.shape != (NB, self.ny, self.nx):
                raise ValueError(f"background shape {bg.shape} != {(NB, self.ny, self.nx)}")
        self._check(load().sac_set_state(self._ctx, _dp(w), _dp(bg), float(t)), "sac_set_state")

    def get_state(self):
        w = np.empty((NF, self.ny, self.nx), dtype=np.float64)
        t = ctypes.c_double()
        self._check(load().sac_get_state(self._ctx, _dp(w), ctypes.byref(t)), "sac_get_state")
        return w, t.value

    def get_state_into(self, w: np.ndarray) -> float:
        """Copy the state into an existing C-contiguous float64 host array (e.g. pinned)."""
        assert w.dtype == np.float64 and w.flags.c_contiguous and w.size == NF * self.nx * self.ny
        t = ctypes.c_double()
        self._check(load().sac_get_state(self._ctx, _dp(w), ctypes.byref(t)), "sac_get_state")
        return t.value

    def _state_ptr(self, t, name: str, nfields: int = NF) -> ctypes.c_void_p:
        return _dev_ptr(t, name, nfields * self.nx * self.ny, _F32 if self.fp32 else _F64, self.params.device)

    def set_state_dev(self, w, bg=None, t: float = 0.0):
        """Device tensors of the context's dtype, shape (6, ny, nx) / (4, ny, nx), contiguous."""
        wp = self._state_ptr(w, "w")
        bp = None if bg is None else self._state_ptr(bg, "bg", NB)
        self._check(load().sac_set_state_dev(self._ctx, wp, bp, float(t)), "sac_set_state_dev")

    def get_state_dev(self, w) -> None:
        wp = self._state_ptr(w, "w")
        self._check(load().sac_get_state_dev(self._ctx, wp, None), "sac_get_state_dev")

    def step(self, dt: float = 0.0) -> float:
        out = ctypes.c_double()
        self._check(load().sac_step(self._ctx, float(dt), ctypes.byref(out)), "sac_step")
        return out.value

    def steps(self, n: int):
        self._check(load().sac_steps(self._ctx, int(n)), "sac_steps")

    def run_to(self, t_end: float, max_steps: int = -1) -> int:
        n = ctypes.c_long()
        self._check(load().sac_run_to(self._ctx, float(t_end), int(max_steps), ctypes.byref(n)), "sac_run_to")
        return n.value

    def set_fixed_dt(self, dt: float):
        """dt > 0: every later CFL step takes dt; dt <= 0: back to the CFL step."""
        self._check(load().sac_set_fixed_dt(self._ctx, float(dt)), "sac_set_fixed_dt")

    def dt(self) -> float:
        out = ctypes.c_double()
        self._check(load().sac_dt(self._ctx, ctypes.byref(out)), "sac_dt")
        return out.value

    def time(self):
        t, n = ctypes.c_double(), ctypes.c_long()
        self._check(load().sac_time(self._ctx, ctypes.byref(t), ctypes.byref(n)), "sac_time")
        return t.value, n.value

    def cmax(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(load().sac_cmax(self._ctx, ctypes.byref(a), ctypes.byref(b)), "sac_cmax")
        return a.value, b.value

    def sums(self) -> np.ndarray:
        out = np.zeros(6)
        self._check(load().sac_sums(self._ctx, _dp(out)), "sac_sums")
        return out

    def divb(self):
        """(max |div B|, mean |div B|, cells counted) of the total field, FP64."""
        a, m, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        self._check(load().sac_divb(self._ctx, ctypes.byref(a), ctypes.byref(m), ctypes.byref(n)), "sac_divb")
        return a.value, m.value, n.value

    def profile_stages(self, nsteps: int) -> np.ndarray:
        """Mean CUDA-event durations [ms]: step control, stage 1..4 kernels."""
        out = np.zeros(5)
        self._check(load().sac_profile_stages(self._ctx, int(nsteps), _dp(out)), "sac_profile_stages")
        return out

    def sync(self):
        self._check(load().sac_sync(self._ctx), "sac_sync")

    def set_tile(self, tile: int):
        """FP32 tile configuration of the later steps: a shape (TILE_32x32, TILE_64x16,
        TILE_32x16), plus TILE_KERNEL_GHOSTS for the in-kernel ghost frame."""
        self._check(load().sac_set_tile(self._ctx, int(tile)), "sac_set_tile")

    def tile(self) -> int:
        out = ctypes.c_int()
        self._check(load().sac_get_tile(self._ctx, ctypes.byref(out)), "sac_get_tile")
        return out.value

    def tune(self, trials: int = 3):
        """Autotune the tile configuration on the current state (restored); returns (tile, ms per step)."""
        t, ms = ctypes.c_int(), ctypes.c_double()
        self._check(load().sac_tune(self._ctx, int(trials), ctypes.byref(t), ctypes.byref(ms)), "sac_tune")
        return t.value, ms.value

    # -- block decomposition (sac_stage / sac_halo_* / sac_*_cmax_bits) --------
    def set_cell_size(self, dx: float, dy: float):
        self._check(load().sac_set_cell_size(self._ctx, float(dx), float(dy)), "sac_set_cell_size")

    def stage(self, k: int):
        self._check(load().sac_stage(self._ctx, int(k)), "sac_stage")

    def halo_size(self, side: int) -> int:
        n = ctypes.c_longlong()
        self._check(load().sac_halo_size(self._ctx, int(side), ctypes.byref(n)), "sac_halo_size")
        return n.value

    def _strip_ptr(self, side: int, strip) -> ctypes.c_void_p:
        return _dev_ptr(strip, "strip", self.halo_size(side), _F32 if self.fp32 else _F64, self.params.device)

    def halo_pack(self, side: int, strip):
        """Pack the strip next to `side` into a device tensor of halo_size(side) elements."""
        sp = self._strip_ptr(side, strip)
        self._check(load().sac_halo_pack(self._ctx, int(side), sp), "sac_halo_pack")

    def halo_unpack(self, side: int, strip):
        sp = self._strip_ptr(side, strip)
        self._check(load().sac_halo_unpack(self._ctx, int(side), sp), "sac_halo_unpack")

    def get_cmax_bits(self, bits):
        """Copy the two running signal-speed keys into a device int64/uint64 tensor of 2."""
        bp = _dev_ptr(bits, "bits", 2, _I64, self.params.device)
        self._check(load().sac_get_cmax_bits(self._ctx, bp), "sac_get_cmax_bits")

    def set_cmax_bits(self, bits):
        bp = _dev_ptr(bits, "bits", 2, _I64, self.params.device)
        self._check(load().sac_set_cmax_bits(self._ctx, bp), "sac_set_cmax_bits")

    def debug_drop_copies(self, on: bool):
        """Test hook of the bounded copy waits (see sac_debug_drop_copies)."""
        self._check(load().sac_debug_drop_copies(self._ctx, int(bool(on))), "sac_debug_drop_copies")


class Batch:
    """Many independent FP32 runs advanced together (one launch per RK stage).

    ``Batch([dict(nx=..., ny=..., gamma=...), ...])``: each dict holds the
    ``sac_params`` fields of one run (precision is FP32 for every run).
    """

    def __init__(self, runs, stream="current", device=0):
        lib = load()
        n = len(runs)
        arr = (SacParams * n)()
        if stream == "current":
            import torch
            stream = torch.cuda.current_stream(device)
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        for k, kw in enumerate(runs):
            p = default_params()
            for key, v in kw.items():
                if key in ("c2", "gravity"):
                    fld = getattr(p, key)
                    for j, x in enumerate(v):
                        fld[j] = x
                else:
                    setattr(p, key, v)
            p.precision = FP32
            p.device = device
            p.stream = stream or None
            arr[k] = p
        self.params = arr
        self.n = n
        self._b = ctypes.c_void_p()
        rc = lib.sac_batch_init(arr, n, ctypes.byref(self._b))
        if rc != SAC_OK:
            raise SacError(rc, f"sac_batch_init failed: {lib.sac_status_string(rc).decode()}")

    def _check(self, rc, what):
        if rc != SAC_OK:
            lib = load()
            raise SacError(rc, f"{what}: {lib.sac_status_string(rc).decode()}: "
                               f"{lib.sac_batch_last_error(self._b).decode()}")

    def close(self):
        if self._b:
            load().sac_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, run, w, bg=None, t=0.0):
        p = self.params[run]
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (NF, p.ny, p.nx):
            raise ValueError(f"state shape {w.shape} != {(NF, p.ny, p.nx)}")
        bg = None if bg is None else np.ascontiguousarray(bg, dtype=np.float64)
        self._check(load().sac_batch_set_state(self._b, run, _dp(w), _dp(bg), float(t)), "sac_batch_set_state")

    def get_state(self, run):
        p = self.params[run]
        w = np.empty((NF, p.ny, p.nx), dtype=np.float64)
        t = ctypes.c_double()
        self._check(load().sac_batch_get_state(self._b, run, _dp(w), ctypes.byref(t)), "sac_batch_get_state")
        return w, t.value

    def steps(self, n):
        self._check(load().sac_batch_steps(self._b, int(n)), "sac_batch_steps")

    def sync(self):
        self._check(load().sac_batch_sync(self._b), "sac_batch_sync")

    def time(self, run):
        t, n = ctypes.c_double(), ctypes.c_long()
        self._check(load().sac_batch_time(self._b, run, ctypes.byref(t), ctypes.byref(n)), "sac_batch_time")
        return t.value, n.value

    def tune(self, trials=3):
        cfg = (ctypes.c_int * 3)()
        ms = ctypes.c_double()
        self._check(load().sac_batch_tune(self._b, int(trials), cfg, ctypes.byref(ms)), "sac_batch_tune")
        return tuple(cfg), ms.value

    def set_config(self, persistent, ctas_per_sm, order):
        self._check(load().sac_batch_set_config(self._b, persistent, ctas_per_sm, order), "sac_batch_set_config")

    def set_tile(self, tile):
        self._check(load().sac_batch_set_tile(self._b, int(tile)), "sac_batch_set_tile")

    def config(self):
        """(persistent, ctas_per_sm, order, tile shape)."""
        cfg = (ctypes.c_int * 4)()
        self._check(load().sac_batch_get_config(self._b, cfg), "sac_batch_get_config")
        return tuple(cfg)


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _stream_handle(stream, device=0):
    if stream == "current":
        import torch
        stream = torch.cuda.current_stream(device)
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    return stream or None


class CNN:
    """The learned coarse-grid correction network of an nx x ny periodic grid."""

    def __init__(self, nx, ny, device=0, stream="current"):
        lib = load()
        self.nx, self.ny, self.device = nx, ny, device
        self.stream = _stream_handle(stream, device)
        self._c = ctypes.c_void_p()
        rc = lib.sac_cnn_init(nx, ny, device, self.stream, ctypes.byref(self._c))
        if rc != SAC_OK:
            raise SacError(rc, f"sac_cnn_init: {lib.sac_status_string(rc).decode()}")
        self.nparams = int(lib.sac_cnn_param_count())

    def _check(self, rc, what):
        if rc != SAC_OK:
            lib = load()
            raise SacError(rc, f"{what}: {lib.sac_status_string(rc).decode()}: {lib.sac_cnn_last_error(self._c).decode()}")

    def close(self):
        if self._c:
            load().sac_cnn_free(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor_path(self, path: int):
        """Convolution kernel: 0 mma.sync, 1 tcgen05 (asynchronous-copy halo),
        2 tcgen05 (tensor-map halo, double-buffered)."""
        self._check(load().sac_cnn_set_tensor_path(self._c, int(path)), "sac_cnn_set_tensor_path")

    def sync(self):
        self._check(load().sac_cnn_sync(self._c), "sac_cnn_sync")

    def set_limiter(self, clip: float = 0.0, keep_positive: bool = False):
        """Limit applied corrections to clip residual scales per field and step (0: off) and,
        with keep_positive, drop them where density or pressure would halve."""
        self._check(load().sac_cnn_set_limiter(self._c, float(clip), int(bool(keep_positive))), "sac_cnn_set_limiter")

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(load().sac_cnn_set_params(self._c, _fp(flat), flat.size), "sac_cnn_set_params")

    def get_params(self):
        out = np.zeros(self.nparams, dtype=np.float32)
        self._check(load().sac_cnn_get_params(self._c, _fp(out), out.size), "sac_cnn_get_params")
        return out

    def set_scales(self, in_scale, out_scale):
        a = np.ascontiguousarray(in_scale, dtype=np.float32)
        b = np.ascontiguousarray(out_scale, dtype=np.float32)
        self._check(load().sac_cnn_set_scales(self._c, _fp(a), _fp(b)), "sac_cnn_set_scales")

    def _ptr(self, t, name: str, per_cell: int = NF) -> ctypes.c_void_p:
        """Device address of a float32 tensor of per_cell values per cell of the grid."""
        return _dev_ptr(t, name, per_cell * self.nx * self.ny, _F32, self.device)

    def forward(self, w_dev, gamma, dx, dy, pred_dev):
        wp, pp = self._ptr(w_dev, "w_dev"), self._ptr(pred_dev, "pred_dev", 8)
        self._check(load().sac_cnn_forward(self._c, wp, gamma, dx, dy, pp), "sac_cnn_forward")

    def grads(self, w_dev, next_dev, gamma, dx, dy):
        wp, np_ = self._ptr(w_dev, "w_dev"), self._ptr(next_dev, "next_dev")
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(load().sac_cnn_grads(self._c, wp, np_, gamma, dx, dy, _fp(g), ctypes.byref(loss)),
                    "sac_cnn_grads")
        return loss.value, g

    def train_step(self, w_dev, next_dev, gamma, dx, dy, lr, want_loss=True):
        wp, np_ = self._ptr(w_dev, "w_dev"), self._ptr(next_dev, "next_dev")
        loss = ctypes.c_double()
        self._check(load().sac_cnn_train_step(self._c, wp, np_, gamma, dx, dy, lr,
                                              ctypes.byref(loss) if want_loss else None), "sac_cnn_train_step")
        return loss.value

    def perturb(self, w_dev, out_dev, amp, seed: int):
        wp, op = self._ptr(w_dev, "w_dev"), self._ptr(out_dev, "out_dev")
        a = np.ascontiguousarray(amp, dtype=np.float32)
        self._check(load().sac_cnn_perturb(self._c, wp, op, _fp(a), int(seed)), "sac_cnn_perturb")

    def apply(self, solver):
        self._check(load().sac_cnn_apply(solver._ctx, self._c), "sac_cnn_apply")


def block_average(fine_dev, nfields, nxf, nyf, r, coarse_dev, stream="current"):
    if r < 1 or nxf % r or nyf % r:
        raise ValueError(f"block size {r} does not divide {nxf} x {nyf}")
    dev = fine_dev.device.index if fine_dev.is_cuda else -1
    fp = _dev_ptr(fine_dev, "fine_dev", nfields * nxf * nyf, _F32, dev)
    cp = _dev_ptr(coarse_dev, "coarse_dev", nfields * (nxf // r) * (nyf // r), _F32, dev)
    rc = load().sac_block_average(fp, nfields, nxf, nyf, r, cp, _stream_handle(stream, max(dev, 0)))
    if rc != SAC_OK:
        raise SacError(rc, "sac_block_average")


def step_noalloc(w_in, w_out, dt: float = 0.0, wait: bool = True, **kw) -> float:
    """One FP32 RK4 step of the device tensors ``w_in`` -> ``w_out`` (float32,
    contiguous, shape (6, ny, nx)) through ``sac_step_noalloc``: no allocation;
    keyword arguments are ``sac_params`` fields (stream: torch stream or handle)."""
    lib = load()
    p = default_params()
    stream = kw.pop("stream", "current")
    for k, v in kw.items():
        if k in ("c2", "gravity"):
            fld = getattr(p, k)
            for j, x in enumerate(v):
                fld[j] = x
        else:
            setattr(p, k, v)
    p.precision = FP32
    # the C side cannot see the buffers' sizes: refuse anything that is not a
    # contiguous float32 (6, ny, nx) tensor on the run's device
    for name, t in (("w_in", w_in), ("w_out", w_out)):
        if tuple(t.shape) != (NF, p.ny, p.nx):
            raise ValueError(f"{name} shape {tuple(t.shape)} != {(NF, p.ny, p.nx)}")
        if str(t.dtype) != "torch.float32" or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor")
        if not t.is_cuda or t.device.index != p.device:
            raise ValueError(f"{name} must live on cuda:{p.device}, not {t.device}")
    if stream == "current":
        import torch
        stream = torch.cuda.current_stream(p.device)
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    p.stream = stream or None
    out = ctypes.c_double(0.0)
    rc = lib.sac_step_noalloc(ctypes.byref(p), ctypes.c_void_p(w_in.data_ptr()), ctypes.c_void_p(w_out.data_ptr()),
                              float(dt), ctypes.byref(out) if wait else None)
    if rc != SAC_OK:
        raise SacError(rc, f"sac_step_noalloc: {lib.sac_status_string(rc).decode()}")
    return out.value


class Solver3:
    """One periodic 3D run (eight fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z):
    ``Solver3(nx=..., ny=..., nz=..., precision=FP32)``; states are FP64 host
    arrays of shape (8, nz, ny, nx).  Calls are synchronous."""

    def __init__(self, stream="current", **kw):
        lib = load()
        p = Sac3Params()
        lib.sac3_default_params(ctypes.byref(p))
        for k, v in kw.items():
            if k == "c2":
                for j, x in enumerate(v):
                    p.c2[j] = x
            else:
                setattr(p, k, v)
        if stream == "current":
            import torch
            stream = torch.cuda.current_stream(p.device)
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        p.stream = stream or None
        self.params = p
        self._ctx = ctypes.c_void_p()
        rc = lib.sac3_init(ctypes.byref(p), ctypes.byref(self._ctx))
        if rc != SAC_OK:
            raise SacError(rc, f"sac3_init failed: {lib.sac_status_string(rc).decode()}")
        self.shape = (8, p.nz, p.ny, p.nx)

    def _check(self, rc: int, what: str):
        if rc != SAC_OK:
            lib = load()
            raise SacError(rc, f"{what}: {lib.sac_status_string(rc).decode()}: {lib.sac3_last_error(self._ctx).decode()}")

    def set_state(self, w, t: float = 0.0):
        a = np.ascontiguousarray(w, dtype=np.float64)
        if a.shape != self.shape:
            raise ValueError(f"state must be {self.shape}, got {a.shape}")
        self._check(load().sac3_set_state(self._ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t),
                    "sac3_set_state")

    def get_state(self):
        w = np.empty(self.shape, dtype=np.float64)
        t = ctypes.c_double()
        self._check(load().sac3_get_state(self._ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.byref(t)), "sac3_get_state")
        return w, t.value

    def step(self, dt: float = 0.0) -> float:
        out = ctypes.c_double()
        self._check(load().sac3_step(self._ctx, dt, ctypes.byref(out)), "sac3_step")
        return out.value

    def steps(self, n: int):
        self._check(load().sac3_steps(self._ctx, n), "sac3_steps")

    def run_to(self, t_end: float, max_steps: int = -1) -> int:
        """CFL steps until t_end (the last one clipped onto it); returns the step count."""
        n = ctypes.c_long(0)
        self._check(load().sac3_run_to(self._ctx, float(t_end), int(max_steps), ctypes.byref(n)), "sac3_run_to")
        return n.value

    def time(self) -> float:
        return load().sac3_time(self._ctx)

    def sums(self) -> np.ndarray:
        """FP64 sums of the eight fields over the interior."""
        out = np.zeros(8)
        self._check(load().sac3_sums(self._ctx, _dp(out)), "sac3_sums")
        return out

    def divb(self):
        """(max |div B|, mean |div B|) of the current state, FP64."""
        a, m = ctypes.c_double(), ctypes.c_double()
        self._check(load().sac3_divb(self._ctx, ctypes.byref(a), ctypes.byref(m)), "sac3_divb")
        return a.value, m.value

    def debug_drop_copies(self, on: bool):
        """Test hook of the bounded copy waits (see sac3_debug_drop_copies)."""
        self._check(load().sac3_debug_drop_copies(self._ctx, int(bool(on))), "sac3_debug_drop_copies")

    def close(self):
        if self._ctx:
            load().sac3_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
