"""ctypes binding of libdos.so: the C ABI of include/dos.h, argument marshalling only.

Every function here has the name of the C entry point it calls and takes plain
integers for device pointers (e.g. ``tensor.data_ptr()``) and CUDA streams.
A non-zero status raises :class:`DosError` carrying ``dos_last_error()``.
There is no fallback: if the library is not built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_void_p

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdos.so")

DOS_OK, DOS_ERR_ARG, DOS_ERR_OOM, DOS_ERR_CUDA, DOS_ERR_STATE, DOS_ERR_TIMEOUT, DOS_ERR_UNSUPPORTED = range(7)
DOS_EVAN_DECAY, DOS_EVAN_ZERO = 0, 1
DOS_LOSS_MSE, DOS_LOSS_MSE_SCALED = 0, 1
DOS_PATH_AUTO, DOS_PATH_MULTIPASS, DOS_PATH_FUSED, DOS_PATH_DFT_GEMM, DOS_PATH_MULTIPASS_BULK, DOS_PATH_DFT_GEMM_X3 = \
    0, 1, 2, 3, 4, 5

ERROR_NAMES = {1: "DOS_ERR_ARG", 2: "DOS_ERR_OOM", 3: "DOS_ERR_CUDA", 4: "DOS_ERR_STATE",
               5: "DOS_ERR_TIMEOUT", 6: "DOS_ERR_UNSUPPORTED"}

# every symbol include/dos.h declares (checked by the CPU tests)
EXPORTS = ("dos_supported_m", "dos_create", "dos_set_stream", "dos_forward", "dos_loss",
           "dos_read_loss", "dos_backward", "dos_step", "dos_output_field", "dos_layer_field",
           "dos_propagate", "dos_set_timing", "dos_kernel_time", "dos_workspace_bytes",
           "dos_last_launch_count", "dos_path", "dos_describe", "dos_destroy", "dos_last_error",
           "dos_loss_noalloc", "dos_efficiency", "dos_quantize_thickness", "dos_set_misalignment")

DOS_NOALLOC_MAX_LAMBDA = 65536

KERNEL_KINDS = ("column_forward", "column_adjoint", "row_forward", "row_adjoint", "row_output",
                "row_seed", "loss", "grad_reduce", "fused_forward", "fused_adjoint",
                "gemm_propagation", "gemm_field")


class DosError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {message}")
        self.code = code


class DosConfig(ctypes.Structure):
    _fields_ = [
        ("n", c_int), ("m", c_int), ("n_layers", c_int), ("n_lambda", c_int),
        ("n_lambda_total", c_int), ("fov", c_int), ("aperture", c_int),
        ("pitch", c_double),
        ("gaps", POINTER(c_double)), ("lambda_", POINTER(c_double)),
        ("n_index", POINTER(c_double)), ("kappa", POINTER(c_double)),
        ("n_medium", c_double), ("h_base", c_double),
        ("evanescent", c_int), ("loss", c_int), ("path", c_int),
        ("detector_bin", c_int),
    ]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdos.so (once) and declare the signatures of include/dos.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: the CUDA library has not been built "
            "(run `python -c 'import __graft_entry__ as g; g.build()'`); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    p = c_void_p
    sig = {
        "dos_supported_m": (c_int, [POINTER(c_int), c_int]),
        "dos_create": (c_int, [POINTER(p), POINTER(DosConfig), p]),
        "dos_set_stream": (c_int, [p, p]),
        "dos_forward": (c_int, [p, p, p, c_int]),
        "dos_loss": (c_int, [p, p, POINTER(c_double), p, p]),
        "dos_read_loss": (c_int, [p, POINTER(c_double)]),
        "dos_backward": (c_int, [p, p, p]),
        "dos_step": (c_int, [p, p, p, p, p, p, POINTER(c_double)]),
        "dos_output_field": (c_int, [p, p]),
        "dos_layer_field": (c_int, [p, c_int, p]),
        "dos_propagate": (c_int, [p, c_int, p, p, c_int]),
        "dos_set_timing": (c_int, [p, c_int]),
        "dos_kernel_time": (c_int, [p, c_int, POINTER(c_int), POINTER(c_double)]),
        "dos_workspace_bytes": (c_size_t, [p]),
        "dos_last_launch_count": (c_int, [p]),
        "dos_path": (c_int, [p]),
        "dos_describe": (c_int, [p, ctypes.c_char_p, c_int]),
        "dos_destroy": (None, [p]),
        "dos_last_error": (ctypes.c_char_p, [p]),
        "dos_loss_noalloc": (c_int, [p, p, c_int, c_int, c_int, c_int, POINTER(c_double), p, p, p]),
        "dos_efficiency": (c_int, [p, p]),
        "dos_set_misalignment": (c_int, [p, POINTER(c_double)]),
        "dos_quantize_thickness": (c_int, [p, p, c_size_t, c_double, c_int, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str) -> None:
    if rc != DOS_OK:
        msg = load().dos_last_error(None)
        raise DosError(rc, where, msg.decode() if msg else "")


def _dptr(x) -> c_double:
    return x.ctypes.data_as(POINTER(c_double)) if x is not None else None


# ------------------------------------------------------------------ entry points
def dos_supported_m() -> list:
    lib = load()
    buf = (c_int * 64)()
    k = lib.dos_supported_m(buf, 64)
    return list(buf[:k])


def dos_create(cfg: DosConfig, stream: int = 0) -> int:
    h = c_void_p()
    _check(load().dos_create(ctypes.byref(h), ctypes.byref(cfg), stream or None), "dos_create")
    return h.value


def dos_set_stream(ctx: int, stream: int) -> None:
    _check(load().dos_set_stream(ctx, stream or None), "dos_set_stream")


def dos_forward(ctx: int, d_h: int, d_I: int, save_for_backward: bool) -> None:
    _check(load().dos_forward(ctx, d_h, d_I or None, int(bool(save_for_backward))), "dos_forward")


def dos_loss(ctx: int, d_T: int, read_loss: bool, d_psnr: int, d_dLdI: int):
    out = c_double()
    _check(load().dos_loss(ctx, d_T, ctypes.byref(out) if read_loss else None, d_psnr or None,
                           d_dLdI or None), "dos_loss")
    return out.value if read_loss else None


def dos_read_loss(ctx: int) -> float:
    out = c_double()
    _check(load().dos_read_loss(ctx, ctypes.byref(out)), "dos_read_loss")
    return out.value


def dos_backward(ctx: int, d_dLdI: int, d_dLdh: int) -> None:
    _check(load().dos_backward(ctx, d_dLdI, d_dLdh), "dos_backward")


def dos_step(ctx: int, d_h: int, d_T: int, d_dLdh: int, d_I: int, d_psnr: int, read_loss: bool):
    out = c_double()
    _check(load().dos_step(ctx, d_h, d_T, d_dLdh, d_I or None, d_psnr or None,
                           ctypes.byref(out) if read_loss else None), "dos_step")
    return out.value if read_loss else None


def dos_output_field(ctx: int, d_o: int) -> None:
    _check(load().dos_output_field(ctx, d_o), "dos_output_field")


def dos_layer_field(ctx: int, layer: int, d_v: int) -> None:
    _check(load().dos_layer_field(ctx, layer, d_v), "dos_layer_field")


def dos_propagate(ctx: int, gap: int, d_in: int, d_out: int, adjoint: bool) -> None:
    _check(load().dos_propagate(ctx, gap, d_in, d_out, int(bool(adjoint))), "dos_propagate")


def dos_set_timing(ctx: int, enable: bool) -> None:
    _check(load().dos_set_timing(ctx, int(bool(enable))), "dos_set_timing")


def dos_kernel_time(ctx: int, kind: int):
    """(launches, total milliseconds) of one kernel kind since timing was enabled."""
    n = c_int()
    ms = c_double()
    _check(load().dos_kernel_time(ctx, kind, ctypes.byref(n), ctypes.byref(ms)), "dos_kernel_time")
    return n.value, ms.value


def dos_workspace_bytes(ctx: int) -> int:
    return int(load().dos_workspace_bytes(ctx))


def dos_last_launch_count(ctx: int) -> int:
    return int(load().dos_last_launch_count(ctx))


def dos_path(ctx: int) -> int:
    return int(load().dos_path(ctx))


def dos_describe(ctx: int) -> str:
    buf = ctypes.create_string_buffer(4096)
    load().dos_describe(ctx, buf, 4096)
    return buf.value.decode()


def dos_destroy(ctx: int) -> None:
    if ctx:
        load().dos_destroy(ctx)


def dos_last_error(ctx: int = 0) -> str:
    msg = load().dos_last_error(ctx or None)
    return msg.decode() if msg else ""


def dos_loss_noalloc(d_I: int, d_T: int, n_lambda: int, fov: int, n_lambda_total: int, loss: int,
                     read_loss: bool, d_psnr: int, d_dLdI: int, stream: int):
    """Scoring with library-owned fixed scratch (no allocation); see include/dos.h."""
    out = c_double()
    _check(load().dos_loss_noalloc(d_I, d_T, n_lambda, fov, n_lambda_total, loss,
                                   ctypes.byref(out) if read_loss else None, d_psnr or None,
                                   d_dLdI or None, stream or None), "dos_loss_noalloc")
    return out.value if read_loss else None


def dos_efficiency(ctx: int, d_eta: int) -> None:
    _check(load().dos_efficiency(ctx, d_eta), "dos_efficiency")


def dos_quantize_thickness(d_h: int, d_hq: int, count: int, h_max: float, bits: int, stream: int) -> None:
    _check(load().dos_quantize_thickness(d_h, d_hq, count, h_max, bits, stream or None), "dos_quantize_thickness")


def dos_set_misalignment(ctx: int, disp) -> None:
    """disp: None or a (K, 3) float64 array of layer displacements [m]."""
    if disp is None:
        _check(load().dos_set_misalignment(ctx, None), "dos_set_misalignment")
        return
    import numpy as np
    arr = np.ascontiguousarray(disp, dtype=np.float64)
    _check(load().dos_set_misalignment(ctx, arr.ctypes.data_as(POINTER(c_double))), "dos_set_misalignment")
