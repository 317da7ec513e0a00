"""CPU checks of the C ABI: the library loads, exports every symbol that
include/dos.h declares, and its host-side validation rejects bad designs
before touching a GPU.  No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2604_02624_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_2604_02624_gb300 import build
        build.build()
    return L.load()


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "dos.h")).read()
    return sorted(set(re.findall(r"DOS_API\s+[\w\s\*]+?\b(dos_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert _header_symbols() == sorted(L.EXPORTS)


def _header_parameters():
    """{name: [parameter declarations]} of every DOS_API function in dos.h."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dos.h")).read(), flags=re.S)
    out = {}
    for name, params in re.findall(r"DOS_API\s+[\w\s\*]+?\b(dos_\w+)\s*\(([^)]*)\)", text):
        params = " ".join(params.split())
        out[name] = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes prototype has the header's number of parameters."""
    decl = _header_parameters()
    import inspect
    src = inspect.getsource(L.load)
    for name, params in decl.items():
        m = re.search(r'"%s": \((.*?), \[(.*?)\]\),' % name, src)
        assert m, name
        args = [a for a in m.group(2).split(",") if a.strip()]
        assert len(args) == len(params), (name, params, args)


def test_boundary_entry_points_have_the_designed_signatures():
    """The calls of the design's boundary: create / forward / loss / backward /
    set_stream / destroy / last_error, with backward taking only the seed and
    the output (the context keeps the thickness of the saved forward) and
    last_error taking the context."""
    decl = _header_parameters()
    assert decl["dos_create"] == ["dos_ctx **out", "const dos_config *cfg", "void *cuda_stream"]
    assert decl["dos_forward"] == ["dos_ctx *ctx", "const float *d_h", "float *d_I", "int save_for_backward"]
    assert decl["dos_loss"] == ["dos_ctx *ctx", "const float *d_T", "double *h_loss", "float *d_psnr",
                                "float *d_dLdI"]
    assert decl["dos_backward"] == ["dos_ctx *ctx", "const float *d_dLdI", "float *d_dLdh"]
    assert decl["dos_set_stream"] == ["dos_ctx *ctx", "void *cuda_stream"]
    assert decl["dos_destroy"] == ["dos_ctx *ctx"]
    assert decl["dos_last_error"] == ["const dos_ctx *ctx"]


def test_library_exports_every_declared_symbol(lib):
    for name in _header_symbols():
        assert hasattr(lib, name), name


def test_library_hides_internal_symbols(lib):
    # internal C++ kernels and helpers must not leak into the dynamic symbol table
    with pytest.raises(AttributeError):
        getattr(lib, "launch_htable")


def test_config_struct_matches_the_header():
    """The ctypes mirror of dos_config has the header's fields, in order and
    with the header's C types (int / double / pointer)."""

    text = open(os.path.join(ROOT, "include", "dos.h")).read()
    body = text[text.index("typedef struct dos_config {"):text.index("} dos_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int|double|const double \*)\s*([a-z_]+);", body)
    names = [n if n != "lambda" else "lambda_" for _, n in fields]
    assert names == [f[0] for f in L.DosConfig._fields_]
    kinds = {"int": ctypes.c_int, "double": ctypes.c_double}
    for (ty, _), (_, ct) in zip(fields, L.DosConfig._fields_):
        if ty.endswith("*"):
            assert issubclass(ct, ctypes._Pointer)
        else:
            assert ct is kinds[ty]


def test_supported_sizes_are_reported(lib):
    ms = L.dos_supported_m()
    for m in (128, 400, 512):
        assert m in ms


def _cfg(**over):
    lam = np.array([500e-9, 600e-9])
    keep = {"gaps": np.array([1e-5, 1e-5]), "lam": lam, "nidx": np.array([1.7, 1.7])}
    c = L.DosConfig()
    c.n, c.m, c.n_layers, c.n_lambda, c.n_lambda_total = 64, 128, 1, 2, 0
    c.fov, c.aperture, c.pitch = 32, 0, 3e-7
    c.gaps = L._dptr(keep["gaps"])
    c.lambda_ = L._dptr(keep["lam"])
    c.n_index = L._dptr(keep["nidx"])
    c.kappa = None
    c.n_medium, c.h_base, c.evanescent, c.loss, c.path = 1.0, 0.0, 0, 0, 0
    for k, v in over.items():
        if isinstance(v, np.ndarray):
            keep[k] = v
            v = L._dptr(v)
        setattr(c, k, v)
    return c, keep


@pytest.mark.parametrize("over,msg", [
    ({"n": 0}, "n must be"),
    ({"m": 100}, "not a supported padded size"),
    ({"m": 32}, "m must be >= n"),
    ({"n_layers": 0}, "n_layers"),
    ({"fov": 33}, "fov"),
    ({"fov": 65}, "fov"),
    ({"aperture": 31}, "aperture"),
    ({"pitch": -1.0}, "pitch"),
    ({"lambda_": np.array([500e-9, -1.0])}, "lambda"),
    ({"gaps": np.array([1e-5, np.nan])}, "gaps"),
    ({"n_medium": 0.0}, "n_medium"),
    ({"evanescent": 7}, "evanescent"),
    ({"loss": 9}, "loss"),
    ({"n_lambda_total": 1}, "n_lambda_total"),
    ({"path": 6}, "path"),
    ({"detector_bin": 3}, "detector_bin"),
    ({"detector_bin": -2}, "detector_bin"),
    ({"path": -1}, "path"),
])
def test_invalid_designs_are_rejected_on_the_host(lib, over, msg):
    cfg, keep = _cfg(**over)
    h = ctypes.c_void_p(123)
    rc = lib.dos_create(ctypes.byref(h), ctypes.byref(cfg), None)
    assert rc == L.DOS_ERR_ARG
    assert h.value is None
    assert msg in L.dos_last_error()


@pytest.mark.parametrize("path", [L.DOS_PATH_AUTO, L.DOS_PATH_MULTIPASS, L.DOS_PATH_FUSED,
                                  L.DOS_PATH_DFT_GEMM, L.DOS_PATH_MULTIPASS_BULK, L.DOS_PATH_DFT_GEMM_X3])
def test_every_declared_path_passes_host_validation(lib, path):
    """Host validation accepts every DOS_PATH_* value (without a GPU the call
    then stops at the first CUDA call, not at argument checking)."""
    cfg, keep = _cfg(path=path)
    h = ctypes.c_void_p()
    rc = lib.dos_create(ctypes.byref(h), ctypes.byref(cfg), None)
    assert rc != L.DOS_ERR_ARG, L.dos_last_error()
    if rc == L.DOS_OK:
        lib.dos_destroy(h)


def test_null_arguments_are_rejected(lib):
    assert lib.dos_create(None, None, None) == L.DOS_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.dos_create(ctypes.byref(h), None, None) == L.DOS_ERR_ARG
    assert lib.dos_forward(None, None, None, 0) == L.DOS_ERR_ARG
    assert lib.dos_backward(None, None, None) == L.DOS_ERR_ARG
    lib.dos_destroy(None)  # no-op
    assert lib.dos_workspace_bytes(None) == 0
