"""The C-ABI library builds, loads and exports every symbol include/sac.h
declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sac3?_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_06423_b300 import build, sac
    build.build()
    return sac.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared("sac.h")
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1710_06423_b300 import sac
    assert sorted(sac.EXPORTS) == _declared("sac.h")


def test_params_struct_layout_matches_header(lib):
    """Default parameters round-trip through the C struct (catches a field-order mismatch)."""
    from paper_1710_06423_b300 import sac
    p = sac.default_params()
    assert (p.nx, p.ny, p.precision, p.hyperdiffusion, p.has_background) == (64, 64, 0, 1, 0)
    assert abs(p.gamma - 5 / 3) < 1e-15 and p.courant == 0.3 and p.c_shk == 0.5
    assert list(p.c2) == [0.02, 0.1, 0.1, 0.02, 0.02, 0.02]
    assert p.x1 == 1.0 and p.y1 == 1.0 and p.stream is None


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("nx", 65537), ("ny", 1 << 20), ("gamma", 1.0), ("courant", 0.0),
                                         ("bc_x", 7), ("precision", 5), ("x1", 0.0)])
def test_bad_params_rejected_before_any_device_call(lib, field, value):
    from paper_1710_06423_b300 import sac
    p = sac.default_params()
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    rc = lib.sac_init(ctypes.byref(p), ctypes.byref(ctx))
    assert rc == sac.SAC_ERR_ARG and not ctx.value


def test_status_strings(lib):
    assert lib.sac_status_string(0) == b"SAC_OK"
    assert lib.sac_status_string(-5) == b"SAC_ERR_NONFINITE"
    assert lib.sac_status_string(3) == b"SAC_UNKNOWN"


def test_params3_struct_layout_matches_header(lib):
    """3D defaults round-trip through the C struct (catches a field-order mismatch)."""
    from paper_1710_06423_b300 import sac
    p = sac.Sac3Params()
    lib.sac3_default_params(ctypes.byref(p))
    assert (p.nx, p.ny, p.nz) == (32, 32, 32)
    assert (p.x1, p.y1, p.z1) == (1.0, 1.0, 1.0)
    assert abs(p.gamma - 5 / 3) < 1e-15 and p.courant == 0.3 and p.hyperdiffusion == 1
    assert list(p.c2) == [0.02, 0.1, 0.1, 0.1, 0.02, 0.02, 0.02, 0.02] and p.c_shk == 0.5
    assert p.precision == sac.FP64 and p.device == 0 and not p.stream


@pytest.mark.parametrize("case", ["cpu_tensor", "wrong_shape", "float64", "strided"])
def test_step_noalloc_refuses_bad_buffers_before_the_call(lib, case):
    """The allocation-free step cannot see the sizes of the caller's buffers, so
    the binding refuses anything but a contiguous float32 (6, ny, nx) tensor on
    the run's device before it reaches the C call."""
    import torch
    from paper_1710_06423_b300 import sac
    nx, ny = 16, 12
    good = torch.zeros((6, ny, nx), dtype=torch.float32)
    bad = {
        "cpu_tensor": good,
        "wrong_shape": torch.zeros((6, ny, nx - 1), dtype=torch.float32),
        "float64": torch.zeros((6, ny, nx), dtype=torch.float64),
        "strided": torch.zeros((6, nx, ny), dtype=torch.float32).transpose(1, 2),
    }[case]
    with pytest.raises(ValueError):
        sac.step_noalloc(bad, bad, 0.0, nx=nx, ny=ny)
