"""The C-ABI library loads and exports every entry point include/wake.h declares (no GPU
calls), and the binding's parameter struct matches the header's layout."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wake.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**\s*(wake_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libwake():
    from paper_1411_3246_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_entry_points_are_exported(libwake):
    from paper_1411_3246_gb300 import wake
    names = _declared()
    assert len(names) >= 14
    assert set(names) == set(wake.EXPORTS)
    for n in names:
        assert hasattr(libwake, n), n


def test_params_struct_layout():
    from paper_1411_3246_gb300 import wake
    # 4 int32 + 13 doubles + 2 int64 + 2 int32 (geometry, reserved), no padding
    assert C.sizeof(wake.wake_params) == 4 * 4 + 13 * 8 + 2 * 8 + 2 * 4
    assert wake.wake_params.rmax.offset == 16
    assert wake.wake_params.n_beam.offset == 16 + 13 * 8
    assert wake.wake_params.geometry.offset == 16 + 13 * 8 + 16


def test_invalid_parameters_rejected_before_any_device_work(libwake):
    """wake_init checks sizes on the host and returns WAKE_EINVAL with a message."""
    import synth
    from paper_1411_3246_gb300 import wake
    bad = wake.params_of(synth.config_linear(nr=4096), wake.WAKE_FP64)
    h = C.c_void_p()
    rc = wake.lib().wake_init(C.byref(bad), 1, None, C.byref(h))
    assert rc == wake.WAKE_EINVAL
    assert b"nr" in wake.lib().wake_last_error()
    odd = wake.params_of(synth.config_blowout(n_beam=0, nr=32, nxi=16), wake.WAKE_FP64)
    odd.ppc = 3
    assert wake.lib().wake_init(C.byref(odd), 1, None, C.byref(h)) == wake.WAKE_EINVAL


def test_corrupt_parameters_rejected(libwake):
    """Non-finite or inconsistent parameters return WAKE_EINVAL from wake_init before any CUDA
    call (runs without a GPU)."""
    import math

    import synth
    from paper_1411_3246_gb300 import wake
    h = C.c_void_p()
    base = synth.config_blowout(n_beam=1024, nr=32, nxi=16)
    for field, value in (("rmax", math.nan), ("ximax", -1.0), ("ds", math.nan), ("gamma_b", 0.5),
                         ("sigma_r", math.nan), ("u_th", -0.1), ("n_drive", 2048), ("nxi", 1), ("geometry", 2)):
        p = wake.params_of(base, wake.WAKE_MIXED)
        setattr(p, field, value)
        assert wake.lib().wake_init(C.byref(p), 1, None, C.byref(h)) == wake.WAKE_EINVAL, field
        assert not h.value
    good = wake.params_of(base, wake.WAKE_MIXED)
    mixed = (wake.wake_params * 2)(good, wake.params_of(base, wake.WAKE_FP64))
    assert wake.lib().wake_init(mixed, 2, None, C.byref(h)) == wake.WAKE_EINVAL
