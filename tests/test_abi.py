"""The C-ABI library loads and exports every entry point include/soap.h declares; argument
validation rejects bad input before touching the GPU (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(soap_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2301_04259_gb300 import _build
    _build.build()
    from paper_2301_04259_gb300 import soap
    return soap


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("soap_init_star", "soap_quiet_spectrum", "soap_active_phases", "soap_rv_ccf",
              "soap_active_rv", "soap_set_host_async", "soap_set_quiet_spectrum_f32",
              "soap_set_active_spectrum_f32", "soap_set_instrument_resolution", "soap_lower_resolution",
              "soap_evolve_radii", "soap_active_phases_radii", "soap_set_facula_limb_brightening",
              "soap_inject_bisectors",
              "soap_free", "soap_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(str(lib.LIB_PATH))
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing


def test_invalid_star_is_rejected_without_a_gpu(lib):
    from paper_2301_04259_gb300.synth import Star
    q = np.ones((2, 64))
    good = dict(grid_n=10, vsini_kms=2.0, incl_deg=90.0, u1=0.3, u2=0.2, lambda_start_A=6000.0,
                lambda_end_A=6001.0, n_px=64, mu_values=np.array([0.3, 0.9]))
    bad = [dict(grid_n=0), dict(n_px=1), dict(lambda_end_A=5000.0), dict(vsini_kms=4e5),
           dict(mu_values=np.array([0.0, 0.5])), dict(incl_deg=200.0), dict(vsini_kms=float("nan")),
           dict(mu_values=np.linspace(0.01, 1, 65))]
    for b in bad:
        st = Star(**{**good, **b})
        qq = np.ones((st.n_mu, st.n_px))
        with pytest.raises(lib.SoapError) as ei:
            lib.soap_init_star(st, qq)
        assert ei.value.status in (lib.SOAP_EINVAL, lib.SOAP_ERANGE)
        assert lib.soap_last_error()
    # too many taps for the pixel size
    st = Star(**{**good, "vsini_kms": 3000.0})
    with pytest.raises(lib.SoapError) as ei:
        lib.soap_init_star(st, q)
    assert ei.value.status == lib.SOAP_ERANGE


def test_null_arguments_are_rejected(lib):
    ctx = ctypes.c_void_p()
    assert lib._lib.soap_init_star(None, None, 0, None, ctypes.byref(ctx)) == lib.SOAP_EINVAL
    assert lib._lib.soap_quiet_spectrum(None, 0, 0, None, 0) == lib.SOAP_EINVAL
    assert lib._lib.soap_active_phases(None, None, 0, None, 0, 1, 0, None, 0) == lib.SOAP_EINVAL
    assert lib._lib.soap_active_rv(None, None, 0, None, 0, 1, 0, None, None, 0, 0.8, -20.0, 0.25, 161,
                                   None, None, 0) == lib.SOAP_EINVAL
    assert lib._lib.soap_set_host_async(None, 1) == lib.SOAP_EINVAL
    assert lib._lib.soap_set_ccf_tensor_cores(None, 1) == lib.SOAP_EINVAL
    assert lib._lib.soap_surrogate_encode(None, 4, None, None) == lib.SOAP_EINVAL
    assert lib._lib.soap_surrogate_encode(None, -1, None, None) == lib.SOAP_EINVAL
    assert lib._lib.soap_surrogate_encode(None, 0, None, None) == lib.SOAP_OK       # nothing to do
    lib._lib.soap_free(None)


def test_batch_entry_points_without_a_gpu(lib):
    assert lib._lib.soap_active_batch(None, None, 0, None, 0, None, 0, 0, None, None, 0) == lib.SOAP_EINVAL
    assert lib._lib.soap_batch_set_rv(None, None, None, 0, 0.82, -30.0, 0.25, 241, 20.0, 0) == lib.SOAP_EINVAL
    assert lib._lib.soap_debug_inject_timeout(None) == lib.SOAP_EINVAL
    n = lib.soap_batch_num_variants()
    assert n >= 2
    seen = set()
    for v in range(n):
        pb, r = lib.soap_batch_variant_info(v)
        assert pb in (1, 2, 4, 8, 16) and r in (1, 2, 4, 8)
        seen.add((pb, r))
    assert len(seen) == n                                    # no duplicate variants
    with pytest.raises(lib.SoapError) as ei:
        lib.soap_batch_variant_info(n)
    assert ei.value.status == lib.SOAP_ERANGE
    assert lib._lib.soap_batch_set_variant(None, 0) == lib.SOAP_EINVAL
    best = ctypes.c_int32()
    assert lib._lib.soap_batch_autotune(None, None, 0, None, 0, None, 0, None, 1, None,
                                        ctypes.byref(best)) == lib.SOAP_EINVAL
