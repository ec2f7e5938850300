"""ctypes binding of libsoap (include/soap.h), with the same names as the C-ABI.

Argument marshalling only: arrays are passed as raw pointers (``torch.Tensor.data_ptr()``
for CUDA tensors, the numpy buffer for host arrays), every computation runs in the CUDA
library.  Importing this module loads ``_lib/libsoap.so`` and raises if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``): there is no fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path
from typing import Optional, Sequence

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libsoap.so"

SOAP_OK, SOAP_EINVAL, SOAP_ENOMEM, SOAP_ECUDA, SOAP_ERANGE, SOAP_ETIMEOUT, SOAP_ESTATE = range(7)
STATUS_NAMES = {0: "SOAP_OK", 1: "SOAP_EINVAL", 2: "SOAP_ENOMEM", 3: "SOAP_ECUDA",
                4: "SOAP_ERANGE", 5: "SOAP_ETIMEOUT", 6: "SOAP_ESTATE"}
SOAP_FP64, SOAP_FP32, SOAP_BF16X3 = 0, 1, 2
SOAP_FORM_TOEPLITZ, SOAP_FORM_DIRECT = 0, 1
SOAP_EFFECT_TOT, SOAP_EFFECT_FLUX, SOAP_EFFECT_BCONV = 1, 2, 4
SOAP_SPOT, SOAP_FACULA = 1, 2
SOAP_BATCH_SPECTRUM, SOAP_BATCH_RESIDUAL = 0, 1
SOAP_MAX_REGIONS, SOAP_MAX_CLASSES, SOAP_MAX_MU, SOAP_MAX_TAPS = 64, 8, 64, 256
TIMERS = ("geometry", "pad_rows", "contrast", "phase_hist", "regions", "contract", "contract_quiet",
          "direct", "ccf", "fit", "ccf_aux", "lsf", "bisectors")
(SOAP_TIMER_GEOMETRY, SOAP_TIMER_PAD_ROWS, SOAP_TIMER_CONTRAST, SOAP_TIMER_PHASE_HIST,
 SOAP_TIMER_REGIONS, SOAP_TIMER_CONTRACT, SOAP_TIMER_CONTRACT_QUIET, SOAP_TIMER_DIRECT,
 SOAP_TIMER_CCF, SOAP_TIMER_FIT) = range(10)


class soap_star_desc(ctypes.Structure):
    _fields_ = [("grid_n", ctypes.c_int32), ("n_mu", ctypes.c_int32), ("n_px", ctypes.c_int64),
                ("vsini_kms", ctypes.c_double), ("incl_deg", ctypes.c_double),
                ("u1", ctypes.c_double), ("u2", ctypes.c_double),
                ("diff_rot_alpha", ctypes.c_double), ("lambda_start_A", ctypes.c_double),
                ("lambda_end_A", ctypes.c_double), ("t_quiet_K", ctypes.c_double),
                ("mu_values", ctypes.POINTER(ctypes.c_double))]


class soap_region(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lat_deg", ctypes.c_double), ("lon_deg", ctypes.c_double),
                ("radius_rstar", ctypes.c_double), ("temp_K", ctypes.c_double)]


class soap_batch_item(ctypes.Structure):
    _fields_ = [("vsini_kms", ctypes.c_double), ("incl_deg", ctypes.c_double),
                ("first_region", ctypes.c_int32), ("n_regions", ctypes.c_int32),
                ("first_phase", ctypes.c_int32), ("n_phases", ctypes.c_int32)]


class soap_surrogate_desc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("hidden", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("n_coef", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("in_lo", ctypes.POINTER(ctypes.c_float)), ("in_hi", ctypes.POINTER(ctypes.c_float))]


class soap_star_info(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_int64), ("tap_min", ctypes.c_int32),
                ("n_taps", ctypes.c_int32), ("delta", ctypes.c_double),
                ("total_intensity", ctypes.c_double), ("fixed_point_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class soap_region_evolution(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int32), ("reserved", ctypes.c_int32), ("area0_msh", ctypes.c_double),
                ("rate_msh_per_day", ctypes.c_double), ("t_peak_day", ctypes.c_double),
                ("fwhm_day", ctypes.c_double), ("asymmetry", ctypes.c_double)]


SOAP_EVOLVE_NONE, SOAP_EVOLVE_LINEAR_GROWTH, SOAP_EVOLVE_LINEAR_DECAY, SOAP_EVOLVE_ASYM_GAUSSIAN = 0, 1, 2, 3


class SoapError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(str(LIB_PATH))
    P, i32, i64, u32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    sig = {
        "soap_init_star": (i32, [ctypes.POINTER(soap_star_desc), P, ctypes.c_int, P, ctypes.POINTER(P)]),
        "soap_set_active_spectrum": (i32, [P, i32, P, ctypes.c_int]),
        "soap_update_star": (i32, [P, ctypes.POINTER(soap_star_desc)]),
        "soap_set_quiet_spectrum": (i32, [P, P, ctypes.c_int]),
        "soap_set_quiet_spectrum_f32": (i32, [P, P, ctypes.c_int]),
        "soap_set_active_spectrum_f32": (i32, [P, i32, P, ctypes.c_int]),
        "soap_set_profiling": (i32, [P, ctypes.c_int]),
        "soap_get_kernel_time": (i32, [P, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
        "soap_reset_kernel_times": (i32, [P]),
        "soap_set_stream": (i32, [P, P]),
        "soap_synchronize": (i32, [P]),
        "soap_set_host_async": (i32, [P, ctypes.c_int]),
        "soap_inject_bisectors": (i32, [P, P, P, i32, P, P, i32, ctypes.c_int]),
        "soap_set_facula_limb_brightening": (i32, [P, ctypes.c_int]),
        "soap_set_ccf_tensor_cores": (i32, [P, ctypes.c_int]),
        "soap_evolve_radii": (i32, [ctypes.POINTER(soap_region_evolution), ctypes.POINTER(soap_region), i32, P, i32, P]),
        "soap_active_phases_radii": (i32, [P, ctypes.POINTER(soap_region), i32, P, i32, P, u32, i32, P, ctypes.c_int]),
        "soap_set_instrument_resolution": (i32, [P, d]),
        "soap_lower_resolution": (i32, [P, P, P, i32, i32, ctypes.c_int]),
        "soap_active_rv": (i32, [P, ctypes.POINTER(soap_region), i32, P, i32, u32, i32, P, P, i32, d, d, d,
                                 i32, P, P, ctypes.c_int]),
        "soap_get_star_info": (i32, [P, ctypes.POINTER(soap_star_info)]),
        "soap_quiet_spectrum": (i32, [P, i32, i32, P, ctypes.c_int]),
        "soap_active_phases": (i32, [P, ctypes.POINTER(soap_region), i32, P, i32, u32, i32, P, ctypes.c_int]),
        "soap_rv_ccf": (i32, [P, P, i32, i32, ctypes.c_int, P, P, i32, d, d, d, i32, P, P, P, ctypes.c_int]),
        "soap_get_launch_count": (i32, [P, ctypes.POINTER(ctypes.c_uint64)]),
        "soap_debug_inject_timeout": (i32, [P]),
        "soap_rv_ccf_static": (i32, [d, d, i64, P, i32, i32, P, P, i32, d, d, d, i32, P, P, P, P]),
        "soap_active_batch": (i32, [P, ctypes.POINTER(soap_batch_item), i32, ctypes.POINTER(soap_region), i32,
                                    P, i32, i32, P, P, ctypes.c_int]),
        "soap_batch_set_rv": (i32, [P, P, P, i32, d, d, d, i32, d, i32]),
        "soap_batch_num_variants": (i32, [ctypes.POINTER(i32)]),
        "soap_batch_variant_info": (i32, [i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "soap_batch_set_variant": (i32, [P, i32]),
        "soap_batch_get_variant": (i32, [P, ctypes.POINTER(i32)]),
        "soap_batch_autotune": (i32, [P, ctypes.POINTER(soap_batch_item), i32, ctypes.POINTER(soap_region), i32,
                                      P, i32, P, i32, P, ctypes.POINTER(i32)]),
        "soap_gemm_bf16_tn": (i32, [i32, i32, i32, P, i64, P, i64, P, i32, P, i64, P]),
        "soap_surrogate_create": (i32, [ctypes.POINTER(soap_surrogate_desc), P, ctypes.POINTER(P)]),
        "soap_surrogate_num_params": (i32, [P, ctypes.POINTER(i64)]),
        "soap_surrogate_set_params": (i32, [P, P]),
        "soap_surrogate_get_params": (i32, [P, P]),
        "soap_surrogate_set_scaling": (i32, [P, P, P]),
        "soap_surrogate_gradients": (i32, [P, P, P, i32, P, ctypes.POINTER(d), P]),
        "soap_surrogate_train": (i32, [P, P, P, i64, i32, P, P, i32, ctypes.c_uint64, P]),
        "soap_surrogate_predict": (i32, [P, P, i64, ctypes.c_float, P, P, P]),
        "soap_surrogate_set_basis": (i32, [P, P, P, i64]),
        "soap_surrogate_set_error_net": (i32, [P, P]),
        "soap_surrogate_reconstruct": (i32, [P, P, i64, P]),
        "soap_surrogate_query": (i32, [P, P, i64, ctypes.c_float, P, P, P]),
        "soap_surrogate_free": (None, [P]),
        "soap_pca_fit": (i32, [P, i64, i64, P, i32, i32, i32, P, P, P, P]),
        "soap_axpy_f32": (i32, [i64, ctypes.c_float, P, P, P]),
        "soap_surrogate_encode": (i32, [P, i64, P, P]),
        "soap_pca_project": (i32, [P, i64, i64, P, P, i32, P, P]),
        "soap_free": (None, [P]),
        "soap_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status: int, where: str):
    if status != SOAP_OK:
        raise SoapError(status, where, _lib.soap_last_error().decode())


def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), 0
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(None)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------------------
# entry points (same names as the C-ABI)
# ---------------------------------------------------------------------------------------
def star_desc(star) -> soap_star_desc:
    mus = np.ascontiguousarray(star.mu_values, dtype=np.float64)
    d = soap_star_desc(grid_n=int(star.grid_n), n_mu=int(mus.size), n_px=int(star.n_px),
                       vsini_kms=float(star.vsini_kms), incl_deg=float(star.incl_deg),
                       u1=float(star.u1), u2=float(star.u2),
                       diff_rot_alpha=float(getattr(star, "diff_rot_alpha", 0.0)),
                       lambda_start_A=float(star.lambda_start_A), lambda_end_A=float(star.lambda_end_A),
                       t_quiet_K=float(getattr(star, "t_quiet_K", 5778.0)),
                       mu_values=mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    d._keep = mus
    return d


def soap_init_star(star, quiet_local, stream=None) -> ctypes.c_void_p:
    """Create a context; quiet_local [n_mu, n_px] float64 (numpy or CUDA tensor)."""
    d = star_desc(star)
    ptr, dev = _ptr(quiet_local)
    out = ctypes.c_void_p()
    _check(_lib.soap_init_star(ctypes.byref(d), ptr, dev, _stream_handle(stream), ctypes.byref(out)),
           "soap_init_star")
    return out


def soap_update_star(ctx, star) -> None:
    d = star_desc(star)
    _check(_lib.soap_update_star(ctx, ctypes.byref(d)), "soap_update_star")


def _is_f32(a) -> bool:
    return str(a.dtype).endswith("float32")


def soap_set_quiet_spectrum(ctx, quiet_local) -> None:
    """float64 local spectra, or float32 ones (SOAP_FP32 path only)."""
    ptr, dev = _ptr(quiet_local)
    if _is_f32(quiet_local):
        _check(_lib.soap_set_quiet_spectrum_f32(ctx, ptr, dev), "soap_set_quiet_spectrum_f32")
    else:
        _check(_lib.soap_set_quiet_spectrum(ctx, ptr, dev), "soap_set_quiet_spectrum")


def soap_set_profiling(ctx, enabled: bool) -> None:
    _check(_lib.soap_set_profiling(ctx, int(bool(enabled))), "soap_set_profiling")


def soap_get_kernel_time(ctx, timer: int):
    """(total device ms, launches) of one timer since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(_lib.soap_get_kernel_time(ctx, int(timer), ctypes.byref(ms), ctypes.byref(n)),
           "soap_get_kernel_time")
    return float(ms.value), int(n.value)


def soap_reset_kernel_times(ctx) -> None:
    _check(_lib.soap_reset_kernel_times(ctx), "soap_reset_kernel_times")


def soap_set_active_spectrum(ctx, type_: int, active_local) -> None:
    """float64 active local spectra, or float32 ones (SOAP_FP32 path only)."""
    ptr, dev = _ptr(active_local)
    if _is_f32(active_local):
        _check(_lib.soap_set_active_spectrum_f32(ctx, int(type_), ptr, dev), "soap_set_active_spectrum_f32")
    else:
        _check(_lib.soap_set_active_spectrum(ctx, int(type_), ptr, dev), "soap_set_active_spectrum")


def soap_set_stream(ctx, stream) -> None:
    _check(_lib.soap_set_stream(ctx, _stream_handle(stream)), "soap_set_stream")


def soap_synchronize(ctx) -> None:
    _check(_lib.soap_synchronize(ctx), "soap_synchronize")


def soap_get_star_info(ctx) -> soap_star_info:
    info = soap_star_info()
    _check(_lib.soap_get_star_info(ctx, ctypes.byref(info)), "soap_get_star_info")
    return info


def soap_quiet_spectrum(ctx, form: int, precision: int, out) -> None:
    ptr, dev = _ptr(out)
    _check(_lib.soap_quiet_spectrum(ctx, int(form), int(precision), ptr, dev), "soap_quiet_spectrum")


def regions_array(regions: Sequence) -> ctypes.Array:
    arr = (soap_region * max(1, len(regions)))()
    for k, r in enumerate(regions):
        arr[k] = soap_region(type=int(r.type), reserved=0, lat_deg=float(r.lat_deg),
                             lon_deg=float(r.lon_deg), radius_rstar=float(r.radius_rstar),
                             temp_K=float(r.temp_K))
    return arr


def soap_active_phases(ctx, regions: Sequence, phases, effects: int, precision: int, out) -> None:
    arr = regions_array(regions)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    ptr, dev = _ptr(out)
    _check(_lib.soap_active_phases(ctx, arr, len(regions), ctypes.c_void_p(ph.ctypes.data), ph.size,
                                   int(effects), int(precision), ptr, dev), "soap_active_phases")


def soap_set_instrument_resolution(ctx, resolving_power: float) -> None:
    _check(_lib.soap_set_instrument_resolution(ctx, float(resolving_power)), "soap_set_instrument_resolution")


def soap_lower_resolution(ctx, spectra, out) -> None:
    """spectra [n_spec][n_px] (float64 or float32) -> out of the same shape; both host or both device."""
    ip, idev = _ptr(spectra)
    op, odev = _ptr(out)
    if idev != odev:
        raise ValueError("spectra and out must both be host or both device")
    f32 = int(_is_f32(spectra))
    if f32 != int(_is_f32(out)):
        raise ValueError("spectra and out must have the same dtype")
    _check(_lib.soap_lower_resolution(ctx, ip, op, f32, int(spectra.shape[0]), idev), "soap_lower_resolution")


def soap_evolve_radii(evolutions: Sequence[dict], regions: Sequence, times_day) -> np.ndarray:
    """Radii [n_times][n_regions] of evolving regions; evolutions[q] is a dict with 'law' and
    any of area0_msh, rate_msh_per_day, t_peak_day, fwhm_day, asymmetry."""
    n = len(regions)
    evo = (soap_region_evolution * max(1, n))()
    for q, e in enumerate(evolutions):
        evo[q] = soap_region_evolution(law=int(e.get("law", 0)), reserved=0,
                                       area0_msh=float(e.get("area0_msh", 10000.0)),
                                       rate_msh_per_day=float(e.get("rate_msh_per_day", 400.0)),
                                       t_peak_day=float(e.get("t_peak_day", 0.0)),
                                       fwhm_day=float(e.get("fwhm_day", 10.0)),
                                       asymmetry=float(e.get("asymmetry", 0.09)))
    t = np.ascontiguousarray(times_day, dtype=np.float64)
    out = np.empty((t.size, n), np.float64)
    _check(_lib.soap_evolve_radii(evo, regions_array(regions), n, ctypes.c_void_p(t.ctypes.data), t.size,
                                  ctypes.c_void_p(out.ctypes.data)), "soap_evolve_radii")
    return out


def soap_active_phases_radii(ctx, regions: Sequence, phases, radii, effects: int, precision: int, out) -> None:
    arr = regions_array(regions)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    rr = np.ascontiguousarray(radii, dtype=np.float64)
    if rr.shape != (ph.size, len(regions)):
        raise ValueError("radii must be [n_phases][n_regions]")
    ptr, dev = _ptr(out)
    _check(_lib.soap_active_phases_radii(ctx, arr, len(regions), ctypes.c_void_p(ph.ctypes.data), ph.size,
                                         ctypes.c_void_p(rr.ctypes.data), int(effects), int(precision), ptr, dev),
           "soap_active_phases_radii")


def soap_set_facula_limb_brightening(ctx, enabled: bool) -> None:
    _check(_lib.soap_set_facula_limb_brightening(ctx, int(bool(enabled))), "soap_set_facula_limb_brightening")


def soap_set_ccf_tensor_cores(ctx, enabled: bool) -> None:
    _check(_lib.soap_set_ccf_tensor_cores(ctx, int(bool(enabled))), "soap_set_ccf_tensor_cores")


def soap_inject_bisectors(ctx, spectra, out, bis_table, orig_table) -> None:
    """spectra, out [n_rows][n_px] float64 (both host or both device); bis_table [n_rows][n_depth],
    orig_table [n_depth] in km/s."""
    ip, idev = _ptr(spectra)
    op, odev = _ptr(out)
    if idev != odev:
        raise ValueError("spectra and out must both be host or both device")
    bt = np.ascontiguousarray(bis_table, dtype=np.float64)
    ot = np.ascontiguousarray(orig_table, dtype=np.float64)
    if bt.ndim != 2 or bt.shape[0] != spectra.shape[0] or bt.shape[1] != ot.size:
        raise ValueError("bis_table must be [n_rows][n_depth] with n_depth = len(orig_table)")
    _check(_lib.soap_inject_bisectors(ctx, ip, op, int(spectra.shape[0]), ctypes.c_void_p(bt.ctypes.data),
                                      ctypes.c_void_p(ot.ctypes.data), ot.size, idev), "soap_inject_bisectors")


def soap_set_host_async(ctx, enabled: bool) -> None:
    _check(_lib.soap_set_host_async(ctx, int(bool(enabled))), "soap_set_host_async")


def soap_active_rv(ctx, regions: Sequence, phases, effect: int, precision: int, mask_lambda,
                   mask_weight, mask_width_kms: float, v_lo: float, v_step: float, n_v: int,
                   spectra_out, rv_out) -> None:
    """Spectra of one effect and their RVs; spectra_out (or None) and rv_out both host or both
    device."""
    arr = regions_array(regions)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    ml = np.ascontiguousarray(mask_lambda, dtype=np.float64)
    mw = np.ascontiguousarray(mask_weight, dtype=np.float64)
    rp, rdev = _ptr(rv_out)
    sp, sdev = _ptr(spectra_out)
    if spectra_out is not None and sdev != rdev:
        raise ValueError("spectra_out and rv_out must both be host or both device")
    _check(_lib.soap_active_rv(ctx, arr, len(regions), ctypes.c_void_p(ph.ctypes.data), ph.size,
                               int(effect), int(precision), ctypes.c_void_p(ml.ctypes.data),
                               ctypes.c_void_p(mw.ctypes.data), ml.size, float(mask_width_kms),
                               float(v_lo), float(v_step), int(n_v), sp, rp, rdev), "soap_active_rv")


def soap_rv_ccf(ctx, spectra, mask_lambda, mask_weight, mask_width_kms: float, v_lo: float,
                v_step: float, n_v: int, rv_out, fit_out=None, ccf_out=None,
                tensor_cores: bool = False) -> None:
    """spectra [n_spec, n_px] float64/float32; outputs all host (numpy) or all device.
    tensor_cores: float32 spectra only, the CCF as a BF16-split tcgen05 GEMM (spectra_f32 = 2)."""
    sp, sdev = _ptr(spectra)
    f32 = int(str(spectra.dtype).endswith("float32"))
    if tensor_cores:
        if not f32:
            raise ValueError("tensor_cores needs float32 spectra")
        f32 = 2
    n_spec = int(spectra.shape[0])
    ml = np.ascontiguousarray(mask_lambda, dtype=np.float64)
    mw = np.ascontiguousarray(mask_weight, dtype=np.float64)
    rp, rdev = _ptr(rv_out)
    fp, fdev = _ptr(fit_out)
    cp, cdev = _ptr(ccf_out)
    if fit_out is not None and fdev != rdev or ccf_out is not None and cdev != rdev:
        raise ValueError("rv_out, fit_out and ccf_out must all be host or all device")
    _check(_lib.soap_rv_ccf(ctx, sp, f32, n_spec, sdev, ctypes.c_void_p(ml.ctypes.data),
                            ctypes.c_void_p(mw.ctypes.data), ml.size, float(mask_width_kms),
                            float(v_lo), float(v_step), int(n_v), rp, fp, cp, rdev), "soap_rv_ccf")


def soap_rv_ccf_static(lambda_start_A: float, lambda_end_A: float, n_px: int, spectra,
                       mask_lambda, mask_weight, mask_width_kms: float, v_lo: float,
                       v_step: float, n_v: int, rv_out, fit_out=None, ccf_out=None,
                       stream=None) -> None:
    """Allocation-free CCF + RV fit (no context); every array must be a CUDA tensor."""
    arrays = [spectra, mask_lambda, mask_weight, rv_out] + [a for a in (fit_out, ccf_out) if a is not None]
    for a in arrays:
        if not (hasattr(a, "is_cuda") and a.is_cuda):
            raise ValueError("soap_rv_ccf_static takes device arrays only")
    sp, _ = _ptr(spectra)
    f32 = int(str(spectra.dtype).endswith("float32"))
    ml, _ = _ptr(mask_lambda)
    mw, _ = _ptr(mask_weight)
    rp, _ = _ptr(rv_out)
    fp, _ = _ptr(fit_out)
    cp, _ = _ptr(ccf_out)
    _check(_lib.soap_rv_ccf_static(float(lambda_start_A), float(lambda_end_A), int(n_px), sp, f32,
                                   int(spectra.shape[0]), ml, mw, int(mask_lambda.shape[0]),
                                   float(mask_width_kms), float(v_lo), float(v_step), int(n_v),
                                   rp, fp, cp, _stream_handle(stream)), "soap_rv_ccf_static")


def batch_items_array(items: Sequence) -> ctypes.Array:
    """items: (vsini_kms, incl_deg, first_region, n_regions, first_phase, n_phases) tuples."""
    arr = (soap_batch_item * max(1, len(items)))()
    for k, t in enumerate(items):
        v, inc, fr, nr, fp, npp = t
        arr[k] = soap_batch_item(vsini_kms=float(v), incl_deg=float(inc), first_region=int(fr),
                                 n_regions=int(nr), first_phase=int(fp), n_phases=int(npp))
    return arr


def _batch_rv_ptr(out, rv_out):
    if rv_out is None:
        return None
    rp, rdev = _ptr(rv_out)
    if rdev != _ptr(out)[1]:
        raise ValueError("out and rv_out must both be host or both device")
    return rp


def soap_active_batch(ctx, items: Sequence, regions: Sequence, phases, out,
                      output: int = 0, rv_out=None) -> None:
    """out: float32 [n_phases, n_px], host (numpy) or device (torch); output SOAP_BATCH_SPECTRUM
    (F) or SOAP_BATCH_RESIDUAL (F - F_q); rv_out: float64 [n_phases] RVs (km/s) of the spectra,
    in the same memory space as out (needs soap_batch_set_rv)."""
    ia = batch_items_array(items)
    ra = regions_array(regions)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    ptr, dev = _ptr(out)
    rp = _batch_rv_ptr(out, rv_out)
    _check(_lib.soap_active_batch(ctx, ia, len(items), ra, len(regions), ctypes.c_void_p(ph.ctypes.data),
                                  ph.size, int(output), ptr, rp, dev), "soap_active_batch")


def soap_batch_set_rv(ctx, mask_lambda, mask_weight, mask_width_kms: float, v_lo: float, v_step: float,
                      n_v: int, fit_margin_kms: float = 20.0, tensor_cores: bool = False) -> None:
    """Mask and common velocity grid of the batched RVs; each configuration fits the grid
    velocities with |v| <= |vsini| + fit_margin_kms (the whole grid when fit_margin_kms <= 0)."""
    ml = np.ascontiguousarray(mask_lambda, dtype=np.float64)
    mw = np.ascontiguousarray(mask_weight, dtype=np.float64)
    _check(_lib.soap_batch_set_rv(ctx, ctypes.c_void_p(ml.ctypes.data), ctypes.c_void_p(mw.ctypes.data), ml.size,
                                  float(mask_width_kms), float(v_lo), float(v_step), int(n_v),
                                  float(fit_margin_kms), int(bool(tensor_cores))), "soap_batch_set_rv")


ITEM_DTYPE = np.dtype([("vsini_kms", "<f8"), ("incl_deg", "<f8"), ("first_region", "<i4"),
                       ("n_regions", "<i4"), ("first_phase", "<i4"), ("n_phases", "<i4")])
REGION_DTYPE = np.dtype([("type", "<i4"), ("reserved", "<i4"), ("lat_deg", "<f8"), ("lon_deg", "<f8"),
                         ("radius_rstar", "<f8"), ("temp_K", "<f8")])
assert ITEM_DTYPE.itemsize == ctypes.sizeof(soap_batch_item)
assert REGION_DTYPE.itemsize == ctypes.sizeof(soap_region)


def batch_columns_arrays(cols):
    """Structured item / region arrays (the C layouts) from a dict of numpy columns."""
    it = np.zeros(len(cols["vsini"]), ITEM_DTYPE)
    it["vsini_kms"], it["incl_deg"] = cols["vsini"], cols["incl"]
    it["first_region"], it["n_regions"] = cols["first_region"], cols["n_regions"]
    it["first_phase"], it["n_phases"] = cols["first_phase"], cols["n_phases"]
    rg = np.zeros(len(cols["type"]), REGION_DTYPE)
    rg["type"], rg["lat_deg"], rg["lon_deg"] = cols["type"], cols["lat"], cols["lon"]
    rg["radius_rstar"], rg["temp_K"] = cols["radius"], cols["temp"]
    return it, rg, np.ascontiguousarray(cols["phases"], np.float64)


def soap_active_batch_arrays(ctx, items, regions, phases, out, output: int = 0, rv_out=None) -> None:
    """soap_active_batch with items / regions given as ITEM_DTYPE / REGION_DTYPE arrays."""
    items = np.ascontiguousarray(items, ITEM_DTYPE)
    regions = np.ascontiguousarray(regions, REGION_DTYPE)
    ph = np.ascontiguousarray(phases, np.float64)
    ptr, dev = _ptr(out)
    rvp = _batch_rv_ptr(out, rv_out)
    ip = ctypes.cast(ctypes.c_void_p(items.ctypes.data), ctypes.POINTER(soap_batch_item))
    rp = ctypes.cast(ctypes.c_void_p(regions.ctypes.data), ctypes.POINTER(soap_region))
    _check(_lib.soap_active_batch(ctx, ip, len(items), rp, len(regions), ctypes.c_void_p(ph.ctypes.data),
                                  ph.size, int(output), ptr, rvp, dev), "soap_active_batch")


def soap_batch_num_variants() -> int:
    n = ctypes.c_int32()
    _check(_lib.soap_batch_num_variants(ctypes.byref(n)), "soap_batch_num_variants")
    return int(n.value)


def soap_batch_variant_info(variant: int):
    """(phases per block, pixels per thread) of a variant."""
    pb, r = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.soap_batch_variant_info(int(variant), ctypes.byref(pb), ctypes.byref(r)),
           "soap_batch_variant_info")
    return int(pb.value), int(r.value)


def soap_batch_set_variant(ctx, variant: int) -> None:
    _check(_lib.soap_batch_set_variant(ctx, int(variant)), "soap_batch_set_variant")


def soap_batch_get_variant(ctx) -> int:
    v = ctypes.c_int32()
    _check(_lib.soap_batch_get_variant(ctx, ctypes.byref(v)), "soap_batch_get_variant")
    return int(v.value)


def soap_batch_autotune(ctx, items: Sequence, regions: Sequence, phases, out, reps: int = 3):
    """Times every variant (out: device float32 scratch); returns (best, ms per variant)."""
    ia = batch_items_array(items)
    ra = regions_array(regions)
    ph = np.ascontiguousarray(phases, dtype=np.float64)
    ptr, dev = _ptr(out)
    if not dev:
        raise ValueError("soap_batch_autotune needs a device output buffer")
    ms = np.zeros(soap_batch_num_variants(), dtype=np.float32)
    best = ctypes.c_int32()
    _check(_lib.soap_batch_autotune(ctx, ia, len(items), ra, len(regions), ctypes.c_void_p(ph.ctypes.data),
                                    ph.size, ptr, int(reps), ctypes.c_void_p(ms.ctypes.data),
                                    ctypes.byref(best)), "soap_batch_autotune")
    return int(best.value), ms


def soap_gemm_bf16_tn(A, B, C, bias=None, activation: int = 0, stream=None) -> None:
    """C[:, :N] = act(A @ B.T + bias) on the tensor cores; A [M, K], B [N, K] bfloat16 CUDA
    tensors (row-contiguous, possibly column slices of wider ones), C float32 [M, >= N]."""
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or C.shape[0] != M or C.shape[1] < N:
        raise ValueError("shape mismatch")
    for t in (A, B, C):
        if not t.is_cuda or t.stride(1) != 1:
            raise ValueError("operands must be CUDA tensors with unit column stride")
    _check(_lib.soap_gemm_bf16_tn(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                  ctypes.c_void_p(B.data_ptr()), B.stride(0),
                                  ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
                                  int(activation), ctypes.c_void_p(C.data_ptr()), C.stride(0),
                                  _stream_handle(stream)), "soap_gemm_bf16_tn")


def soap_get_launch_count(ctx) -> int:
    n = ctypes.c_uint64()
    _check(_lib.soap_get_launch_count(ctx, ctypes.byref(n)), "soap_get_launch_count")
    return int(n.value)


def soap_debug_inject_timeout(ctx) -> None:
    """Mark the context's device status word as a timed-out tensor-core wait would (for testing
    error reporting)."""
    _check(_lib.soap_debug_inject_timeout(ctx), "soap_debug_inject_timeout")


def soap_free(ctx) -> None:
    _lib.soap_free(ctx)


def soap_last_error() -> str:
    return _lib.soap_last_error().decode()


# ---------------------------------------------------------------------------------------
# surrogate (device arrays are torch CUDA tensors, host arrays numpy)
# ---------------------------------------------------------------------------------------
def _dev(t, dtype=None):
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda) or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and str(t.dtype) != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


def soap_surrogate_create(in_lo, in_hi, batch: int, stream=None, n_in=8, hidden=256, n_hidden=4,
                          n_coef=128) -> ctypes.c_void_p:
    lo = np.ascontiguousarray(in_lo, np.float32)
    hi = np.ascontiguousarray(in_hi, np.float32)
    d = soap_surrogate_desc(n_in=n_in, hidden=hidden, n_hidden=n_hidden, n_coef=n_coef, batch=int(batch),
                            in_lo=lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                            in_hi=hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    out = ctypes.c_void_p()
    _check(_lib.soap_surrogate_create(ctypes.byref(d), _stream_handle(stream), ctypes.byref(out)),
           "soap_surrogate_create")
    return out


def soap_surrogate_num_params(s) -> int:
    n = ctypes.c_int64()
    _check(_lib.soap_surrogate_num_params(s, ctypes.byref(n)), "soap_surrogate_num_params")
    return int(n.value)


def soap_surrogate_set_params(s, flat) -> None:
    a, p = _host(flat, np.float32)
    _check(_lib.soap_surrogate_set_params(s, p), "soap_surrogate_set_params")


def soap_surrogate_get_params(s) -> np.ndarray:
    out = np.empty(soap_surrogate_num_params(s), np.float32)
    _check(_lib.soap_surrogate_get_params(s, ctypes.c_void_p(out.ctypes.data)), "soap_surrogate_get_params")
    return out


def soap_surrogate_set_scaling(s, coef_mean, coef_std) -> None:
    m, pm = _host(coef_mean, np.float32)
    sd, ps = _host(coef_std, np.float32)
    _check(_lib.soap_surrogate_set_scaling(s, pm, ps), "soap_surrogate_set_scaling")


def soap_surrogate_gradients(s, x, t, w_out):
    """(loss, flat gradients) of one batch; x [n, 8] and t [n, 129] float32 CUDA tensors."""
    w, pw = _host(w_out, np.float32)
    loss = ctypes.c_double()
    g = np.empty(soap_surrogate_num_params(s), np.float32)
    _check(_lib.soap_surrogate_gradients(s, _dev(x, "torch.float32"), _dev(t, "torch.float32"), int(x.shape[0]),
                                         pw, ctypes.byref(loss), ctypes.c_void_p(g.ctypes.data)),
           "soap_surrogate_gradients")
    return float(loss.value), g


def soap_surrogate_train(s, x, t, epochs: int, lr, w_out, stage: int = 0, seed: int = 0) -> np.ndarray:
    lr = np.broadcast_to(np.asarray(lr, np.float32), (int(epochs),))
    lr, plr = _host(lr, np.float32)
    w, pw = _host(w_out, np.float32)
    losses = np.zeros(max(1, int(epochs)), np.float64)
    _check(_lib.soap_surrogate_train(s, _dev(x, "torch.float32"), _dev(t, "torch.float32"), int(x.shape[0]),
                                     int(epochs), plr, pw, int(stage), ctypes.c_uint64(int(seed)),
                                     ctypes.c_void_p(losses.ctypes.data)), "soap_surrogate_train")
    return losses[:int(epochs)]


def soap_surrogate_predict(s, x, rv_err_max_cms: float, coef=None, pred_err=None, accepted=None) -> None:
    _check(_lib.soap_surrogate_predict(s, _dev(x, "torch.float32"), int(x.shape[0]), float(rv_err_max_cms),
                                       _dev(coef), _dev(pred_err), _dev(accepted)), "soap_surrogate_predict")


def soap_surrogate_set_error_net(s, error_net) -> None:
    _check(_lib.soap_surrogate_set_error_net(s, error_net), "soap_surrogate_set_error_net")


def soap_surrogate_set_basis(s, mean, basis) -> None:
    _check(_lib.soap_surrogate_set_basis(s, _dev(mean, "torch.float32"), _dev(basis, "torch.float32"),
                                         int(mean.shape[0])), "soap_surrogate_set_basis")


def soap_surrogate_reconstruct(s, coef, out) -> None:
    _check(_lib.soap_surrogate_reconstruct(s, _dev(coef, "torch.float32"), int(coef.shape[0]),
                                           _dev(out, "torch.float32")), "soap_surrogate_reconstruct")


def soap_surrogate_query(s, x, rv_err_max_cms: float, out, accepted, pred_err=None) -> None:
    _check(_lib.soap_surrogate_query(s, _dev(x, "torch.float32"), int(x.shape[0]), float(rv_err_max_cms),
                                     _dev(out, "torch.float32"), _dev(pred_err), _dev(accepted, "torch.uint8")),
           "soap_surrogate_query")


def soap_surrogate_free(s) -> None:
    _lib.soap_surrogate_free(s)


def soap_pca_fit(X, omega, k: int, n_power: int = 2, stream=None):
    """(mean [p], basis [k, p], singular values [k]) of the rows of X [n, p] (CUDA float32)."""
    import torch
    n, p = X.shape
    l = omega.shape[1]
    mean = torch.empty(p, dtype=torch.float32, device=X.device)
    basis = torch.empty((k, p), dtype=torch.float32, device=X.device)
    sv = np.zeros(k, np.float64)
    _check(_lib.soap_pca_fit(_dev(X, "torch.float32"), n, p, _dev(omega, "torch.float32"), int(l), int(k),
                             int(n_power), _dev(mean), _dev(basis), ctypes.c_void_p(sv.ctypes.data),
                             _stream_handle(stream)), "soap_pca_fit")
    return mean, basis, sv


def soap_surrogate_encode(params, out, stream=None) -> None:
    """Network inputs out [n, 8] of query parameters [n, 8] (CUDA float32 tensors)."""
    if params.shape != out.shape or params.shape[-1] != 8:
        raise ValueError("params and out must both be [n, 8]")
    _check(_lib.soap_surrogate_encode(_dev(params, "torch.float32"), int(params.shape[0]), _dev(out, "torch.float32"),
                                      _stream_handle(stream)), "soap_surrogate_encode")


def soap_axpy_f32(alpha: float, x, y, stream=None) -> None:
    """y += alpha x (CUDA float32 tensors of equal size)."""
    if x.numel() != y.numel():
        raise ValueError("size mismatch")
    _check(_lib.soap_axpy_f32(int(x.numel()), float(alpha), _dev(x, "torch.float32"), _dev(y, "torch.float32"),
                              _stream_handle(stream)), "soap_axpy_f32")


def soap_pca_project(X, mean, basis, out, stream=None) -> None:
    _check(_lib.soap_pca_project(_dev(X, "torch.float32"), X.shape[0], X.shape[1], _dev(mean, "torch.float32"),
                                 _dev(basis, "torch.float32"), basis.shape[0], _dev(out, "torch.float32"),
                                 _stream_handle(stream)), "soap_pca_project")


# ---------------------------------------------------------------------------------------
# convenience: a context that frees itself
# ---------------------------------------------------------------------------------------
class Disk:
    """Owns one soap context (soap_init_star ... soap_free)."""

    def __init__(self, star, quiet_local, active_local: Optional[dict] = None, stream=None):
        self.star = star
        self.ctx = soap_init_star(star, quiet_local, stream)
        for t, a in (active_local or {}).items():
            soap_set_active_spectrum(self.ctx, t, a)

    def close(self):
        if self.ctx:
            soap_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
