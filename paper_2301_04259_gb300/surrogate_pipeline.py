"""Training and checked querying of the surrogate: the order of libsoap calls.

Every computation is a libsoap call (batched method, PCA, network training and queries, CCF and
RV fit); this module chooses the calls, holds the device buffers (torch CUDA tensors) and does
host bookkeeping on small arrays (normalisation constants, learning-rate schedule, per-query
RV errors).

Stages
  1. residual spectra F - F_q of n_train random queries (soap_active_batch, residual output)
  2. PCA basis of those residuals (soap_pca_fit), coefficients (soap_pca_project), standardised
  3. network trained on (query -> standardised coefficients) (soap_surrogate_train, stage 0)
  4. calibration: for n_cal new queries the plain method's spectra and RVs against the RVs of
     F_q + surrogate residual (soap_rv_ccf); the RV-error head learns log10 of that error
     (stage 1)
  5. queries: soap_surrogate_query; rows not accepted (out of range, or predicted error above
     the threshold) are recomputed by the plain method.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import soap as S
from . import synth

RV_ERR_MAX_CMS = 10.0

# Network inputs: 8 numbers that fix the residual spectrum of a query, computed from its 8
# parameters.  The region's centre at the query's phase, in the observer's frame (x across the
# disk along the rotational velocity gradient, y up, z toward the observer: the same frame and
# angles as the library's region geometry, rigid rotation), replaces latitude, longitude, phase
# and inclination: the spectrum depends on them only through that point (the cells a region
# covers and their velocities vsini * x follow from it), and periodically in longitude and phase.
# Slots: (y, x, radius, spot temperature, z, vsini * x, vsini, facula filling).
NET_LO = np.array([-1.0, -1.0, 0.01, 3800.0, -1.0, -10.0, 1.0, 0.0])
NET_HI = np.array([1.0, 1.0, 0.2, 5600.0, 1.0, 10.0, 10.0, 3.0])


def encode(params) -> np.ndarray:
    """Network inputs (float32 [n, 8]) of query parameters [n, 8] (synth.SURROGATE_INPUTS order),
    on the host in FP64: the statement soap_surrogate_encode (the device form the pipeline uses)
    is tested against."""
    q = np.asarray(params, np.float64)
    lat = np.deg2rad(q[:, 0])
    lon = np.deg2rad(q[:, 1] + 360.0 * q[:, 4])
    inc = np.deg2rad(q[:, 5])
    px = np.cos(lat) * np.sin(lon)
    ps = np.sin(lat)
    pc = np.cos(lat) * np.cos(lon)
    x = np.empty_like(q)
    x[:, 0] = ps * np.sin(inc) - pc * np.cos(inc)
    x[:, 1] = px
    x[:, 2] = q[:, 2]
    x[:, 3] = q[:, 3]
    x[:, 4] = ps * np.cos(inc) + pc * np.sin(inc)
    x[:, 5] = q[:, 6] * px
    x[:, 6] = q[:, 6]
    x[:, 7] = q[:, 7]
    return x.astype(np.float32)


def encode_dev(params_host):
    """Device network inputs [n, 8] of host query parameters (uploaded, then soap_surrogate_encode)."""
    torch = _torch()
    q = torch.from_numpy(np.ascontiguousarray(params_host, np.float32)).to("cuda:0")
    x = torch.empty_like(q)
    S.soap_surrogate_encode(q, x, torch.cuda.current_stream())
    return x


def _torch():
    import torch
    return torch


def plain_residuals(ctx, params, out, output=S.SOAP_BATCH_RESIDUAL) -> None:
    """out[k] = F - F_q (or F) of query k by the batched method."""
    it, rg, ph = S.batch_columns_arrays(synth.surrogate_layout_columns(params))
    S.soap_active_batch_arrays(ctx, it, rg, ph, out, output=output)


def rv_cms(ctx, case, spectra):
    """RVs (cm/s) of device float32 spectra [n, n_px] by CCF + Gaussian fit (velocity grid of the
    largest vsini of the query ranges)."""
    torch = _torch()
    lo, step, nv = synth.velocity_grid(float(synth.SURROGATE_HI[6]))
    rv = torch.empty(spectra.shape[0], dtype=torch.float64, device=spectra.device)
    S.soap_rv_ccf(ctx, spectra, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, step, nv, rv)
    return rv.cpu().numpy() * 1e5


@dataclass
class Surrogate:
    handle: object
    mean: object
    basis: object
    coef_mean: np.ndarray
    coef_std: np.ndarray
    sv: np.ndarray
    accept_thr_cms: float = RV_ERR_MAX_CMS   # threshold on the predicted error, calibrated
    error_net: object = None                     # network predicting the RV error (output 128)
    log: dict = field(default_factory=dict)

    def free(self):
        if self.handle:
            S.soap_surrogate_free(self.handle)
            self.handle = None
        if self.error_net:
            S.soap_surrogate_free(self.error_net)
            self.error_net = None


def _cosine(epochs, lr_max, lr_min):
    e = np.arange(max(1, epochs))
    return lr_min + 0.5 * (lr_max - lr_min) * (1.0 + np.cos(np.pi * e / max(1, epochs)))


def rv_sensitivity(ctx, case, mean, basis, scale, vsini=5.5, incl=60.0):
    """cm/s of RV change per unit of each PCA coefficient (times `scale`), linearised around the
    quiet star at a mid-range vsini: RV(F_q + eps scale_j v_j) - RV(F_q), divided by eps."""
    torch = _torch()
    k, n_px = basis.shape
    q = np.array([[0.0, 0.0, 0.01, 4800.0, 0.5, incl, vsini, 0.0]], np.float32)
    F0 = torch.empty((1, n_px), dtype=torch.float32, device=basis.device)
    q[0, 0] = 0.0
    cols = synth.surrogate_layout_columns(q)
    cols["n_regions"][:] = 0                                  # the quiet star alone
    it, rg, ph = S.batch_columns_arrays(cols)
    S.soap_active_batch_arrays(ctx, it, rg[:0], ph, F0, output=S.SOAP_BATCH_SPECTRUM)
    eps = 0.05
    P = F0.repeat(k + 1, 1)
    for j in range(k):                                        # row j: F0 + eps scale_j v_j
        S.soap_axpy_f32(float(eps * scale[j]), basis[j].contiguous(), P[j])
    S.soap_synchronize(ctx)
    rv = rv_cms(ctx, case, P)
    return (rv[:k] - rv[k]) / eps


def calibrate_threshold(pred, err, limit=RV_ERR_MAX_CMS, miss=0.01, z=2.326):
    """Largest threshold on the predicted error such that, among the calibration queries it
    accepts, the fraction with a true error above `limit` is at most `miss` with one-sided
    confidence ~99%: the Wilson score upper bound (z = 2.326) of the observed fraction must not
    exceed `miss`.  (Taking the largest threshold whose observed fraction is <= miss picks the
    calibration set's luckiest point; new queries then exceed `miss` about half the time.  The
    scan over thresholds is itself a search over many candidates, so a 95% bound (z = 1.645)
    still let held-out queries reach 1.2%.)"""
    order = np.argsort(pred)
    bad = np.cumsum(err[order] > limit).astype(np.float64)
    n = np.arange(1, len(order) + 1, dtype=np.float64)
    p = bad / n
    ub = (p + z * z / (2 * n) + z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n))) / (1 + z * z / n)
    ok = ub <= miss
    if not ok.any():
        return 0.0
    last = np.flatnonzero(ok)[-1]
    return float(pred[order][last])


def train(ctx, case, n_train=200_000, n_cal=32_768, n_err=65_536, epochs=200, err_epochs=150, batch=4096,
          k=128, l=160, n_power=2, seed=0, lr=3e-3, chunk=50_000, rv_weighted=True) -> Surrogate:
    torch = _torch()
    dev = "cuda:0"
    n_px = case.star.n_px
    log = {}
    t0 = time.time()
    x = synth.surrogate_params(seed, n_train)
    R = torch.empty((n_train, n_px), dtype=torch.float32, device=dev)
    for a in range(0, n_train, chunk):
        plain_residuals(ctx, x[a:a + chunk], R[a:a + chunk])
    S.soap_synchronize(ctx)
    log["data_s"] = time.time() - t0
    t0 = time.time()
    omega = torch.from_numpy(synth.gaussian_test_matrix(seed + 1, n_px, l)).to(dev)
    mean, basis, sv = S.soap_pca_fit(R, omega, k, n_power=n_power)
    coef = torch.empty((n_train, k), dtype=torch.float32, device=dev)
    S.soap_pca_project(R, mean, basis, coef)
    del R, omega
    log["pca_s"] = time.time() - t0
    c = coef.double().cpu().numpy()
    cm, cs = c.mean(axis=0), c.std(axis=0)
    cs = np.where(cs > 0, cs, 1.0)
    t = np.zeros((n_train, k + 1), np.float32)
    t[:, :k] = (c - cm) / cs
    del coef
    h = S.soap_surrogate_create(NET_LO, NET_HI, batch)
    model = Surrogate(h, mean, basis, cm.astype(np.float32), cs.astype(np.float32), sv, log=log)
    S.soap_surrogate_set_params(h, synth.surrogate_init(seed + 2))
    S.soap_surrogate_set_scaling(h, model.coef_mean, model.coef_std)
    S.soap_surrogate_set_basis(h, mean, basis)
    w0 = np.zeros(k + 1, np.float32)
    if rv_weighted:
        # squared RV change per standard deviation of each coefficient: the loss is then the
        # linearised RV error (plus a small uniform floor that keeps every component fitted)
        sens = rv_sensitivity(ctx, case, mean, basis, model.coef_std)
        wr = sens.astype(np.float64) ** 2
        wr = wr / wr.sum()
        w0[:k] = (0.9 * wr + 0.1 / k).astype(np.float32)
        log["rv_sens_cms_per_sd"] = sens[:8].tolist()
    else:
        w0[:k] = 1.0 / k
    t0 = time.time()
    xd = encode_dev(x)
    td = torch.from_numpy(t).to(dev)
    log["loss"] = S.soap_surrogate_train(h, xd, td, epochs, _cosine(epochs, lr, lr * 0.02), w0, stage=0,
                                         seed=seed + 3).tolist()
    torch.cuda.synchronize()
    log["train_s"] = time.time() - t0
    log["train_samples_per_s"] = n_train * epochs / max(log["train_s"], 1e-9)
    del xd, td
    # RV-error head: a network of the same shape trained (all layers) on the plain method's
    # errors, by the plain method, of n_err new queries; the acceptance threshold is then calibrated on n_cal more
    t0 = time.time()
    if n_err < batch:
        raise ValueError("n_err must hold at least one training batch")
    xc = synth.surrogate_params(seed + 4, n_err)
    err = plain_rv_errors(ctx, case, model, xc)
    tc = np.zeros((n_err, k + 1), np.float32)
    tc[:, k] = np.log10(err + 0.1)
    w1 = np.zeros(k + 1, np.float32)
    w1[k] = 1.0
    model.error_net = S.soap_surrogate_create(NET_LO, NET_HI, batch)
    S.soap_surrogate_set_params(model.error_net, synth.surrogate_init(seed + 7))
    log["head_loss"] = S.soap_surrogate_train(model.error_net, encode_dev(xc),
                                              torch.from_numpy(tc).to(dev), err_epochs,
                                              _cosine(err_epochs, lr, lr * 0.02), w1, stage=2,
                                              seed=seed + 5).tolist()
    S.soap_surrogate_set_error_net(h, model.error_net)
    xv = synth.surrogate_params(seed + 6, n_cal)
    err_v = plain_rv_errors(ctx, case, model, xv)
    pe = torch.empty(n_cal, dtype=torch.float32, device=dev)
    S.soap_surrogate_predict(h, encode_dev(xv), RV_ERR_MAX_CMS, pred_err=pe)
    model.accept_thr_cms = calibrate_threshold(pe.cpu().numpy(), err_v)
    log["calib_s"] = time.time() - t0
    log["calib_err_cms_median"] = float(np.median(err))
    log["accept_thr_cms"] = model.accept_thr_cms
    return model


def plain_rv_errors(ctx, case, model, x, chunk=8192):
    """|RV(F_q + surrogate residual) - RV(F)| in cm/s for queries x, F from the plain method."""
    torch = _torch()
    dev = "cuda:0"
    n_px = case.star.n_px
    out = []
    for a in range(0, len(x), chunk):
        xa = x[a:a + chunk]
        m = len(xa)
        F = torch.empty((m, n_px), dtype=torch.float32, device=dev)
        Rt = torch.empty_like(F)
        plain_residuals(ctx, xa, F, output=S.SOAP_BATCH_SPECTRUM)
        plain_residuals(ctx, xa, Rt, output=S.SOAP_BATCH_RESIDUAL)
        Rh = torch.empty_like(F)
        acc = torch.empty(m, dtype=torch.uint8, device=dev)
        S.soap_surrogate_query(model.handle, encode_dev(xa), 1e30, Rh, acc)
        S.soap_synchronize(ctx)
        Fh = F.clone()
        S.soap_axpy_f32(-1.0, Rt, Fh)
        S.soap_axpy_f32(1.0, Rh, Fh)
        out.append(np.abs(rv_cms(ctx, case, Fh) - rv_cms(ctx, case, F)))
    return np.concatenate(out) if out else np.zeros(0)


def query(ctx, model, x_host, sink=None, thr_cms=None, chunk=65536):
    """Answer every query: residual spectra F - F_q reconstructed by the surrogate where it is
    accepted, computed by the plain method elsewhere, in chunks of `chunk` spectra.  Each chunk
    is handed to sink(indices, spectra) (host int64 query indices, device [m, n_px]) before the
    buffer is reused.  Returns the acceptance mask (host bool array)."""
    torch = _torch()
    dev = model.basis.device
    n = len(x_host)
    k, n_px = model.basis.shape
    x_dev = encode_dev(x_host)
    coef = torch.empty((n, k), dtype=torch.float32, device=dev)
    acc = torch.empty(n, dtype=torch.uint8, device=dev)
    thr = model.accept_thr_cms if thr_cms is None else thr_cms
    S.soap_surrogate_predict(model.handle, x_dev, thr, coef=coef, accepted=acc)
    a = acc.cpu().numpy().astype(bool)
    ia, ir = np.flatnonzero(a), np.flatnonzero(~a)
    buf = torch.empty((min(chunk, max(n, 1)), n_px), dtype=torch.float32, device=dev)
    if ia.size:
        ca = coef.index_select(0, torch.from_numpy(ia).to(dev))
        for c0 in range(0, ia.size, chunk):
            m = min(chunk, ia.size - c0)
            S.soap_surrogate_reconstruct(model.handle, ca[c0:c0 + m], buf[:m])
            if sink:
                sink(ia[c0:c0 + m], buf[:m])
    for c0 in range(0, ir.size, chunk):
        idx = ir[c0:c0 + chunk]
        plain_residuals(ctx, x_host[idx], buf[:idx.size])
        if sink:
            sink(idx, buf[:idx.size])
    return a


def query_coefficients(ctx, model, x_host, coef_out, thr_cms=None, chunk=65536):
    """Answer every query with the 128 PCA coefficients of its residual spectrum F - F_q: the
    network's where it is accepted, the plain method's residual spectrum projected onto the basis
    elsewhere (the fallback, so every answer meets the acceptance guarantee).  coef_out: device
    [n, 128].  Returns the acceptance mask (host bool array)."""
    torch = _torch()
    dev = model.basis.device
    n = len(x_host)
    k, n_px = model.basis.shape
    x_dev = encode_dev(x_host)
    acc = torch.empty(n, dtype=torch.uint8, device=dev)
    thr = model.accept_thr_cms if thr_cms is None else thr_cms
    S.soap_surrogate_predict(model.handle, x_dev, thr, coef=coef_out, accepted=acc)
    a = acc.cpu().numpy().astype(bool)
    ir = np.flatnonzero(~a)
    if ir.size:
        buf = torch.empty((min(chunk, ir.size), n_px), dtype=torch.float32, device=dev)
        cb = torch.empty((min(chunk, ir.size), k), dtype=torch.float32, device=dev)
        for c0 in range(0, ir.size, chunk):
            idx = ir[c0:c0 + chunk]
            m = idx.size
            plain_residuals(ctx, x_host[idx], buf[:m])
            S.soap_pca_project(buf[:m], model.mean, model.basis, cb[:m])
            coef_out.index_copy_(0, torch.from_numpy(idx).to(dev), cb[:m])
    return a
