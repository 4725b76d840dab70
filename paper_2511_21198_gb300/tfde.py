"""Thin ctypes binding of libtfde (C ABI declared in include/tfde.h).

The functions keep the C names and only marshal arguments: device buffers are
passed as torch CUDA tensors (float64, contiguous) or raw integer addresses,
streams as torch.cuda.Stream, raw cudaStream_t integers or None (the current
torch stream).  Every non-zero status raises TfdeError.  There is no CPU
fallback: a missing library raises at load time.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_float, c_int, c_longlong, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtfde.so")

TFDE_OK, TFDE_EINVAL, TFDE_ENOMEM, TFDE_ECUDA, TFDE_ENOCONV = 0, 1, 2, 3, 4
TFDE_EBREAKDOWN, TFDE_ENAN, TFDE_ETIMEOUT, TFDE_EUNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "TFDE_OK", 1: "TFDE_EINVAL", 2: "TFDE_ENOMEM", 3: "TFDE_ECUDA", 4: "TFDE_ENOCONV",
                5: "TFDE_EBREAKDOWN", 6: "TFDE_ENAN", 7: "TFDE_ETIMEOUT", 8: "TFDE_EUNSUPPORTED"}
TFDE_FP64, TFDE_MIXED = 0, 1
TFDE_OP_A, TFDE_OP_RHS, TFDE_OP_FAST, TFDE_OP_STIFF = 0, 1, 2, 4


class tfde_params(Structure):
    _fields_ = [("n", c_int * 3), ("lo", c_double * 3), ("hi", c_double * 3), ("delta", c_double * 3),
                ("kp", c_double * 3), ("km", c_double * 3), ("dt", c_double)]


class tfde_info(Structure):
    _fields_ = [("iters", c_int), ("restarts", c_int), ("refine_sweeps", c_int), ("fallback", c_int),
                ("relres", c_double), ("relres0", c_double), ("ms", c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tfde_kernel_stats(Structure):
    _fields_ = [("launches", ctypes.c_ulonglong), ("timed", ctypes.c_ulonglong), ("ms", c_double),
                ("bytes", c_double), ("flops", c_double)]


TFDE_KIND_SPLIT, TFDE_KIND_EXACT, TFDE_KIND_CONV, TFDE_KIND_FFT = 0, 1, 2, 3
TFDE_NKINDS = 4


class tfde_spectrum_info(Structure):
    _fields_ = [("steps", c_int), ("sym_min", c_double), ("sym_max", c_double), ("skew_rho", c_double),
                ("varsigma", c_double), ("omega", c_double), ("omega_est", c_double)]


class tfde_tune_entry(Structure):
    _fields_ = [("grouped", c_int), ("kmajor", c_int), ("out_mode", c_int), ("stage_bytes", c_int), ("n", c_int),
                ("tiles", c_longlong), ("grid", c_int), ("stages", c_int), ("us", c_float), ("us_default", c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tfde_stats(Structure):
    _fields_ = [("kernel_launches", ctypes.c_ulonglong), ("kind", tfde_kernel_stats * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TfdeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

EXPORTS = ["tfde_assemble", "tfde_destroy", "tfde_matvec", "tfde_precond", "tfde_pcg", "tfde_pgmres",
           "tfde_cn_step", "tfde_cn_advance", "tfde_set_guess_order", "tfde_source_example2", "tfde_coefficients", "tfde_host_coefficients",
           "tfde_stats_reset", "tfde_stats_get", "tfde_mass_apply_noalloc", "tfde_batch_create", "tfde_batch_destroy",
           "tfde_batch_count", "tfde_batch_set_guess_order", "tfde_batch_set_spectral_inner", "tfde_batch_graph_cycles", "tfde_batch_set_symmetric_pcg", "tfde_batch_pcg_solves", "tfde_batch_pcg_graph_launches", "tfde_batch_grouped_prepares", "tfde_batch_cn_advance", "tfde_cn_advance_host", "tfde_cn_advance_guess", "tfde_cnn_create", "tfde_cnn_destroy",
           "tfde_cnn_set_params", "tfde_cnn_get_params", "tfde_cnn_get_grads", "tfde_cnn_predict", "tfde_cnn_accumulate", "tfde_cnn_predict_hist", "tfde_cnn_accumulate_hist",
           "tfde_cnn_adam_step", "tfde_selftest_wait", "tfde_set_device_loop", "tfde_device_loop_launches", "tfde_set_spectral_inner", "tfde_spectrum", "tfde_tune", "tfde_batch_tune",
           "tfde_tune_get", "tfde_tune_set", "tfde_tune_clear", "tfde_last_error", "tfde_version"]


def load(path: str | None = None):
    """Load the in-tree libtfde.so (raises if it has not been built); `path`
    loads another build of the same library without making it the default."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2511_21198_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp = c_void_p
    sig = {
        "tfde_assemble": ([POINTER(tfde_params), c_int, vp, POINTER(vp)], c_int),
        "tfde_destroy": ([vp], c_int),
        "tfde_matvec": ([vp, c_int, vp, vp, vp], c_int),
        "tfde_precond": ([vp, vp, vp, vp], c_int),
        "tfde_pcg": ([vp, vp, vp, c_double, c_int, POINTER(tfde_info), vp], c_int),
        "tfde_pgmres": ([vp, vp, vp, c_int, c_double, c_int, POINTER(tfde_info), vp], c_int),
        "tfde_cn_step": ([vp, vp, vp, vp, vp, c_double, POINTER(tfde_info), vp], c_int),
        "tfde_cn_advance": ([vp, vp, vp, c_int, c_double, POINTER(tfde_info), vp], c_int),
        "tfde_cn_advance_host": ([vp, vp, vp, vp, vp, c_int, c_double, POINTER(tfde_info), vp], c_int),
        "tfde_set_guess_order": ([vp, c_int], c_int),
        "tfde_source_example2": ([vp, c_double, c_double, vp, vp], c_int),
        "tfde_coefficients": ([vp, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double)], c_int),
        "tfde_host_coefficients": ([POINTER(tfde_params), c_int, POINTER(c_double), POINTER(c_double),
                                    POINTER(c_double), POINTER(c_double)], c_int),
        "tfde_stats_reset": ([c_int], c_int),
        "tfde_stats_get": ([POINTER(tfde_stats)], c_int),
        "tfde_mass_apply_noalloc": ([POINTER(c_int), vp, vp, vp], c_int),
        "tfde_batch_create": ([POINTER(tfde_params), c_int, c_int, vp, POINTER(c_void_p)], c_int),
        "tfde_batch_destroy": ([vp], c_int),
        "tfde_batch_count": ([vp], c_int),
        "tfde_batch_set_guess_order": ([vp, c_int], c_int),
        "tfde_batch_cn_advance": ([vp, POINTER(c_void_p), POINTER(c_void_p), c_int, c_double, POINTER(tfde_info),
                                   vp], c_int),
        "tfde_cn_advance_guess": ([vp, vp, vp, vp, c_int, c_double, POINTER(tfde_info), POINTER(c_int), vp], c_int),
        "tfde_cnn_create": ([POINTER(c_int), POINTER(c_void_p)], c_int),
        "tfde_cnn_destroy": ([vp], c_int),
        "tfde_cnn_set_params": ([vp, POINTER(c_float)], c_int),
        "tfde_cnn_get_params": ([vp, POINTER(c_float)], c_int),
        "tfde_cnn_get_grads": ([vp, POINTER(c_float)], c_int),
        "tfde_cnn_predict": ([vp, vp, vp, POINTER(c_double), vp, vp], c_int),
        "tfde_cnn_accumulate": ([vp, vp, vp, POINTER(c_double), vp, POINTER(c_double), vp], c_int),
        "tfde_cnn_adam_step": ([vp, c_float, vp], c_int),
        "tfde_cnn_predict_hist": ([vp, vp, vp, vp, vp, POINTER(c_double), vp, vp], c_int),
        "tfde_cnn_accumulate_hist": ([vp, vp, vp, vp, vp, POINTER(c_double), vp, POINTER(c_double), vp], c_int),
        "tfde_selftest_wait": ([c_longlong, POINTER(c_int), vp], c_int),
        "tfde_set_device_loop": ([vp, c_int], c_int),
        "tfde_set_spectral_inner": ([vp, c_int], c_int),
        "tfde_device_loop_launches": ([vp], c_longlong),
        "tfde_batch_set_spectral_inner": ([vp, c_int], c_int),
        "tfde_batch_graph_cycles": ([vp], c_longlong),
        "tfde_batch_set_symmetric_pcg": ([vp, c_int], c_int),
        "tfde_batch_pcg_solves": ([vp], c_longlong),
        "tfde_batch_pcg_graph_launches": ([vp], c_longlong),
        "tfde_batch_grouped_prepares": ([vp], c_longlong),
        "tfde_spectrum": ([POINTER(tfde_params), c_int, vp, POINTER(tfde_spectrum_info), vp], c_int),
        "tfde_tune": ([vp, c_int, vp], c_int),
        "tfde_batch_tune": ([vp, c_int, vp], c_int),
        "tfde_tune_get": ([POINTER(tfde_tune_entry), c_int, POINTER(c_int)], c_int),
        "tfde_tune_set": ([POINTER(tfde_tune_entry), c_int], c_int),
        "tfde_tune_clear": ([], c_int),
        "tfde_last_error": ([], c_char_p),
        "tfde_version": ([], c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(st: int, where: str):
    if st != TFDE_OK:
        raise TfdeError(st, where, load().tfde_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(n, delta, kp, km, dt, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> tfde_params:
    if isinstance(n, int):
        n = (n, n, n)
    p = tfde_params()
    for a in range(3):
        p.n[a], p.lo[a], p.hi[a] = int(n[a]), float(lo[a]), float(hi[a])
        p.delta[a], p.kp[a], p.km[a] = float(delta[a]), float(kp[a]), float(km[a])
    p.dt = float(dt)
    return p


def tfde_assemble(params: tfde_params, precision: int = TFDE_FP64, stream=None) -> int:
    h = c_void_p()
    _check(load().tfde_assemble(byref(params), precision, _stream(stream), byref(h)), "tfde_assemble")
    return h.value


def tfde_destroy(prob: int) -> None:
    _check(load().tfde_destroy(prob), "tfde_destroy")


def tfde_matvec(prob: int, op: int, x, y, stream=None) -> None:
    _check(load().tfde_matvec(prob, op, _ptr(x), _ptr(y), _stream(stream)), "tfde_matvec")


def tfde_precond(prob: int, r, z, stream=None) -> None:
    _check(load().tfde_precond(prob, _ptr(r), _ptr(z), _stream(stream)), "tfde_precond")


def tfde_pcg(prob: int, b, x, tol: float, maxit: int, stream=None, check: bool = True) -> tfde_info:
    info = tfde_info()
    st = load().tfde_pcg(prob, _ptr(b), _ptr(x), tol, maxit, byref(info), _stream(stream))
    if check:
        _check(st, "tfde_pcg")
    info.status = st
    return info


def tfde_pgmres(prob: int, b, x, restart: int, tol: float, maxit: int, stream=None,
                check: bool = True) -> tfde_info:
    info = tfde_info()
    st = load().tfde_pgmres(prob, _ptr(b), _ptr(x), restart, tol, maxit, byref(info), _stream(stream))
    if check:
        _check(st, "tfde_pgmres")
    info.status = st
    return info


def tfde_cn_step(prob: int, u_prev, F_half, x0, u_next, tol: float, stream=None,
                 check: bool = True) -> tfde_info:
    info = tfde_info()
    st = load().tfde_cn_step(prob, _ptr(u_prev), _ptr(F_half), _ptr(x0), _ptr(u_next), tol,
                             byref(info), _stream(stream))
    if check:
        _check(st, "tfde_cn_step")
    info.status = st
    return info


def tfde_set_guess_order(prob: int, order: int) -> None:
    _check(load().tfde_set_guess_order(prob, order), "tfde_set_guess_order")


def tfde_batch_set_guess_order(batch: int, order: int) -> None:
    _check(load().tfde_batch_set_guess_order(batch, order), "tfde_batch_set_guess_order")


def tfde_cn_advance(prob: int, u, F_half, restart: bool, tol: float, stream=None, check: bool = True) -> tfde_info:
    info = tfde_info()
    st = load().tfde_cn_advance(prob, _ptr(u), _ptr(F_half), 1 if restart else 0, tol, byref(info), _stream(stream))
    if check:
        _check(st, "tfde_cn_advance")
    info.status = st
    return info


def tfde_source_example2(prob: int, cP: float, cS: float, F, stream=None) -> None:
    _check(load().tfde_source_example2(prob, cP, cS, _ptr(F), _stream(stream)), "tfde_source_example2")


def tfde_coefficients(prob: int, axis: int, n_axis: int):
    """Host copies of (q, lambda_tau, eta) for one axis."""
    q = (c_double * (n_axis + 1))()
    lam = (c_double * n_axis)()
    eta = c_double()
    _check(load().tfde_coefficients(prob, axis, q, lam, byref(eta)), "tfde_coefficients")
    return list(q), list(lam), eta.value


def tfde_host_coefficients(params: tfde_params, axis: int):
    """Host-only (q, lambda_tau, lambda_mass, eta) of one axis; no GPU needed."""
    n = params.n[axis]
    q = (c_double * (n + 1))()
    lt = (c_double * n)()
    lm = (c_double * n)()
    eta = c_double()
    _check(load().tfde_host_coefficients(byref(params), axis, q, lt, lm, byref(eta)), "tfde_host_coefficients")
    return list(q), list(lt), list(lm), eta.value


def tfde_stats_reset(time_tc: bool = False) -> None:
    _check(load().tfde_stats_reset(1 if time_tc else 0), "tfde_stats_reset")


def tfde_stats_get() -> tfde_stats:
    st = tfde_stats()
    _check(load().tfde_stats_get(byref(st)), "tfde_stats_get")
    return st


def tfde_mass_apply_noalloc(n, x, y, stream=None) -> None:
    """y = A_N x through the entry point that allocates nothing (grids of at
    most 2^18 points; the first call on a device must precede stream capture)."""
    dims = (c_int * 3)(*[int(v) for v in n])
    _check(load().tfde_mass_apply_noalloc(dims, _ptr(x), _ptr(y), _stream(stream)), "tfde_mass_apply_noalloc")


def tfde_spectrum(params: tfde_params, steps: int, v0, stream=None) -> tfde_spectrum_info:
    out = tfde_spectrum_info()
    _check(load().tfde_spectrum(byref(params), int(steps), _ptr(v0), byref(out), _stream(stream)), "tfde_spectrum")
    return out


def tfde_set_device_loop(prob: int, enable: bool) -> None:
    _check(load().tfde_set_device_loop(prob, int(bool(enable))), "tfde_set_device_loop")


def tfde_batch_set_spectral_inner(batch: int, enable: bool) -> None:
    _check(load().tfde_batch_set_spectral_inner(batch, int(bool(enable))), "tfde_batch_set_spectral_inner")


def tfde_device_loop_launches(prob: int) -> int:
    return int(load().tfde_device_loop_launches(prob))


def tfde_batch_graph_cycles(batch: int) -> int:
    return int(load().tfde_batch_graph_cycles(batch))


def tfde_batch_set_symmetric_pcg(batch: int, enable: bool) -> None:
    _check(load().tfde_batch_set_symmetric_pcg(batch, int(bool(enable))), "tfde_batch_set_symmetric_pcg")


def tfde_batch_pcg_solves(batch: int) -> int:
    return int(load().tfde_batch_pcg_solves(batch))


def tfde_batch_pcg_graph_launches(batch: int) -> int:
    return int(load().tfde_batch_pcg_graph_launches(batch))


def tfde_batch_grouped_prepares(batch: int) -> int:
    return int(load().tfde_batch_grouped_prepares(batch))


def tfde_set_spectral_inner(prob: int, enable: bool) -> None:
    _check(load().tfde_set_spectral_inner(prob, int(bool(enable))), "tfde_set_spectral_inner")


def tfde_selftest_wait(limit_ns: int, stream=None) -> tuple[int, int]:
    """Run the bounded-wait diagnostic; returns (status, tmem_freed) without
    raising (TFDE_ETIMEOUT is the expected status)."""
    freed = c_int(0)
    st = load().tfde_selftest_wait(int(limit_ns), ctypes.byref(freed), _stream(stream))
    return st, freed.value


def tfde_tune(prob: int, reps: int = 20, stream=None) -> None:
    _check(load().tfde_tune(prob, reps, _stream(stream)), "tfde_tune")


def tfde_batch_tune(batch: int, reps: int = 20, stream=None) -> None:
    _check(load().tfde_batch_tune(batch, reps, _stream(stream)), "tfde_batch_tune")


def tfde_tune_get() -> list[dict]:
    """The autotuner's table as a list of dicts (the tfde_tune_entry fields)."""
    cnt = c_int(0)
    arr = (tfde_tune_entry * 4096)()
    _check(load().tfde_tune_get(arr, 4096, byref(cnt)), "tfde_tune_get")
    return [arr[i].as_dict() for i in range(cnt.value)]


def tfde_tune_set(entries: list[dict]) -> None:
    arr = (tfde_tune_entry * max(len(entries), 1))()
    for i, e in enumerate(entries):
        for k, _ in tfde_tune_entry._fields_:
            setattr(arr[i], k, e[k])
    _check(load().tfde_tune_set(arr, len(entries)), "tfde_tune_set")


def tfde_tune_clear() -> None:
    _check(load().tfde_tune_clear(), "tfde_tune_clear")


def save_tuning(path: str, gpu_name: str) -> None:
    """Write the autotuner's table to a JSON cache, under this GPU's name
    (other GPUs' entries in the file are kept)."""
    import json
    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    cache[gpu_name] = tfde_tune_get()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def load_tuning(path: str, gpu_name: str) -> int:
    """Apply the cached table of this GPU from a JSON cache; returns the
    number of entries applied (0 when the file or the GPU is absent)."""
    import json
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        entries = json.load(f).get(gpu_name, [])
    if entries:
        tfde_tune_set(entries)
    return len(entries)


def tfde_last_error() -> str:
    return load().tfde_last_error().decode()


def tfde_version() -> str:
    return load().tfde_version().decode()


def tfde_batch_create(params_list, restart: int = 20, stream=None) -> int:
    """Batch of independent mixed-precision problems (see tfde_batch_create in tfde.h)."""
    arr = (tfde_params * len(params_list))(*params_list)
    h = c_void_p()
    _check(load().tfde_batch_create(arr, len(params_list), restart, _stream(stream), byref(h)), "tfde_batch_create")
    return h.value


def tfde_batch_destroy(batch: int) -> None:
    _check(load().tfde_batch_destroy(batch), "tfde_batch_destroy")


def tfde_batch_cn_advance(batch: int, u_list, F_list, restart: bool, tol: float, stream=None,
                          check: bool = True) -> list:
    """One in-place CN step of every problem; returns the per-problem tfde_info list."""
    C = len(u_list)
    us = (c_void_p * C)(*[_ptr(u) for u in u_list])
    Fs = None if F_list is None else (c_void_p * C)(*[_ptr(f) for f in F_list])
    infos = (tfde_info * C)()
    st = load().tfde_batch_cn_advance(batch, us, Fs, 1 if restart else 0, tol, infos, _stream(stream))
    if check:
        _check(st, "tfde_batch_cn_advance")
    out = list(infos)
    for i in out:
        i.status = st
    return out


CNN_PARAMS = 4 * (16 * 16 * 27 + 16)


def tfde_cn_advance_host(prob: int, u_host_in, u_host_out, u, F_half, restart: bool, tol: float, stream=None,
                         check: bool = True) -> tfde_info:
    """tfde_cn_advance with the state copied from and to host tensors (CPU,
    page-locked for the copies to overlap the step); u is the device state."""
    info = tfde_info()
    st = load().tfde_cn_advance_host(prob, _ptr(u_host_in), _ptr(u_host_out), _ptr(u), _ptr(F_half),
                                     1 if restart else 0, tol, byref(info), _stream(stream))
    if check:
        _check(st, "tfde_cn_advance_host")
    info.status = st
    return info


def tfde_cn_advance_guess(prob: int, u, F_half, x0, restart: bool, tol: float, stream=None,
                          check: bool = True):
    """Chained CN step starting from x0 when its FP64 residual beats u^{m-1}'s;
    returns (info, used_guess)."""
    info = tfde_info()
    used = c_int(0)
    st = load().tfde_cn_advance_guess(prob, _ptr(u), _ptr(F_half), _ptr(x0), 1 if restart else 0, tol, byref(info),
                                      byref(used), _stream(stream))
    if check:
        _check(st, "tfde_cn_advance_guess")
    info.status = st
    return info, bool(used.value)


def tfde_cnn_create(n) -> int:
    arr = (c_int * 3)(*[int(v) for v in n])
    h = c_void_p()
    _check(load().tfde_cnn_create(arr, byref(h)), "tfde_cnn_create")
    return h.value


def tfde_cnn_destroy(net: int) -> None:
    _check(load().tfde_cnn_destroy(net), "tfde_cnn_destroy")


def _f32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != CNN_PARAMS:
        raise ValueError(f"expected {CNN_PARAMS} parameters, got {a.size}")
    return a


def tfde_cnn_set_params(net: int, params) -> None:
    a = _f32(params)
    _check(load().tfde_cnn_set_params(net, a.ctypes.data_as(POINTER(c_float))), "tfde_cnn_set_params")


def tfde_cnn_get_params(net: int):
    import numpy as np
    a = np.zeros(CNN_PARAMS, dtype=np.float32)
    _check(load().tfde_cnn_get_params(net, a.ctypes.data_as(POINTER(c_float))), "tfde_cnn_get_params")
    return a


def tfde_cnn_get_grads(net: int):
    import numpy as np
    a = np.zeros(CNN_PARAMS, dtype=np.float32)
    _check(load().tfde_cnn_get_grads(net, a.ctypes.data_as(POINTER(c_float))), "tfde_cnn_get_grads")
    return a


def tfde_cnn_predict(net: int, u, dtF, coef, x0, stream=None) -> None:
    c = (c_double * 9)(*[float(v) for v in coef])
    _check(load().tfde_cnn_predict(net, _ptr(u), _ptr(dtF), c, _ptr(x0), _stream(stream)), "tfde_cnn_predict")


def tfde_cnn_accumulate(net: int, u, dtF, coef, u_next, stream=None) -> float:
    c = (c_double * 9)(*[float(v) for v in coef])
    loss = c_double(0.0)
    _check(load().tfde_cnn_accumulate(net, _ptr(u), _ptr(dtF), c, _ptr(u_next), byref(loss), _stream(stream)),
           "tfde_cnn_accumulate")
    return loss.value


def tfde_cnn_predict_hist(net: int, u, u1, u2, dtF, coef, x0, stream=None) -> None:
    c = (c_double * 9)(*[float(v) for v in coef])
    _check(load().tfde_cnn_predict_hist(net, _ptr(u), _ptr(u1), _ptr(u2), _ptr(dtF), c, _ptr(x0), _stream(stream)),
           "tfde_cnn_predict_hist")


def tfde_cnn_accumulate_hist(net: int, u, u1, u2, dtF, coef, u_next, stream=None) -> float:
    c = (c_double * 9)(*[float(v) for v in coef])
    loss = c_double(0.0)
    _check(load().tfde_cnn_accumulate_hist(net, _ptr(u), _ptr(u1), _ptr(u2), _ptr(dtF), c, _ptr(u_next),
                                           byref(loss), _stream(stream)), "tfde_cnn_accumulate_hist")
    return loss.value


def tfde_cnn_adam_step(net: int, lr: float, stream=None) -> None:
    _check(load().tfde_cnn_adam_step(net, lr, _stream(stream)), "tfde_cnn_adam_step")
