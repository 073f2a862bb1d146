"""Python binding of ``libhmcpotts.so`` (the C ABI in ``include/hmcpotts.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed
through, after a check that each is a contiguous CUDA tensor of the element
size and at least the length the call reads or writes, since the C ABI cannot
see sizes); streams default to torch's current stream.  If the shared library
has not been built, every call raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmcpotts.so")

HP_OK, HP_ERR_ARG, HP_ERR_CUDA, HP_ERR_OOM, HP_ERR_TIMEOUT, HP_ERR_STATE, HP_ERR_CHECKSUM = 0, -1, -2, -3, -4, -5, -6
FIELD_NONE, FIELD_GRAIN, FIELD_POINT = 0, 1, 2
ORIENT_ANGLE, ORIENT_SO3, ORIENT_ZROT = 0, 1, 2
SWEEP_AUTO, SWEEP_PHASE, SWEEP_FUSED = 0, 1, 2

_lock = threading.Lock()
_lib = None


class HPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class hp_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("L", C.c_int64 * 3), ("nbr", C.c_int32), ("J_fix", C.c_int32),
                ("seed", C.c_uint64), ("n_grains", C.c_int32), ("field_mode", C.c_int32)]


class hp_cp_params(C.Structure):
    _fields_ = [("C11", C.c_double), ("C12", C.c_double), ("C44", C.c_double), ("tau0", C.c_double),
                ("taus", C.c_double), ("h0", C.c_double), ("beta", C.c_double), ("G", C.c_double),
                ("e_incr", C.c_double), ("energy_scale", C.c_double), ("w_weight", C.c_double)]


class hp_sur_scales(C.Structure):
    _fields_ = [("stress", C.c_float), ("strain", C.c_float), ("w", C.c_float), ("erho", C.c_float)]


class hp_stats(C.Structure):
    _fields_ = [("sites", C.c_int64), ("alive", C.c_int64), ("mean_area", C.c_double), ("field_sum", C.c_int64),
                ("mean_field", C.c_double), ("hist_total", C.c_int64), ("families", C.c_double * 4),
                ("mean_mmax", C.c_double)]

    def as_dict(self):
        return {"sites": self.sites, "alive": self.alive, "mean_area": self.mean_area, "field_sum": self.field_sum,
                "mean_field": self.mean_field, "hist_total": self.hist_total, "families": list(self.families),
                "mean_mmax": self.mean_mmax}


class hp_sur_train_params(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int64), ("group", C.c_int32), ("lr", C.c_float),
                ("lr_floor", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("log_every", C.c_int32)]


class hp_elastic_params(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("tol", C.c_double), ("max_iter", C.c_int32), ("start_from_mean", C.c_int32)]


class hp_si_in(C.Structure):
    _fields_ = [("gamma_s", C.c_double), ("m_s", C.c_double), ("l0", C.c_double), ("gamma_mc", C.c_double),
                ("m_mc", C.c_double), ("Delta", C.c_double), ("J", C.c_double), ("tau_mc", C.c_double)]


class hp_si_out(C.Structure):
    _fields_ = [("E0", C.c_double), ("t0", C.c_double), ("seconds_per_mcs", C.c_double), ("b_per_bs", C.c_double)]


class hp_cp_state(C.Structure):
    _fields_ = [("P", C.c_int64), ("eps_p", C.c_void_p), ("gamma", C.c_void_p), ("g", C.c_void_p)]


class hp_det_state(C.Structure):
    _fields_ = [("P", C.c_int64), ("eps_p", C.c_void_p), ("gamma", C.c_void_p)]


_SIGS = {
    "hp_last_error_message": ([], C.c_char_p),
    "hp_version": ([], C.c_char_p),
    "hp_last_error": ([C.c_void_p, C.c_char_p, C.c_size_t], C.c_int),
    "hp_set_spins": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "hp_get_spins": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "hp_measure": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(hp_stats), C.c_void_p, C.c_int32,
                    C.c_void_p], C.c_int),
    "hp_sur_train": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                      C.POINTER(hp_sur_train_params), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_kernel_launches": ([C.POINTER(C.c_uint64)], C.c_int),
    "hp_create": ([C.POINTER(hp_desc), C.POINTER(C.c_void_p)], C.c_int),
    "hp_destroy": ([C.c_void_p], C.c_int),
    "hp_bind": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_init_voronoi": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_init_voronoi_static": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_orientations": ([C.c_int32, C.c_uint64, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "hp_set_field": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "hp_build_threshold_table": ([C.c_double, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "hp_set_threshold_table": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "hp_set_sweep_kernel": ([C.c_void_p, C.c_int32], C.c_int),
    "hp_sweep": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "hp_sweep_variants": ([C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "hp_sweep_status": ([C.POINTER(C.c_int32)], C.c_int),
    "hp_debug_wait_timeout": ([C.c_int32, C.c_int64, C.c_int32, C.c_void_p], C.c_int),
    "hp_set_sweep_variant": ([C.c_void_p, C.c_int32], C.c_int),
    "hp_sweep_autotune": ([C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p], C.c_int),
    "hp_ensemble_create": ([C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "hp_ensemble_destroy": ([C.c_void_p], C.c_int),
    "hp_ensemble_set_variant": ([C.c_void_p, C.c_int32], C.c_int),
    "hp_ensemble_autotune": ([C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p], C.c_int),
    "hp_ensemble_sweep": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "hp_get_sweep_counter": ([C.c_void_p, C.POINTER(C.c_uint64)], C.c_int),
    "hp_set_sweep_counter": ([C.c_void_p, C.c_uint64], C.c_int),
    "hp_grain_counts": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_texture": ([C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_grain_field": ([C.c_int32, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                        C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_gaussian_field": ([C.c_int32, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "hp_texture_fit": ([C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "hp_checkpoint_save": ([C.c_void_p, C.c_char_p, C.c_void_p], C.c_int),
    "hp_checkpoint_load": ([C.c_void_p, C.c_char_p, C.c_void_p], C.c_int),
    "hp_philox": ([C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "hp_cp_reset": ([C.POINTER(hp_cp_params), C.POINTER(hp_cp_state), C.c_void_p], C.c_int),
    "hp_cp_step": ([C.POINTER(hp_cp_params), C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint32, C.c_int32,
                    C.POINTER(hp_cp_state), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_elastic_solve": ([C.POINTER(hp_cp_params), C.POINTER(hp_elastic_params), C.c_void_p, C.c_void_p, C.c_void_p,
                          C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                          C.c_void_p], C.c_int),
    "hp_debug_return_map": ([C.POINTER(hp_cp_params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                             C.c_void_p], C.c_int),
    "hp_det_reset": ([C.POINTER(hp_det_state), C.c_void_p], C.c_int),
    "hp_det_step": ([C.POINTER(hp_cp_params), C.c_void_p, C.c_void_p, C.c_uint32, C.c_int32,
                     C.POINTER(hp_det_state), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_det_step_strain": ([C.POINTER(hp_cp_params), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(hp_det_state), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_cp_step_strain": ([C.POINTER(hp_cp_params), C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                           C.POINTER(hp_cp_state), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_set_anisotropy": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                           C.c_void_p], C.c_int),
    "hp_build_read_shockley": ([C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p],
                               C.c_int),
    "hp_si_links": ([C.POINTER(hp_si_in), C.POINTER(hp_si_out)], C.c_int),
    "hp_angle_units": ([C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "hp_mlp_param_count": ([C.POINTER(C.c_int64)], C.c_int),
    "hp_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "hp_mlp_gradients": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
                         C.c_int),
    "hp_debug_gelu": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_mlp_adam": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_float, C.c_float,
                     C.c_float, C.c_void_p], C.c_int),
    "hp_mlp_status": ([C.POINTER(C.c_int32)], C.c_int),
    "hp_sur_generate": ([C.POINTER(hp_cp_params), C.c_uint64, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                         C.POINTER(hp_sur_scales), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hp_sur_field": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(hp_sur_scales), C.c_double,
                      C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
}


def exported_symbols():
    """Names the binding expects the library to export (all of include/hmcpotts.h)."""
    return sorted(_SIGS)


def lib():
    """Load the CUDA library; raise if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1007_3509_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc):
    if rc != HP_OK:
        raise HPError(rc, lib().hp_last_error_message().decode())


def _dev(t, n, itemsize, what):
    """Device pointer of a buffer the library reads or writes n elements of.

    The C ABI takes raw pointers and cannot see sizes, so a torch tensor is
    checked here: on a CUDA device, contiguous, of the element size the call
    expects, and holding at least n elements.  None passes through (optional
    buffers) and so does an int (a raw device pointer the caller vouches for).
    """
    if t is None or isinstance(t, int):
        return t
    bad = None
    if not getattr(t, "is_cuda", False):
        bad = "needs a CUDA tensor"
    elif not t.is_contiguous():
        bad = "needs a contiguous tensor"
    elif t.element_size() != itemsize:
        bad = f"needs {itemsize}-byte elements, got {t.dtype}"
    elif t.numel() < n:
        bad = f"needs at least {n} elements, got {t.numel()}"
    if bad:
        raise HPError(HP_ERR_ARG, f"{what}: {bad}")
    return t.data_ptr()


def _orient_len(kind, G):
    return G if kind == ORIENT_ANGLE else 4 * G


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _host(a, n, dtype, what):
    """Host pointer of a numpy array or CPU torch tensor of at least n elements
    of `dtype` (contiguous); the array itself is returned too, to be kept alive."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda:
            raise HPError(HP_ERR_ARG, f"{what}: expected a host buffer")
        a = a.numpy()
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"] or a.size < n:
        raise HPError(HP_ERR_ARG, f"{what}: needs a contiguous {np.dtype(dtype).name} host array of >= {n} elements")
    return a.ctypes.data, a


def hp_last_error(n=512) -> str:
    buf = C.create_string_buffer(n)
    _check(lib().hp_last_error(None, buf, n))
    return buf.value.decode()


def version() -> str:
    return lib().hp_version().decode()


def hp_kernel_launches() -> int:
    v = C.c_uint64(0)
    _check(lib().hp_kernel_launches(C.byref(v)))
    return v.value


def hp_build_threshold_table(kT: float, zero_rule: int = 0, cap: int = 1 << 16):
    """Host FP64 Metropolis threshold table; returns (uint32 array of D+1 entries, D)."""
    out = np.zeros(cap, dtype=np.uint32)
    D = C.c_int32(0)
    _check(lib().hp_build_threshold_table(float(kT), int(zero_rule), out.ctypes.data, cap, C.byref(D)))
    return out[: D.value + 1].copy(), D.value


def hp_orientations(G, seed, kind, orient, stream=None):
    o = _dev(orient, _orient_len(kind, G), 4, "hp_orientations orient")
    _check(lib().hp_orientations(int(G), C.c_uint64(seed), int(kind), o, _stream(stream)))


def hp_grain_field(quat, C11, C12, C44, sigma, k_disl, energy_scale, b_out, w_out=None, mmax_out=None,
                   stream=None):
    G = quat.shape[0]
    w = "hp_grain_field"
    _check(lib().hp_grain_field(int(G), _dev(quat, 4 * G, 4, w + " quat"), C11, C12, C44, sigma, k_disl,
                                energy_scale, _dev(b_out, G, 4, w + " b_out"), _dev(w_out, G, 4, w + " w_out"),
                                _dev(mmax_out, G, 4, w + " mmax_out"), _stream(stream)))


def hp_texture(G, kind, orient, counts, bins, hist, stream=None):
    so3 = kind == ORIENT_SO3
    w = "hp_texture"
    _check(lib().hp_texture(int(G), int(kind), _dev(orient, _orient_len(kind, G), 4, w + " orient"),
                            _dev(counts, G, 8, w + " counts"), _dev(bins, 2 * G if so3 else G, 4, w + " bins"),
                            _dev(hist, 24 if so3 else 90, 8, w + " hist"), _stream(stream)))


def hp_gaussian_field(G, angle, scale, b_out, stream=None):
    _check(lib().hp_gaussian_field(int(G), _dev(angle, G, 4, "hp_gaussian_field angle"), float(scale),
                                   _dev(b_out, G, 4, "hp_gaussian_field b_out"), _stream(stream)))


def hp_texture_fit(hist):
    """Fit g (degrees) of Eq. (10) to a 90-bin angle histogram (host numpy int64)."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    g, r = C.c_double(0), C.c_double(0)
    _check(lib().hp_texture_fit(h.ctypes.data, int(h.size), C.byref(g), C.byref(r)))
    return g.value, r.value


def hp_philox(seed, ctr, out, stream=None):
    n = ctr.numel() // 4
    _check(lib().hp_philox(C.c_uint64(seed), _dev(ctr, 4 * n, 4, "hp_philox ctr"), n,
                           _dev(out, 4 * n, 4, "hp_philox out"), _stream(stream)))


_param_count = None


def hp_mlp_param_count():
    global _param_count
    if _param_count is None:
        n = C.c_int64(0)
        _check(lib().hp_mlp_param_count(C.byref(n)))
        _param_count = n.value
    return _param_count


def hp_mlp_forward(params, X, Y, stream=None):
    M, P, w = int(X.shape[0]), hp_mlp_param_count(), "hp_mlp_forward"
    _check(lib().hp_mlp_forward(_dev(params, P, 4, w + " params"), _dev(X, 11 * M, 4, w + " X"), M,
                                _dev(Y, 2 * M, 4, w + " Y"), _stream(stream)))


def hp_mlp_gradients(params, X, T, grads, loss=None, stream=None):
    M, P, w = int(X.shape[0]), hp_mlp_param_count(), "hp_mlp_gradients"
    _check(lib().hp_mlp_gradients(_dev(params, P, 4, w + " params"), _dev(X, 11 * M, 4, w + " X"),
                                  _dev(T, 2 * M, 4, w + " T"), M, _dev(grads, P, 4, w + " grads"),
                                  _dev(loss, 1, 4, w + " loss"), _stream(stream)))


def hp_debug_gelu(z, g, dg, stream=None):
    n, w = int(z.numel()), "hp_debug_gelu"
    _check(lib().hp_debug_gelu(_dev(z, n, 4, w + " z"), n, _dev(g, n, 4, w + " g"), _dev(dg, n, 4, w + " dg"),
                               _stream(stream)))


def hp_mlp_adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    P, w = hp_mlp_param_count(), "hp_mlp_adam"
    _check(lib().hp_mlp_adam(_dev(params, P, 4, w + " params"), _dev(grads, P, 4, w + " grads"),
                             _dev(m, P, 4, w + " m"), _dev(v, P, 4, w + " v"), int(step), float(lr), float(beta1),
                             float(beta2), float(eps), _stream(stream)))


def hp_mlp_status():
    v = C.c_int32(0)
    _check(lib().hp_mlp_status(C.byref(v)))
    return v.value


SUR_SCALES = hp_sur_scales(100.0, 1e-3, 0.01, 0.002)


def hp_sur_generate(prm, seed, quat, n_orient, K, n_incr, X, Y, load_out=None, scales=SUR_SCALES, stream=None):
    rows, w = int(n_orient) * int(n_incr), "hp_sur_generate"
    _check(lib().hp_sur_generate(C.byref(prm), C.c_uint64(seed), _dev(quat, 4 * int(n_orient), 4, w + " quat"),
                                 int(n_orient), int(K), int(n_incr), C.byref(scales), _dev(X, 11 * rows, 4, w + " X"),
                                 _dev(Y, 2 * rows, 4, w + " Y"), _dev(load_out, 7 * int(n_incr), 4, w + " load_out"),
                                 _stream(stream)))


def hp_sur_field(params, quat, G, load, energy_scale, b_out, e_out=None, scales=SUR_SCALES, stream=None):
    ld = np.ascontiguousarray(load, dtype=np.float32)
    if ld.size != 7:
        raise HPError(HP_ERR_ARG, "hp_sur_field: load needs 7 values (stress, slip)")
    w = "hp_sur_field"
    _check(lib().hp_sur_field(_dev(params, hp_mlp_param_count(), 4, w + " params"), _dev(quat, 4 * int(G), 4,
                                                                                         w + " quat"),
                              int(G), ld.ctypes.data, C.byref(scales), float(energy_scale),
                              _dev(b_out, int(G), 4, w + " b_out"), _dev(e_out, int(G), 4, w + " e_out"),
                              _stream(stream)))


def hp_sur_train(params, m, v, X, Y, steps, batch=65536, group=1, lr=2e-3, lr_floor=0.02, beta1=0.9, beta2=0.999,
                 eps=1e-8, step0=0, loss=None, log_every=0, stream=None):
    """Adam training loop of the library (minibatches of whole row groups, cosine
    learning-rate decay); returns the host loss log (numpy float32, may be empty)."""
    M, P, w = int(X.shape[0]), hp_mlp_param_count(), "hp_sur_train"
    tp = hp_sur_train_params(int(steps), int(batch or 0), int(group), float(lr), float(lr_floor), float(beta1),
                             float(beta2), float(eps), int(log_every))
    log = np.zeros(max(1, int(steps) // int(log_every)) if log_every else 1, dtype=np.float32)
    _check(lib().hp_sur_train(_dev(params, P, 4, w + " params"), _dev(m, P, 4, w + " m"), _dev(v, P, 4, w + " v"),
                              _dev(X, 11 * M, 4, w + " X"), _dev(Y, 2 * M, 4, w + " Y"), M, C.byref(tp), int(step0),
                              _dev(loss, 1, 4, w + " loss"), log.ctypes.data if log_every else None,
                              _stream(stream)))
    return log[: int(steps) // int(log_every)] if log_every else log[:0]


def cp_params(C11, C12, C44, tau0, taus, h0, beta, e_incr, energy_scale=1.0, G=None, w_weight=1.0):
    if G is None:
        G = (C11 - C12 + 3.0 * C44) / 5.0
    return hp_cp_params(C11, C12, C44, tau0, taus, h0, beta, G, e_incr, energy_scale, w_weight)


def hp_cp_reset(prm, P, eps_p, gamma, g, stream=None):
    P, w = int(P), "hp_cp_reset"
    st = hp_cp_state(P, _dev(eps_p, 6 * P, 4, w + " eps_p"), _dev(gamma, P, 4, w + " gamma"),
                     _dev(g, P, 4, w + " g"))
    _check(lib().hp_cp_reset(C.byref(prm), C.byref(st), _stream(stream)))


def hp_cp_step(prm, seed, grain, quat, t0, n_incr, eps_p, gamma, g, sigma=None, w=None, erho=None, b=None,
               stream=None):
    P, wh = int(grain.numel()), "hp_cp_step"
    st = hp_cp_state(P, _dev(eps_p, 6 * P, 4, wh + " eps_p"), _dev(gamma, P, 4, wh + " gamma"),
                     _dev(g, P, 4, wh + " g"))
    _check(lib().hp_cp_step(C.byref(prm), C.c_uint64(seed), _dev(grain, P, 4, wh + " grain"),
                            _dev(quat, 0, 4, wh + " quat"), C.c_uint32(t0), int(n_incr), C.byref(st),
                            _dev(sigma, 6 * P, 4, wh + " sigma"), _dev(w, P, 4, wh + " w"),
                            _dev(erho, P, 4, wh + " erho"), _dev(b, P, 4, wh + " b"), _stream(stream)))


def hp_elastic_solve(prm, shape, grain, quat, E, eps, eps_p=None, sigma=None, tol=1e-6, max_iter=200,
                     start_from_mean=True, stream=None):
    """Periodic elastic equilibrium on the grid shape = (nx, ny, nz); eps (device
    float[6 N]) is the initial guess and the solution.  Returns (iterations, last
    relative change)."""
    N = int(np.prod(shape))
    w = "hp_elastic_solve"
    ep = hp_elastic_params((C.c_int32 * 3)(*[int(v) for v in shape]), float(tol), int(max_iter),
                           1 if start_from_mean else 0)
    Ev = (C.c_double * 6)(*[float(v) for v in E])
    it, ch = C.c_int32(0), C.c_double(0)
    G = quat.numel() // 4
    _check(lib().hp_elastic_solve(C.byref(prm), C.byref(ep), _dev(grain, N, 4, w + " grain"),
                                  _dev(quat, 4 * G, 4, w + " quat"), _dev(eps_p, 6 * N, 4, w + " eps_p"), Ev,
                                  _dev(eps, 6 * N, 4, w + " eps"), _dev(sigma, 6 * N, 4, w + " sigma"),
                                  C.byref(it), C.byref(ch), _stream(stream)))
    return it.value, ch.value


def hp_cp_step_strain(prm, seed, grain, quat, t, eps_total, eps_p, gamma, g, sigma=None, w=None, erho=None, b=None,
                      stream=None):
    P = int(grain.numel())
    nm = "hp_cp_step_strain"
    st = hp_cp_state(P, _dev(eps_p, 6 * P, 4, nm + " eps_p"), _dev(gamma, P, 4, nm + " gamma"),
                     _dev(g, P, 4, nm + " g"))
    _check(lib().hp_cp_step_strain(C.byref(prm), C.c_uint64(seed), _dev(grain, P, 4, nm + " grain"),
                                   _dev(quat, quat.numel(), 4, nm + " quat"), C.c_uint32(t),
                                   _dev(eps_total, 6 * P, 4, nm + " eps_total"), C.byref(st),
                                   _dev(sigma, 6 * P, 4, nm + " sigma"), _dev(w, P, 4, nm + " w"),
                                   _dev(erho, P, 4, nm + " erho"), _dev(b, P, 4, nm + " b"), _stream(stream)))


def hp_debug_return_map(prm, at, g, k, x, stream=None):
    n, w = int(at.numel()), "hp_debug_return_map"
    _check(lib().hp_debug_return_map(C.byref(prm), _dev(at, n, 4, w + " at"), _dev(g, n, 4, w + " g"),
                                     _dev(k, n, 8, w + " k"), n, _dev(x, n, 8, w + " x"), _stream(stream)))


def _det_state(P, eps_p, gamma, who):
    return hp_det_state(P, _dev(eps_p, 6 * P, 8, who + " eps_p"), _dev(gamma, P, 8, who + " gamma"))


def hp_det_reset(P, eps_p, gamma, stream=None):
    st = _det_state(int(P), eps_p, gamma, "hp_det_reset")
    _check(lib().hp_det_reset(C.byref(st), _stream(stream)))


def hp_det_step(prm, grain, quat, t0, n_incr, eps_p, gamma, sigma=None, n_active=None, stream=None):
    """Deterministic multi-slip increments t0+1 .. t0+n_incr (FP64 state: eps_p
    double[6 P], gamma double[P]; sigma double[6 P] and n_active int32[P] optional)."""
    P, wh = int(grain.numel()), "hp_det_step"
    st = _det_state(P, eps_p, gamma, wh)
    _check(lib().hp_det_step(C.byref(prm), _dev(grain, P, 4, wh + " grain"), _dev(quat, 0, 4, wh + " quat"),
                             C.c_uint32(t0), int(n_incr), C.byref(st), _dev(sigma, 6 * P, 8, wh + " sigma"),
                             _dev(n_active, P, 4, wh + " n_active"), _stream(stream)))


def hp_det_step_strain(prm, grain, quat, eps_total, eps_p, gamma, sigma=None, n_active=None, stream=None):
    P, wh = int(grain.numel()), "hp_det_step_strain"
    st = _det_state(P, eps_p, gamma, wh)
    _check(lib().hp_det_step_strain(C.byref(prm), _dev(grain, P, 4, wh + " grain"), _dev(quat, 0, 4, wh + " quat"),
                                    _dev(eps_total, 6 * P, 4, wh + " eps_total"), C.byref(st),
                                    _dev(sigma, 6 * P, 8, wh + " sigma"), _dev(n_active, P, 4, wh + " n_active"),
                                    _stream(stream)))


def hp_build_read_shockley(J_max, theta_max, bin_w, nbins, unit_per_degree, mobility=False):
    """Host Read-Shockley tables: (int32 J[nbins] in 256 = 1 J units, uint32 mobility or None)."""
    J = np.zeros(nbins, dtype=np.int32)
    m = np.zeros(nbins, dtype=np.uint32) if mobility else None
    _check(lib().hp_build_read_shockley(float(J_max), float(theta_max), int(bin_w), int(nbins), int(unit_per_degree),
                                        J.ctypes.data, None if m is None else m.ctypes.data))
    return J, m


def hp_angle_units(G, kind, orient, unit_per_degree, period, out, stream=None):
    w = "hp_angle_units"
    _check(lib().hp_angle_units(int(G), int(kind), _dev(orient, _orient_len(kind, G), 4, w + " orient"),
                                int(unit_per_degree), int(period), _dev(out, G, 4, w + " out"), _stream(stream)))


def hp_si_links(gamma_s, m_s, l0, gamma_mc, m_mc, Delta=1.0, J=1.0, tau_mc=1.0):
    """Eq. (8) links: returns dict(E0, t0, seconds_per_mcs, b_per_bs)."""
    i = hp_si_in(gamma_s, m_s, l0, gamma_mc, m_mc, Delta, J, tau_mc)
    o = hp_si_out()
    _check(lib().hp_si_links(C.byref(i), C.byref(o)))
    return {"E0": o.E0, "t0": o.t0, "seconds_per_mcs": o.seconds_per_mcs, "b_per_bs": o.b_per_bs}


def hp_sweep_status():
    v = C.c_int32(0)
    _check(lib().hp_sweep_status(C.byref(v)))
    return v.value


def hp_debug_wait_timeout(unit, limit_cycles, late=True, stream=None):
    """Run the bounded-wait probe of the sweep (unit 0) or surrogate (unit 1) kernels."""
    _check(lib().hp_debug_wait_timeout(int(unit), int(limit_cycles), 1 if late else 0, _stream(stream)))


def hp_sweep_variants(nbr):
    n = C.c_int32(0)
    _check(lib().hp_sweep_variants(int(nbr), C.byref(n)))
    return n.value


class Ensemble:
    """Independent lattices swept together (an ``hp_ensemble``)."""

    def __init__(self, members):
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m._h for m in self.members])
        h = C.c_void_p()
        _check(lib().hp_ensemble_create(arr, len(self.members), C.byref(h)))
        self._h = h
        self.nbr = self.members[0].nbr

    def close(self):
        if self._h:
            lib().hp_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hp_ensemble_set_variant(self, v):
        _check(lib().hp_ensemble_set_variant(self._h, int(v)))

    def hp_ensemble_autotune(self, n_mcs=2, stream=None):
        n = hp_sweep_variants(self.nbr)
        ms = np.zeros(max(n, 1), dtype=np.float32)
        ch = C.c_int32(0)
        _check(lib().hp_ensemble_autotune(self._h, int(n_mcs), ms.ctypes.data, C.byref(ch), _stream(stream)))
        return ch.value, ms

    def hp_ensemble_sweep(self, n_mcs, stream=None):
        _check(lib().hp_ensemble_sweep(self._h, int(n_mcs), _stream(stream)))


class Lattice:
    """One periodic Potts lattice (an ``hp_handle``)."""

    def __init__(self, dim, L, nbr, J_fix, seed, n_grains, field_mode=FIELD_NONE):
        Ls = list(L) + [1] * (3 - len(L))
        d = hp_desc(int(dim), (C.c_int64 * 3)(*Ls), int(nbr), int(J_fix), C.c_uint64(seed), int(n_grains),
                    int(field_mode))
        h = C.c_void_p()
        _check(lib().hp_create(C.byref(d), C.byref(h)))
        self._h = h
        self.dim, self.L, self.nbr, self.N = dim, tuple(L), nbr, int(np.prod(L))
        self.n_grains, self.field_mode = n_grains, field_mode
        self._keep = []

    def close(self):
        if self._h:
            lib().hp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hp_bind(self, q, mp=None):
        _check(lib().hp_bind(self._h, _dev(q, self.N, 4, "hp_bind q"), _dev(mp, self.N, 4, "hp_bind mp")))
        self._keep = [q, mp]

    def _voronoi_out(self, orient_kind, orient, seed_pos, w):
        G = self.n_grains
        return (_dev(orient, _orient_len(orient_kind, G), 4, w + " orient"), _dev(seed_pos, G, 8, w + " seed_pos"))

    def hp_init_voronoi(self, orient_kind=ORIENT_ANGLE, orient=None, seed_pos=None, stream=None):
        o, sp = self._voronoi_out(orient_kind, orient, seed_pos, "hp_init_voronoi")
        _check(lib().hp_init_voronoi(self._h, int(orient_kind), o, sp, _stream(stream)))

    def hp_init_voronoi_static(self, orient_kind=ORIENT_ANGLE, orient=None, seed_pos=None, stream=None):
        """Same as hp_init_voronoi, with no device allocation (fixed-size static scratch)."""
        o, sp = self._voronoi_out(orient_kind, orient, seed_pos, "hp_init_voronoi_static")
        _check(lib().hp_init_voronoi_static(self._h, int(orient_kind), o, sp, _stream(stream)))

    def hp_set_field(self, table):
        _check(lib().hp_set_field(self._h, _dev(table, 0, 4, "hp_set_field table"), int(table.numel())))
        self._table = table

    def hp_set_threshold_table(self, thr, D, stream=None):
        thr = np.ascontiguousarray(thr, dtype=np.uint32)
        _check(lib().hp_set_threshold_table(self._h, thr.ctypes.data, int(D), _stream(stream)))

    def hp_set_sweep_kernel(self, kind):
        _check(lib().hp_set_sweep_kernel(self._h, int(kind)))

    def hp_set_sweep_variant(self, v):
        _check(lib().hp_set_sweep_variant(self._h, int(v)))

    def hp_sweep_autotune(self, n_mcs=4, stream=None):
        """Time every tile variant; returns (chosen, per-variant ms)."""
        n = hp_sweep_variants(self.nbr)
        ms = np.zeros(max(n, 1), dtype=np.float32)
        ch = C.c_int32(0)
        _check(lib().hp_sweep_autotune(self._h, int(n_mcs), ms.ctypes.data, C.byref(ch), _stream(stream)))
        return ch.value, ms

    def hp_sweep(self, n_mcs, stream=None):
        _check(lib().hp_sweep(self._h, int(n_mcs), _stream(stream)))

    def hp_get_sweep_counter(self):
        v = C.c_uint64(0)
        _check(lib().hp_get_sweep_counter(self._h, C.byref(v)))
        return v.value

    def hp_set_sweep_counter(self, v):
        _check(lib().hp_set_sweep_counter(self._h, C.c_uint64(v)))

    def hp_checkpoint_save(self, path, stream=None):
        _check(lib().hp_checkpoint_save(self._h, str(path).encode(), _stream(stream)))

    def hp_checkpoint_load(self, path, stream=None):
        _check(lib().hp_checkpoint_load(self._h, str(path).encode(), _stream(stream)))

    def hp_set_spins(self, q, mp=None, stream=None):
        """Load the lattice state from a host array (numpy / CPU tensor) or a CUDA tensor."""
        self._spins_io(q, mp, stream, "hp_set_spins", lib().hp_set_spins)

    def hp_get_spins(self, q, mp=None, stream=None):
        """Copy the lattice state into a host array (numpy / CPU tensor) or a CUDA tensor."""
        self._spins_io(q, mp, stream, "hp_get_spins", lib().hp_get_spins)

    def _spins_io(self, q, mp, stream, w, fn):
        host = not getattr(q, "is_cuda", False)
        if host:
            pq, keep_q = _host(q, self.N, np.int32, w + " q")
            pm, keep_m = _host(mp, self.N, np.int32, w + " mp") if mp is not None else (None, None)
            self._io_keep = (keep_q, keep_m)
        else:
            pq, pm = _dev(q, self.N, 4, w + " q"), _dev(mp, self.N, 4, w + " mp")
        _check(fn(self._h, pq, pm, 1 if host else 0, _stream(stream)))

    def hp_measure(self, orient_kind=None, orient=None, acc=None, stream=None):
        """Synchronous counts / alive / texture / mean field; returns (hp_stats, hist).
        Pass a previous (hp_stats, hist) as `acc` to add this lattice to it."""
        kind = ORIENT_ANGLE if orient_kind is None else int(orient_kind)
        nb = 0 if orient is None else (24 if kind == ORIENT_SO3 else 90)
        if acc is None:
            st, hist = hp_stats(), np.zeros(max(nb, 1), dtype=np.int64)
        else:
            st, hist = acc
        if hist.size < nb or hist.dtype != np.int64:
            raise HPError(HP_ERR_ARG, "hp_measure: histogram too small")
        o = None if orient is None else _dev(orient, _orient_len(kind, self.n_grains), 4, "hp_measure orient")
        _check(lib().hp_measure(self._h, kind, o, 0 if acc is None else 1, C.byref(st),
                                hist.ctypes.data if nb else None, int(hist.size), _stream(stream)))
        return st, hist

    def hp_set_anisotropy(self, angle, period, bin_w, J, mobility=None, stream=None):
        """Misorientation-dependent pair energy and mobility (angle: CUDA int32[G] or None to clear)."""
        if angle is None:
            _check(lib().hp_set_anisotropy(self._h, None, 0, 0, 0, None, None, _stream(stream)))
            self._aniso = None
            return
        J = np.ascontiguousarray(J, dtype=np.int32)
        m = None if mobility is None else np.ascontiguousarray(mobility, dtype=np.uint32)
        _check(lib().hp_set_anisotropy(self._h, _dev(angle, self.n_grains, 4, "hp_set_anisotropy angle"), int(period),
                                       int(bin_w), int(J.size), J.ctypes.data, None if m is None else m.ctypes.data,
                                       _stream(stream)))
        self._aniso = angle

    def hp_grain_counts(self, counts, alive=None, stream=None):
        _check(lib().hp_grain_counts(self._h, _dev(counts, self.n_grains, 8, "hp_grain_counts counts"),
                                     _dev(alive, 1, 4, "hp_grain_counts alive"), _stream(stream)))
