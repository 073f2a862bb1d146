"""Python binding of ``libhmcpotts.so`` (the C ABI in ``include/hmcpotts.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed
through); streams default to torch's current stream.  If the shared library
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


class hp_cp_state(C.Structure):
    _fields_ = [("P", C.c_int64), ("eps_p", C.c_void_p), ("gamma", C.c_void_p), ("g", C.c_void_p)]


_SIGS = {
    "hp_last_error_message": ([], C.c_char_p),
    "hp_version": ([], C.c_char_p),
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
    "hp_mlp_param_count": ([C.POINTER(C.c_int64)], C.c_int),
    "hp_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "hp_mlp_gradients": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
                         C.c_int),
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


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


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
    _check(lib().hp_orientations(int(G), C.c_uint64(seed), int(kind), _ptr(orient), _stream(stream)))


def hp_grain_field(quat, C11, C12, C44, sigma, k_disl, energy_scale, b_out, w_out=None, mmax_out=None,
                   stream=None):
    G = quat.shape[0]
    _check(lib().hp_grain_field(int(G), _ptr(quat), C11, C12, C44, sigma, k_disl, energy_scale, _ptr(b_out),
                                _ptr(w_out), _ptr(mmax_out), _stream(stream)))


def hp_texture(G, kind, orient, counts, bins, hist, stream=None):
    _check(lib().hp_texture(int(G), int(kind), _ptr(orient), _ptr(counts), _ptr(bins), _ptr(hist),
                            _stream(stream)))


def hp_gaussian_field(G, angle, scale, b_out, stream=None):
    _check(lib().hp_gaussian_field(int(G), _ptr(angle), float(scale), _ptr(b_out), _stream(stream)))


def hp_texture_fit(hist):
    """Fit g (degrees) of Eq. (10) to a 90-bin angle histogram (host numpy int64)."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    g, r = C.c_double(0), C.c_double(0)
    _check(lib().hp_texture_fit(h.ctypes.data, int(h.size), C.byref(g), C.byref(r)))
    return g.value, r.value


def hp_philox(seed, ctr, out, stream=None):
    n = ctr.numel() // 4
    _check(lib().hp_philox(C.c_uint64(seed), _ptr(ctr), n, _ptr(out), _stream(stream)))


def hp_mlp_param_count():
    n = C.c_int64(0)
    _check(lib().hp_mlp_param_count(C.byref(n)))
    return n.value


def hp_mlp_forward(params, X, Y, stream=None):
    _check(lib().hp_mlp_forward(_ptr(params), _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)))


def hp_mlp_gradients(params, X, T, grads, loss=None, stream=None):
    _check(lib().hp_mlp_gradients(_ptr(params), _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grads), _ptr(loss),
                                  _stream(stream)))


def hp_mlp_adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().hp_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(step), float(lr), float(beta1),
                             float(beta2), float(eps), _stream(stream)))


def hp_mlp_status():
    v = C.c_int32(0)
    _check(lib().hp_mlp_status(C.byref(v)))
    return v.value


SUR_SCALES = hp_sur_scales(100.0, 1e-3, 0.01, 0.002)


def hp_sur_generate(prm, seed, quat, n_orient, K, n_incr, X, Y, load_out=None, scales=SUR_SCALES, stream=None):
    _check(lib().hp_sur_generate(C.byref(prm), C.c_uint64(seed), _ptr(quat), int(n_orient), int(K), int(n_incr),
                                 C.byref(scales), _ptr(X), _ptr(Y), _ptr(load_out), _stream(stream)))


def hp_sur_field(params, quat, G, load, energy_scale, b_out, e_out=None, scales=SUR_SCALES, stream=None):
    ld = np.ascontiguousarray(load, dtype=np.float32)
    _check(lib().hp_sur_field(_ptr(params), _ptr(quat), int(G), ld.ctypes.data, C.byref(scales),
                              float(energy_scale), _ptr(b_out), _ptr(e_out), _stream(stream)))


def cp_params(C11, C12, C44, tau0, taus, h0, beta, e_incr, energy_scale=1.0, G=None, w_weight=1.0):
    if G is None:
        G = (C11 - C12 + 3.0 * C44) / 5.0
    return hp_cp_params(C11, C12, C44, tau0, taus, h0, beta, G, e_incr, energy_scale, w_weight)


def hp_cp_reset(prm, P, eps_p, gamma, g, stream=None):
    st = hp_cp_state(int(P), _ptr(eps_p), _ptr(gamma), _ptr(g))
    _check(lib().hp_cp_reset(C.byref(prm), C.byref(st), _stream(stream)))


def hp_cp_step(prm, seed, grain, quat, t0, n_incr, eps_p, gamma, g, sigma=None, w=None, erho=None, b=None,
               stream=None):
    st = hp_cp_state(int(grain.numel()), _ptr(eps_p), _ptr(gamma), _ptr(g))
    _check(lib().hp_cp_step(C.byref(prm), C.c_uint64(seed), _ptr(grain), _ptr(quat), C.c_uint32(t0), int(n_incr),
                            C.byref(st), _ptr(sigma), _ptr(w), _ptr(erho), _ptr(b), _stream(stream)))


def hp_sweep_status():
    v = C.c_int32(0)
    _check(lib().hp_sweep_status(C.byref(v)))
    return v.value


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
        _check(lib().hp_bind(self._h, _ptr(q), _ptr(mp)))
        self._keep = [q, mp]

    def hp_init_voronoi(self, orient_kind=ORIENT_ANGLE, orient=None, seed_pos=None, stream=None):
        _check(lib().hp_init_voronoi(self._h, int(orient_kind), _ptr(orient), _ptr(seed_pos), _stream(stream)))

    def hp_init_voronoi_static(self, orient_kind=ORIENT_ANGLE, orient=None, seed_pos=None, stream=None):
        """Same as hp_init_voronoi, with no device allocation (fixed-size static scratch)."""
        _check(lib().hp_init_voronoi_static(self._h, int(orient_kind), _ptr(orient), _ptr(seed_pos),
                                            _stream(stream)))

    def hp_set_field(self, table):
        _check(lib().hp_set_field(self._h, _ptr(table), int(table.numel())))
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

    def hp_grain_counts(self, counts, alive=None, stream=None):
        _check(lib().hp_grain_counts(self._h, _ptr(counts), _ptr(alive), _stream(stream)))
