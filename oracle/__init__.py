"""CPU oracle for the hybrid Monte Carlo method (arXiv 1007.3509).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or executes anything in this package.

The arithmetic lives in ``hmc_oracle.c`` (plain C, FP64 / exact integers) and,
for the surrogate network, in ``mlp.py`` (numpy FP64).  This module only
marshals numpy arrays into the C functions.  Every function cites the passage
of the paper it follows; see the C source for the definitions.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmc_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


class CPParams(C.Structure):
    """Crystal-plasticity constants (Table 1): moduli and stresses in MPa."""
    _fields_ = [("C11", C.c_double), ("C12", C.c_double), ("C44", C.c_double),
                ("tau0", C.c_double), ("taus", C.c_double), ("h0", C.c_double),
                ("beta", C.c_double), ("G", C.c_double), ("e_incr", C.c_double)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _declare(L):
    i32, i64, u32, u64, dbl, f32 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double, C.c_float
    P = C.POINTER
    L.oracle_philox4x32_10.argtypes = [u64, P(u32), P(u32)]
    L.oracle_philox_batch.argtypes = [u64, P(u32), i64, P(u32)]
    L.oracle_threshold_table.argtypes = [dbl, C.c_int, P(u32), i32, P(i32)]
    L.oracle_sweep.argtypes = [C.c_int, P(i64), C.c_int, i32, u64, u32, i32, P(u32), i32,
                               P(i32), P(i32), P(i32), P(i64)]
    L.oracle_sweep_phase_slab.argtypes = [C.c_int, P(i64), C.c_int, i32, u64, u32, C.c_int, P(u32), i32, i64, i64,
                                          P(i32), P(i32), P(i32), P(i64)]
    L.oracle_sweep_aniso.argtypes = [C.c_int, P(i64), C.c_int, u64, u32, i32, P(u32), i32, P(i32), i32, i32, i32,
                                     P(i32), P(u32), P(i32), P(i32), P(i32), P(i64)]
    L.oracle_read_shockley.argtypes = [dbl, dbl, i32, i32, i32, P(i32), P(u32)]
    L.oracle_voronoi_seeds.argtypes = [C.c_int, P(i64), i32, u64, P(i64)]
    L.oracle_voronoi_site.argtypes = [C.c_int, P(i64), i32, P(i64), i64]
    L.oracle_voronoi_site.restype = i32
    L.oracle_voronoi.argtypes = [C.c_int, P(i64), i32, u64, P(i32), P(i64)]
    L.oracle_orientations.argtypes = [i32, u64, C.c_int, P(f32)]
    L.oracle_grain_counts.argtypes = [i64, P(i32), i32, P(i64), P(i32)]
    L.oracle_grain_bins.argtypes = [i32, C.c_int, P(f32), P(i32), P(dbl)]
    L.oracle_mcp_run_strain.argtypes = [P(CPParams), u64, i64, P(i32), P(f32), u32, P(dbl), P(dbl), P(dbl),
                                        P(dbl), P(dbl), P(dbl)]
    L.oracle_directional_modulus.argtypes = [P(dbl), P(dbl)]
    L.oracle_directional_modulus.restype = dbl
    L.oracle_max_schmid.argtypes = [P(dbl)]
    L.oracle_max_schmid.restype = dbl
    L.oracle_loading_axis.argtypes = [P(f32), P(dbl)]
    L.oracle_grain_field.argtypes = [i32, P(f32), P(dbl), dbl, dbl, dbl, P(dbl), P(dbl), P(dbl), P(i32)]
    L.oracle_quantise.argtypes = [i64, P(dbl), P(i32)]
    L.oracle_gaussian_field.argtypes = [i32, P(f32), dbl, P(dbl), P(i32)]
    L.oracle_slip_systems.argtypes = [P(dbl), P(dbl)]
    L.oracle_mcp_increment.argtypes = [P(CPParams), u64, i64, u32, P(f32), P(dbl), P(dbl), P(dbl),
                                       P(dbl), P(dbl), P(i32), P(i32)]
    L.oracle_mcp_probabilities.argtypes = [P(CPParams), u32, P(f32), P(dbl), dbl, P(i32), P(dbl)]
    L.oracle_mcp_run.argtypes = [P(CPParams), u64, i64, P(i32), P(f32), u32, i32, P(dbl), P(dbl),
                                 P(dbl), P(dbl), P(dbl)]
    L.oracle_mcp_energies.argtypes = [P(CPParams), i64, P(dbl), P(dbl), P(dbl), P(dbl)]


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (rc={rc})")


# ----------------------------------------------------------------------------
# RNG: Philox4x32-10 (Salmon et al., SC'11)
# ----------------------------------------------------------------------------
def philox(seed: int, ctr) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (shape (n, 4) uint32) under a 64-bit key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    out = np.empty_like(c)
    lib().oracle_philox_batch(C.c_uint64(seed), _p(c, C.c_uint32), c.shape[0], _p(out, C.c_uint32))
    return out


TAG_SWEEP, TAG_MCP, TAG_VORONOI, TAG_SURROGATE = 0, 1, 2, 3


def counters(unit, step, tag, sub) -> np.ndarray:
    """Counter words (unit lo, unit hi, step, tag<<24 | sub) for arrays of units."""
    unit = np.asarray(unit, dtype=np.uint64)
    c = np.empty(unit.shape + (4,), dtype=np.uint32)
    c[..., 0] = (unit & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    c[..., 1] = (unit >> np.uint64(32)).astype(np.uint32)
    c[..., 2] = np.uint32(step)
    c[..., 3] = np.uint32((tag << 24) | sub)
    return c


# ----------------------------------------------------------------------------
# Metropolis threshold table (Sec. 4)
# ----------------------------------------------------------------------------
def threshold_table(kT: float, zero_rule: int = 0, cap: int = 1 << 16):
    thr = np.zeros(cap, dtype=np.uint32)
    D = C.c_int32(0)
    _check(lib().oracle_threshold_table(float(kT), int(zero_rule), _p(thr, C.c_uint32), cap, C.byref(D)),
           "threshold_table")
    return thr[: D.value + 1].copy(), D.value


# ----------------------------------------------------------------------------
# Potts sweep (Eq. (7), Sec. 4, Sec. 6)
# ----------------------------------------------------------------------------
def sweep(dim, L, nbr, J_fix, seed, sweep0, n_mcs, thr, D, q, b=None, mp=None):
    """Run ``n_mcs`` Monte Carlo steps on copies of (q, b, mp); returns (q, b, mp, flips)."""
    Ls = np.array(list(L) + [1] * (3 - len(L)), dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.int32).copy()
    b = None if b is None else np.ascontiguousarray(b, dtype=np.int32).copy()
    mp = None if mp is None else np.ascontiguousarray(mp, dtype=np.int32).copy()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    flips = C.c_int64(0)
    _check(lib().oracle_sweep(dim, _p(Ls, C.c_int64), nbr, int(J_fix), C.c_uint64(seed), C.c_uint32(sweep0),
                              int(n_mcs), _p(thr, C.c_uint32), int(D), _p(q, C.c_int32), _p(b, C.c_int32),
                              _p(mp, C.c_int32), C.byref(flips)), "sweep")
    return q, b, mp, flips.value


def sweep_aniso(dim, L, nbr, seed, sweep0, n_mcs, thr, D, q, ang, period, bin_w, Jtab, mtab=None, b=None, mp=None):
    """Sweep with misorientation-dependent pair energy and mobility (Eq. (7) with
    J_{q_i,q_n}; see the C source).  Returns (q, b, mp, flips)."""
    Lq = _L3(L)
    q = np.ascontiguousarray(q, dtype=np.int32).copy()
    b = None if b is None else np.ascontiguousarray(b, dtype=np.int32).copy()
    mp = None if mp is None else np.ascontiguousarray(mp, dtype=np.int32).copy()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    ang = np.ascontiguousarray(ang, dtype=np.int32)
    Jtab = np.ascontiguousarray(Jtab, dtype=np.int32)
    mtab = None if mtab is None else np.ascontiguousarray(mtab, dtype=np.uint32)
    fl = np.zeros(1, dtype=np.int64)
    _check(lib().oracle_sweep_aniso(dim, _p(Lq, C.c_int64), nbr, C.c_uint64(seed), C.c_uint32(sweep0), n_mcs,
                                    _p(thr, C.c_uint32), D, _p(ang, C.c_int32), int(period), int(bin_w),
                                    int(Jtab.size), _p(Jtab, C.c_int32), _p(mtab, C.c_uint32), _p(q, C.c_int32),
                                    _p(b, C.c_int32), _p(mp, C.c_int32), _p(fl, C.c_int64)), "sweep_aniso")
    return q, b, mp, int(fl[0])


def read_shockley(J_max, theta_max, bin_w, nbins, unit_per_degree, mobility=False):
    """Read-Shockley energy table (int32, 256 = 1 J) and optionally the mobility table (uint32)."""
    J = np.empty(nbins, dtype=np.int32)
    m = np.empty(nbins, dtype=np.uint32) if mobility else None
    _check(lib().oracle_read_shockley(float(J_max), float(theta_max), int(bin_w), int(nbins), int(unit_per_degree),
                                      _p(J, C.c_int32), _p(m, C.c_uint32)), "read_shockley")
    return J, m


def sweep_phase_slab(dim, L, nbr, J_fix, seed, sweep, colour, thr, D, s0, ns, q, b=None, mp=None):
    """One colour phase on a slab array of (ns + 2) layers (ghosts included), in place."""
    Ls = np.array(list(L) + [1] * (3 - len(L)), dtype=np.int64)
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    flips = C.c_int64(0)
    _check(lib().oracle_sweep_phase_slab(dim, _p(Ls, C.c_int64), nbr, int(J_fix), C.c_uint64(seed), C.c_uint32(sweep),
                                         int(colour), _p(thr, C.c_uint32), int(D), int(s0), int(ns),
                                         _p(q, C.c_int32), _p(b, C.c_int32), _p(mp, C.c_int32), C.byref(flips)),
           "sweep_phase_slab")
    return flips.value


# ----------------------------------------------------------------------------
# Initial polycrystal
# ----------------------------------------------------------------------------
def _L3(L):
    return np.array(list(L) + [1] * (3 - len(L)), dtype=np.int64)


def voronoi_seeds(dim, L, G, seed):
    pos = np.empty(G, dtype=np.int64)
    _check(lib().oracle_voronoi_seeds(dim, _p(_L3(L), C.c_int64), G, C.c_uint64(seed), _p(pos, C.c_int64)),
           "voronoi_seeds")
    return pos


def voronoi_sites(dim, L, pos, sites):
    Ls = _L3(L)
    pos = np.ascontiguousarray(pos, dtype=np.int64)
    f = lib().oracle_voronoi_site
    return np.array([f(dim, _p(Ls, C.c_int64), len(pos), _p(pos, C.c_int64), int(s)) for s in sites],
                    dtype=np.int32)


def voronoi(dim, L, G, seed):
    N = int(np.prod(L))
    q = np.empty(N, dtype=np.int32)
    pos = np.empty(G, dtype=np.int64)
    _check(lib().oracle_voronoi(dim, _p(_L3(L), C.c_int64), G, C.c_uint64(seed), _p(q, C.c_int32),
                                _p(pos, C.c_int64)), "voronoi")
    return q, pos


def orientations(G, seed, kind):
    """kind 0: angle about z; 1: SO(3)-uniform quaternion; 2: quaternion of the kind-0 angle about z."""
    out = np.empty(G * (1 if kind == 0 else 4), dtype=np.float32)
    _check(lib().oracle_orientations(G, C.c_uint64(seed), kind, _p(out, C.c_float)), "orientations")
    return out if kind == 0 else out.reshape(G, 4)


# ----------------------------------------------------------------------------
# Statistics and texture
# ----------------------------------------------------------------------------
def grain_counts(q, G):
    q = np.ascontiguousarray(q, dtype=np.int32).ravel()
    counts = np.empty(G, dtype=np.int64)
    alive = C.c_int32(0)
    _check(lib().oracle_grain_counts(q.size, _p(q, C.c_int32), G, _p(counts, C.c_int64), C.byref(alive)),
           "grain_counts")
    return counts, alive.value


def grain_bins(orient, kind):
    o = np.ascontiguousarray(orient, dtype=np.float32)
    G = o.shape[0]
    bins = np.empty(G * (1 if kind != 1 else 2), dtype=np.int32)
    near = np.empty(G, dtype=np.float64)
    _check(lib().oracle_grain_bins(G, kind, _p(o, C.c_float), _p(bins, C.c_int32), _p(near, C.c_double)),
           "grain_bins")
    return (bins if kind != 1 else bins.reshape(G, 2)), near


def histogram(counts, bins, kind):
    """Area-weighted texture histogram: hist[b] = sum of counts of grains in bin b."""
    if kind != 1:
        h = np.zeros(90, dtype=np.int64)
        np.add.at(h, bins, counts)
    else:
        h = np.zeros(24, dtype=np.int64)
        np.add.at(h, bins[:, 0], counts)
        np.add.at(h, bins[:, 1], counts)
    return h


# ----------------------------------------------------------------------------
# Closed-form energies (Sec. 5)
# ----------------------------------------------------------------------------
def directional_modulus(Cc, d):
    Cc = np.ascontiguousarray(Cc, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    return lib().oracle_directional_modulus(_p(Cc, C.c_double), _p(d, C.c_double))


def max_schmid(d):
    d = np.ascontiguousarray(d, dtype=np.float64)
    return lib().oracle_max_schmid(_p(d, C.c_double))


def loading_axis(quat):
    q = np.ascontiguousarray(quat, dtype=np.float32)
    d = np.empty(3, dtype=np.float64)
    lib().oracle_loading_axis(_p(q, C.c_float), _p(d, C.c_double))
    return d


def grain_field(quat, Cc, sigma, k_disl, energy_scale):
    q = np.ascontiguousarray(quat, dtype=np.float32)
    G = q.shape[0]
    Cc = np.ascontiguousarray(Cc, dtype=np.float64)
    w, mm, e = (np.empty(G) for _ in range(3))
    b = np.empty(G, dtype=np.int32)
    _check(lib().oracle_grain_field(G, _p(q, C.c_float), _p(Cc, C.c_double), float(sigma), float(k_disl),
                                    float(energy_scale), _p(w, C.c_double), _p(mm, C.c_double),
                                    _p(e, C.c_double), _p(b, C.c_int32)), "grain_field")
    return w, mm, e, b


def gaussian_field(angle, scale=1.0):
    """Eq. (9) per grain from its angle: returns (e [J], quantised b)."""
    a = np.ascontiguousarray(angle, dtype=np.float32)
    e = np.empty(a.size)
    b = np.empty(a.size, dtype=np.int32)
    lib().oracle_gaussian_field(a.size, _p(a, C.c_float), float(scale), _p(e, C.c_double), _p(b, C.c_int32))
    return e, b


def quantise(e):
    e = np.ascontiguousarray(e, dtype=np.float64).ravel()
    b = np.empty(e.size, dtype=np.int32)
    lib().oracle_quantise(e.size, _p(e, C.c_double), _p(b, C.c_int32))
    return b


def slip_systems():
    n = np.empty((12, 3)); m = np.empty((12, 3))
    lib().oracle_slip_systems(_p(n, C.c_double), _p(m, C.c_double))
    return n, m


# ----------------------------------------------------------------------------
# Monte Carlo crystal plasticity (Sec. 2, Eqs. (1)-(4), Table 1)
# ----------------------------------------------------------------------------
def cp_params(C11, C12, C44, tau0, taus, h0, beta, e_incr, G=None):
    if G is None:
        G = (C11 - C12 + 3.0 * C44) / 5.0
    return CPParams(C11, C12, C44, tau0, taus, h0, beta, G, e_incr)


def mcp_increment(P, seed, p_index, t, quat, eps_p, gamma):
    """One increment for one point; returns (eps_p, gamma, sigma, near_R, near_tau, chosen, n_cand)."""
    q = np.ascontiguousarray(quat, dtype=np.float32)
    ep = np.ascontiguousarray(eps_p, dtype=np.float64).copy()
    gm = np.array([gamma], dtype=np.float64)
    sg = np.empty(6)
    nR, nT = C.c_double(0), C.c_double(0)
    ch, nc = C.c_int32(0), C.c_int32(0)
    lib().oracle_mcp_increment(C.byref(P), C.c_uint64(seed), int(p_index), C.c_uint32(t), _p(q, C.c_float),
                               _p(ep, C.c_double), _p(gm, C.c_double), _p(sg, C.c_double), C.byref(nR),
                               C.byref(nT), C.byref(ch), C.byref(nc))
    return ep, gm[0], sg, nR.value, nT.value, ch.value, nc.value


def mcp_probabilities(P, t, quat, eps_p, gamma):
    q = np.ascontiguousarray(quat, dtype=np.float32)
    ep = np.ascontiguousarray(eps_p, dtype=np.float64)
    cand = np.empty(12, dtype=np.int32)
    prob = np.empty(12)
    n = lib().oracle_mcp_probabilities(C.byref(P), C.c_uint32(t), _p(q, C.c_float), _p(ep, C.c_double),
                                       float(gamma), _p(cand, C.c_int32), _p(prob, C.c_double))
    return cand[:n].copy(), prob[:n].copy()


def mcp_run(P, seed, grain, quat, t0, n_incr, eps_p, gamma):
    """Run n_incr increments over all points; returns (eps_p, gamma, sigma, near_R, near_tau)."""
    grain = np.ascontiguousarray(grain, dtype=np.int32)
    q = np.ascontiguousarray(quat, dtype=np.float32)
    n = grain.size
    ep = np.ascontiguousarray(eps_p, dtype=np.float64).reshape(n, 6).copy()
    gm = np.ascontiguousarray(gamma, dtype=np.float64).copy()
    sg = np.empty((n, 6))
    nR = np.empty(n); nT = np.empty(n)
    _check(lib().oracle_mcp_run(C.byref(P), C.c_uint64(seed), n, _p(grain, C.c_int32), _p(q, C.c_float),
                                C.c_uint32(t0), int(n_incr), _p(ep, C.c_double), _p(gm, C.c_double),
                                _p(sg, C.c_double), _p(nR, C.c_double), _p(nT, C.c_double)), "mcp_run")
    return ep, gm, sg, nR, nT


def mcp_run_strain(P, seed, grain, quat, t, eps_total, eps_p, gamma):
    """One increment t over all points, point p driven by its own sample-frame
    total strain eps_total[p] (Voigt xx yy zz yz xz xy, tensor components);
    returns (eps_p, gamma, sigma, near_R, near_tau)."""
    grain = np.ascontiguousarray(grain, dtype=np.int32)
    q = np.ascontiguousarray(quat, dtype=np.float32)
    n = grain.size
    et = np.ascontiguousarray(eps_total, dtype=np.float64).reshape(n, 6)
    ep = np.ascontiguousarray(eps_p, dtype=np.float64).reshape(n, 6).copy()
    gm = np.ascontiguousarray(gamma, dtype=np.float64).copy()
    sg = np.empty((n, 6))
    nR = np.empty(n); nT = np.empty(n)
    _check(lib().oracle_mcp_run_strain(C.byref(P), C.c_uint64(seed), n, _p(grain, C.c_int32), _p(q, C.c_float),
                                       C.c_uint32(t), _p(et, C.c_double), _p(ep, C.c_double), _p(gm, C.c_double),
                                       _p(sg, C.c_double), _p(nR, C.c_double), _p(nT, C.c_double)), "mcp_run_strain")
    return ep, gm, sg, nR, nT


def mcp_energies(P, sigma, gamma):
    s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1, 6)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    w = np.empty(g.size); er = np.empty(g.size)
    _check(lib().oracle_mcp_energies(C.byref(P), g.size, _p(s, C.c_double), _p(g, C.c_double),
                                     _p(w, C.c_double), _p(er, C.c_double)), "mcp_energies")
    return w, er


# ----------------------------------------------------------------------------
# Texture fit of Eq. (10) (Sec. 5)
# ----------------------------------------------------------------------------
def folded_centres():
    """1-degree bin centres, angles above 45 degrees folded to negative (Sec. 5)."""
    c = np.arange(90) + 0.5
    return np.where(c > 45.0, c - 90.0, c)


def texture_fit(hist):
    """Least-squares fit of f(phi) = exp(-phi^2/(2g^2))/(g sqrt(2 pi)) to the folded,
    per-degree normalised histogram (scipy.optimize.curve_fit)."""
    from scipy.optimize import curve_fit
    h = np.asarray(hist, dtype=np.float64)
    dens = h / h.sum()
    phi = folded_centres()

    def f(x, g):
        return np.exp(-x * x / (2.0 * g * g)) / (g * np.sqrt(2.0 * np.pi))

    sd = np.sqrt(max(np.sum(dens * phi * phi), 1e-6))
    (g,), _ = curve_fit(f, phi, dens, p0=[sd], bounds=(0.5, 2000.0), xtol=1e-14, ftol=1e-14, gtol=1e-14)
    return float(g)
