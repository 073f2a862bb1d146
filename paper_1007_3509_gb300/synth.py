"""Seeded synthetic inputs shared by the tests, smoke() and bench.py.

This module holds no arithmetic of the method: it only draws random lattices,
fields, material-point states and network weights with numpy, and lists the
workload presets (sizes, seeds, temperatures, material constants) with the
paper passage or workload each one follows.  Both the CUDA path and the CPU
oracle take their inputs from here, so neither feeds the other.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field

import numpy as np

# Elastic constants [MPa] and plasticity constants of Table 1 (nickel).  The
# table prints "C22" for the second modulus; it is read as C12.
TABLE1 = dict(C11=250.8e3, C12=150.0e3, C44=123.5e3, tau0=8.0, taus=122.0, h0=440.0, beta=1000.0)
# Cubic nickel constants [MPa] used by the 2D Moore and 3D workloads.
NI_BJ = dict(C11=246.5e3, C12=147.3e3, C44=124.7e3)


@dataclass
class Workload:
    name: str
    dim: int
    L: tuple
    nbr: int
    G: int
    seed: int
    kT: float
    n_mcs: int
    J: float = 1.0
    orient_kind: int = 0          # 0: one angle about z, 1: SO(3) quaternion
    field: str = "grain_uniform"  # grain_uniform | grain_closed_form | cp
    sigma: float = 100.0          # uniaxial load [MPa] along x
    k_disl: float = 0.05          # dislocation-energy weight of the max Schmid factor [MJ/m^3]
    energy_scale: float = 1.0     # MC energy units (J) per MJ/m^3
    extra: dict = dc_field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(np.prod(self.L))


# The five measured workloads.
W2D_SMALL = Workload("2d-128-nbr4-g64", 2, (128, 128), 4, 64, 1000, 0.5, 100, field="grain_uniform")
W2D_MOORE = Workload("2d-4096-moore8-g1e4", 2, (4096, 4096), 8, 10_000, 1001, 0.6, 1000, orient_kind=1,
                     field="grain_closed_form", sigma=100.0, k_disl=0.05, energy_scale=1.0)
W3D_CP = Workload("3d-512-moore26-g2e5-cp", 3, (512, 512, 512), 26, 200_000, 1002, 0.7, 500, orient_kind=1,
                  field="cp", extra=dict(refresh_every=50, incr_per_refresh=2, e_incr=1e-4, energy_scale=7.0))
W3D_SURROGATE = Workload("3d-1024-moore26-g1e6-surrogate", 3, (1024, 1024, 1024), 26, 1_000_000, 1004, 0.7, 500,
                         orient_kind=1, field="cp",
                         extra=dict(refresh_every=50, incr_per_refresh=2, e_incr=1e-4, energy_scale=7.0,
                                    train_samples=1_000_000, train_seed=3000))


def ensemble_members(R: int = 256, seed: int = 2000):
    """Replica list of the batched ensemble: edge in {64,96,128,192,256}, kT U[0.5,0.9],
    load U[50,200] MPa, 500-20000 grains, one seed per replica (seed + r)."""
    rng = np.random.default_rng(seed)
    edges = rng.choice(np.array([64, 96, 128, 192, 256]), size=R)
    kTs = rng.uniform(0.5, 0.9, size=R)
    loads = rng.uniform(50.0, 200.0, size=R)
    grains = rng.integers(500, 20_001, size=R)
    return [dict(edge=int(edges[r]), kT=float(kTs[r]), sigma=float(loads[r]), G=int(grains[r]), seed=seed + r)
            for r in range(R)]


def random_lattice(shape, Q, seed):
    return np.random.default_rng(seed).integers(0, Q, size=int(np.prod(shape)), dtype=np.int32)


def blocky_lattice(shape, Q, seed, block=4):
    """Random lattice made of constant blocks (many interior sites, like grains)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape)
    coarse = [max(1, (s + block - 1) // block) for s in shape]
    c = rng.integers(0, Q, size=tuple(reversed(coarse)), dtype=np.int32)
    idx = np.ix_(*[np.arange(s) // block for s in reversed(shape)])
    return np.ascontiguousarray(c[idx]).ravel()


def random_field(n, lo, hi, seed):
    """Uniform integer field in [lo, hi] (fixed point units)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n, dtype=np.int32)


def uniform_energies(G, hi, seed):
    """Per-grain stored energy U[0, hi) in MC units (J)."""
    return np.random.default_rng(seed).uniform(0.0, hi, size=G)


def disc_lattice(L, R, inside=1, outside=0):
    x = np.arange(L[0]) - L[0] / 2 + 0.5
    y = np.arange(L[1]) - L[1] / 2 + 0.5
    X, Y = np.meshgrid(x, y)
    return np.where(X * X + Y * Y < R * R, inside, outside).astype(np.int32).ravel()


def half_plane_lattice(L, axis=0):
    shape = tuple(reversed(L))
    idx = np.indices(shape)[len(L) - 1 - axis]
    return (idx >= L[axis] // 2).astype(np.int32).ravel()


def random_quaternions(n, seed):
    q = np.random.default_rng(seed).normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def mlp_init(seed, layers=(11, 64, 64, 64, 2)):
    """He-style initial weights [out, in] and zero biases, FP64."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(layers) - 1):
        params.append(rng.normal(0.0, np.sqrt(2.0 / layers[i]), size=(layers[i + 1], layers[i])))
        params.append(np.zeros(layers[i + 1]))
    return params
