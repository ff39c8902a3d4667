"""Shared test helpers: seeded problems built from the synthetic generators
with labels rasterised by the oracle (never by the CUDA path), and a probe
of the device's default memory pool for the tests of allocation-free
calls."""
from __future__ import annotations

import ctypes

import numpy as np

import oracle as O
from paper_2605_20816_gb300 import synth


def power_problem(shape, N, seed, d_gen=1):
    """Grain map of a seeded power diagram (sites U[-1,1]^dim, weights
    U(0,0.05)), labels compacted to the non-empty grains."""
    g = O.Grid(shape)
    y, w = synth.power_params(seed, N, dim=len(shape))
    lab, _ = O.assign(g, N, d_gen, O.theta_from_apd(len(shape), d_gen, y, w))
    lab, N_eff, _ = synth.compact(lab)
    return g, lab.astype(np.int32), N_eff


def poly_problem(shape, N, d, seed, noise=0.0):
    """Grain map of a seeded degree-d polynomial diagram: degree <= 1
    coefficients of a zero-weight power diagram from uniform sites, higher
    coefficients standard normal; optional boundary label noise."""
    dim = len(shape)
    g = O.Grid(shape)
    K = O.K(dim, d)
    y, z = synth.poly_params(seed, N, dim, K)
    th = O.theta_from_apd(dim, d, y, np.zeros(N))
    th[:, dim + 1:] = z[:, dim + 1:]
    lab, gap = O.assign(g, N, d, th)
    if noise > 0:
        lab = synth.boundary_noise(lab, shape, noise, seed + 7)
    lab, N_eff, used = synth.compact(lab)
    return g, lab.astype(np.int32), N_eff, th[used]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# CUmemPool_attribute values of the CUDA driver API
USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8


class DefaultPool:
    """The current device's default stream-ordered memory pool, read through
    the driver API: the pool that the library's stream-ordered scratch comes from."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0
