"""Seeded synthetic inputs shaped like the paper's DEM workloads.

This module is the only code shared by the CPU oracle and the GPU library: it
draws positions, charges, clump layouts and batch layouts and contains none of
the multipole method's arithmetic.  Every generator is deterministic in its
seed (NumPy PCG64 unless stated otherwise).

Shapes (the paper prints no input files; its driver directories are not
available, so these recipes stand in for them):

* ``uniform_charges``  - points uniform in a cube with charges +-1, the shape of
  the identical-charged-particles example (Sec. 3.1, uniform in (r, 1-r)^3).
* ``dem_coulomb``      - polydisperse hard spheres packed by random sequential
  addition to a target solid fraction, Gaussian charges (Sec. 3.1 with a
  realistic radius spread; Eq. 3 interaction).
* ``clumps``           - rigid clumps carrying several point charges at random
  body-frame offsets under a random rotation (Sec. 2.3, Sec. 3.2).
* ``plummer``          - a Plummer sphere with lognormal masses, the shape of a
  self-gravitating cloud (Sec. 3.4, Eq. 4).
* ``batched``          - many independent systems of uneven size.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def _rsa_lib():
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        out_dir = os.path.join(_HERE, "_build")
        os.makedirs(out_dir, exist_ok=True)
        so = os.path.join(out_dir, "librsa.so")
        src = os.path.join(_HERE, "rsa.c")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC",
                                   "-shared", src, "-o", tmp, "-lm"])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.rsa_pack.restype = ctypes.c_int
        lib.rsa_pack.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
        _LIB = lib
        return lib


def build() -> None:
    """Compile the RSA packer (host C)."""
    _rsa_lib()


def uniform_charges(n: int, seed: int, lo: float = 0.0, hi: float = 1.0):
    """n points uniform in [lo, hi)^3, charges uniform on {-1, +1}."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(n, 3))
    q = rng.choice(np.array([-1.0, 1.0]), size=n)
    return x, q


def rsa_spheres(n: int, seed: int, phi: float = 0.4, rmin: float = 0.5, rmax: float = 1.5,
                max_attempts: int = 10000, max_restarts: int = 20):
    """Polydisperse hard spheres by random sequential addition.

    Returns (centres [n,3], radii [n], side, achieved solid fraction).  Radii
    are U[rmin, rmax] inserted in descending order with hard walls at 0 and
    side; the side is set so that the solid fraction is ``phi`` and grows by
    1 % per stall (see rsa.c).
    """
    lib = _rsa_lib()
    xyz = np.empty((n, 3), dtype=np.float64)
    rad = np.empty(n, dtype=np.float64)
    side = ctypes.c_double(0.0)
    rc = lib.rsa_pack(n, seed, phi, rmin, rmax, max_attempts, max_restarts,
                      xyz.ctypes.data, rad.ctypes.data, ctypes.byref(side))
    if rc < 0:
        raise RuntimeError(f"rsa_pack failed with code {rc}")
    L = side.value
    frac = float(np.sum(4.0 / 3.0 * np.pi * rad ** 3) / L ** 3)
    return xyz, rad, L, frac


def dem_coulomb(n: int, seed: int, phi: float = 0.4, q_sigma: float = 1e-12):
    """RSA packing (radii U[0.5, 1.5] mm, coordinates in mm) with charges
    q ~ N(0, q_sigma^2) coulombs."""
    xyz, rad, L, frac = rsa_spheres(n, seed, phi=phi)
    rng = np.random.default_rng(seed + 7)
    q = rng.normal(0.0, q_sigma, size=n)
    return xyz, q, {"side_mm": L, "solid_fraction": frac, "radius_mm": rad}


def random_unit_quaternions(rng, m: int):
    """Uniform random rotations: normalised 4-D Gaussian, (w, x, y, z)."""
    g = rng.normal(size=(m, 4))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def quat_rotate(qs, v):
    """Rotate vectors v [m,k,3] by unit quaternions qs [m,4] (Hamilton, w first)."""
    w = qs[:, 0][:, None, None]
    u = qs[:, 1:][:, None, :]
    t = 2.0 * np.cross(u, v)
    return v + w * t + np.cross(u, t)


def clumps(n_clumps: int, seed: int, charges_per_clump: int = 4, spacing: float = 3.0,
           body_radius: float = 1.0, q_sigma: float = 1e-12):
    """Rigid clumps: centres uniform in a cube of side spacing*n_clumps^(1/3),
    ``charges_per_clump`` charges at body offsets uniform in a ball of radius
    ``body_radius`` rotated by a random unit quaternion; charges N(0, q_sigma^2).

    Returns (xyz [n,3], q [n], offsets [n_clumps+1] int64, centres [n_clumps,3]).
    """
    rng = np.random.default_rng(seed)
    side = spacing * n_clumps ** (1.0 / 3.0)
    centres = rng.uniform(0.0, side, size=(n_clumps, 3))
    k = charges_per_clump
    d = rng.normal(size=(n_clumps, k, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    rr = body_radius * rng.uniform(size=(n_clumps, k, 1)) ** (1.0 / 3.0)
    body = d * rr
    quats = random_unit_quaternions(rng, n_clumps)
    world = quat_rotate(quats, body) + centres[:, None, :]
    xyz = world.reshape(-1, 3)
    q = rng.normal(0.0, q_sigma, size=n_clumps * k)
    offsets = np.arange(n_clumps + 1, dtype=np.int64) * k
    return xyz, q, offsets, centres


def plummer(n: int, seed: int, a: float = 1.0, rcut: float = 20.0, mass_sigma: float = 1.0):
    """Plummer sphere of scale ``a`` truncated at ``rcut * a``; masses
    lognormal(0, mass_sigma).  Radius by inverting the cumulative mass
    M(<r) = r^3 / (r^2 + a^2)^(3/2): r = a (X^(-2/3) - 1)^(-1/2)."""
    rng = np.random.default_rng(seed)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.05) + 16
        X = rng.uniform(size=m)
        X = X[X > 0]
        r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = r[r <= rcut * a]
        d = rng.normal(size=(r.shape[0], 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        out = np.concatenate([out, d * r[:, None]], axis=0)
    x = out[:n]
    mass = rng.lognormal(0.0, mass_sigma, size=n)
    return x, mass


def batch_sizes(n_systems: int, seed: int, nmin: int = 10_000, nmax: int = 200_000):
    """System sizes floor(exp(U(ln nmin, ln nmax)))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=n_systems))).astype(np.int64)


def batched(n_systems: int, seed: int, nmin: int = 10_000, nmax: int = 200_000):
    """Independent systems: even ones uniform in the unit cube, odd ones
    Plummer (a = 1, cut at 20); charges +-1.  Returns (xyz, q, offsets)."""
    sizes = batch_sizes(n_systems, seed, nmin, nmax)
    xs, qs = [], []
    for k, nk in enumerate(sizes):
        if k % 2 == 0:
            x, q = uniform_charges(int(nk), seed * 1000 + k)
        else:
            x, _ = plummer(int(nk), seed * 1000 + k)
            q = np.random.default_rng(seed * 1000 + k + 500).choice(np.array([-1.0, 1.0]), size=int(nk))
        xs.append(x)
        qs.append(q)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs), np.concatenate(qs), offsets
