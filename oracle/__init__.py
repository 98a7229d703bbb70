"""FP64 CPU oracle of the two-species multi-range pseudo-potential LB model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It wraps the
plain C implementation in ``lb_oracle.c`` (built with gcc on first use) and
shares no code with the GPU library.

Arrays follow the oracle's array-of-sites layout: ``f`` has shape
``(ny, nx, 2, 9)`` (species A = 0, B = 1; D2Q9 direction index last).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_HDR = os.path.join(_HERE, "lb_oracle.h")
_LIB = os.path.join(_HERE, "liblboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into liblboracle.so (gcc, -O2, IEEE semantics)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE",
                               "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``or_params`` (lb_oracle.h)."""
    _fields_ = [
        ("tau", C.c_double * 2), ("Ga", C.c_double * 2), ("Gr", C.c_double * 2),
        ("GX", C.c_double), ("rho0", C.c_double), ("u_wall", C.c_double),
        ("init_amp", C.c_double), ("g_x", C.c_double),
        ("kolmo_amp", C.c_double), ("kolmo_k", C.c_double),
        ("nx", C.c_int32), ("ny", C.c_int32), ("boundary", C.c_int32),
        ("psi_form", C.c_int32), ("force_scheme", C.c_int32),
        ("init_shear", C.c_int32), ("stress_every", C.c_int32),
        ("pad_", C.c_int32), ("stress_t0", C.c_int64),
    ]


class Accum(C.Structure):
    _fields_ = [("sum_bot", C.c_double), ("sum_top", C.c_double),
                ("samples", C.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(Params)
            L.or_velocities.argtypes = [C.POINTER(C.c_int32)] * 2
            L.or_weights.argtypes = [dp, dp]
            L.or_opposite.argtypes = [C.c_int32]
            L.or_opposite.restype = C.c_int32
            L.or_psi.argtypes = [pp, C.c_double]
            L.or_psi.restype = C.c_double
            L.or_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.or_mix64.argtypes = [C.c_uint64]
            L.or_mix64.restype = C.c_uint64
            L.or_uniform.argtypes = [C.c_uint64, C.c_uint64]
            L.or_uniform.restype = C.c_double
            L.or_init_seeded.argtypes = [pp, C.c_uint64, dp]
            L.or_init_fields.argtypes = [pp, dp, dp, dp, dp, dp]
            L.or_moments.argtypes = [pp, dp, dp, dp, dp]
            L.or_forces.argtypes = [pp, dp, dp, dp]
            L.or_forces_interaction.argtypes = [pp, dp, dp, dp]
            L.or_step.argtypes = [pp, dp, dp, C.c_int64, C.POINTER(Accum)]
            L.or_step.restype = C.c_int
            L.or_run.argtypes = [pp, dp, C.c_int64, C.c_int64, C.POINTER(Accum)]
            L.or_run.restype = C.c_int
            L.or_stream_only.argtypes = [pp, dp, C.c_int64]
            L.or_fields.argtypes = [pp, dp, dp, dp, dp, dp]
            L.or_totals.argtypes = [pp, dp, dp]
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(nx, ny, *, Ga, Gr, GX, rho0, tau=(1.0, 1.0), boundary=0, psi_form=0,
                force_scheme=0, u_wall=0.0, init_amp=0.03, init_shear=0,
                g_x=0.0, kolmo_amp=0.0, kolmo_k=0.0, stress_every=1,
                stress_t0=0) -> Params:
    p = Params()
    p.tau[:] = tau
    p.Ga[:] = Ga
    p.Gr[:] = Gr
    p.GX, p.rho0, p.u_wall, p.init_amp = GX, rho0, u_wall, init_amp
    p.g_x, p.kolmo_amp, p.kolmo_k = g_x, kolmo_amp, kolmo_k
    p.nx, p.ny, p.boundary, p.psi_form = nx, ny, boundary, psi_form
    p.force_scheme, p.init_shear = force_scheme, init_shear
    p.stress_every, p.stress_t0 = stress_every, stress_t0
    return p


def velocities():
    cx = (C.c_int32 * 25)()
    cy = (C.c_int32 * 25)()
    lib().or_velocities(cx, cy)
    return np.array(cx[:]), np.array(cy[:])


def weights():
    w = np.zeros(9)
    p = np.zeros(25)
    lib().or_weights(_ptr(w), _ptr(p))
    return w, p


def opposite(i):
    return lib().or_opposite(i)


def psi(P, rho):
    return lib().or_psi(C.byref(P), float(rho))


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().or_feq(float(rho), float(ux), float(uy), _ptr(out))
    return out


def mix64(z):
    return lib().or_mix64(z & (2**64 - 1))


def uniform(seed, idx):
    return lib().or_uniform(seed, idx)


def empty_f(P):
    return np.zeros((P.ny, P.nx, 2, 9))


def init_seeded(P, seed):
    f = empty_f(P)
    lib().or_init_seeded(C.byref(P), seed, _ptr(f))
    return f


def init_fields(P, rhoA, rhoB, ux=None, uy=None):
    f = empty_f(P)
    rhoA = np.ascontiguousarray(rhoA, dtype=np.float64)
    rhoB = np.ascontiguousarray(rhoB, dtype=np.float64)
    ux = None if ux is None else np.ascontiguousarray(ux, dtype=np.float64)
    uy = None if uy is None else np.ascontiguousarray(uy, dtype=np.float64)
    lib().or_init_fields(C.byref(P), _ptr(rhoA), _ptr(rhoB), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def moments(P, f):
    n = P.nx * P.ny
    rho, jx, jy = np.zeros(2 * n), np.zeros(2 * n), np.zeros(2 * n)
    lib().or_moments(C.byref(P), _ptr(f), _ptr(rho), _ptr(jx), _ptr(jy))
    sh = (2, P.ny, P.nx)
    return rho.reshape(sh), jx.reshape(sh), jy.reshape(sh)


def forces(P, rho, interaction_only=False):
    """rho: (2, ny, nx) -> (Fx, Fy), each (2, ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    n = P.nx * P.ny
    Fx, Fy = np.zeros(2 * n), np.zeros(2 * n)
    fn = lib().or_forces_interaction if interaction_only else lib().or_forces
    fn(C.byref(P), _ptr(rho), _ptr(Fx), _ptr(Fy))
    return Fx.reshape(2, P.ny, P.nx), Fy.reshape(2, P.ny, P.nx)


def step(P, f, t=0, acc=None):
    scratch = np.zeros(f.size)
    bad = lib().or_step(C.byref(P), _ptr(f), _ptr(scratch), t,
                        C.byref(acc) if acc is not None else None)
    return bad


def run(P, f, nsteps, t0=0, acc=None):
    """Advance f in place by nsteps; returns 1 if a density went non-finite."""
    return lib().or_run(C.byref(P), _ptr(f), t0, nsteps,
                        C.byref(acc) if acc is not None else None)


def stream_only(P, f, nsteps):
    lib().or_stream_only(C.byref(P), _ptr(f), nsteps)


def fields(P, f):
    n = P.nx * P.ny
    out = [np.zeros(n) for _ in range(4)]
    lib().or_fields(C.byref(P), _ptr(f), *[_ptr(a) for a in out])
    return [a.reshape(P.ny, P.nx) for a in out]


def totals(P, f):
    out = np.zeros(4)
    lib().or_totals(C.byref(P), _ptr(f), _ptr(out))
    return out
