"""GB300-native two-species multi-range pseudo-potential lattice Boltzmann.

Thin ctypes binding of the C ABI in ``include/lb.h`` (liblbgb.so).  Every
step of the model runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory (the workspace handed to
``lb_create_in``) and the CUDA stream.  There is no CPU fallback: if the
library is missing the import of a function raises ``RuntimeError``.

Model: Benzi, Chibbaro & Succi, "Mesoscopic lattice Boltzmann modeling of
flowing soft systems" (arXiv:0807.4471), Eqs. (1)-(2).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB
_lock = threading.Lock()
_lib = None

LB_OK, LB_ERR_INVALID, LB_ERR_NOMEM, LB_ERR_CUDA = 0, -1, -2, -3
LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE, LB_ERR_UNSUPPORTED = -4, -5, -6, -7
LB_FP64, LB_FP32, LB_FP16_OFFSET, LB_BF16_OFFSET = 0, 1, 2, 3
LB_PERIODIC, LB_COUETTE = 0, 1
LB_PSI_SQRT_RHO0, LB_PSI_RHO0 = 0, 1
LB_FORCE_SHIFT, LB_FORCE_SOURCE = 0, 1
PRECISIONS = {"fp64": LB_FP64, "fp32": LB_FP32, "fp16": LB_FP16_OFFSET, "bf16": LB_BF16_OFFSET}


class lb_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("boundary", C.c_int32),
        ("precision", C.c_int32), ("psi_form", C.c_int32), ("force_scheme", C.c_int32),
        ("init_shear", C.c_int32), ("stress_every", C.c_int32), ("stress_t0", C.c_int64),
        ("tau_A", C.c_double), ("tau_B", C.c_double), ("G_A1", C.c_double),
        ("G_A2", C.c_double), ("G_B1", C.c_double), ("G_B2", C.c_double),
        ("G_X", C.c_double), ("rho0", C.c_double), ("u_wall", C.c_double),
        ("init_amp", C.c_double), ("rho_ref", C.c_double), ("g_x", C.c_double),
        ("kolmo_amp", C.c_double), ("kolmo_k", C.c_double), ("rounding", C.c_int32),
        ("tile_rows", C.c_int32),
    ]


class lb_stress_out(C.Structure):
    _fields_ = [
        ("mass_A", C.c_double), ("mass_B", C.c_double), ("mom_x", C.c_double),
        ("mom_y", C.c_double), ("sigma_bot", C.c_double), ("sigma_top", C.c_double),
        ("sigma_mean", C.c_double), ("nu_eff", C.c_double), ("response_R", C.c_double),
        ("samples", C.c_int64), ("step", C.c_int64),
    ]


class LbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lb_status_string(status)} (status {status})")


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load liblbgb.so (build it first with ``build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA extension {_LIB_PATH} is missing: run "
                               "paper_0807_4471_gb300.build.build() (there is no CPU fallback)")
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(lb_params)
        H = C.c_void_p
        dp = C.POINTER(C.c_double)
        sig = {
            "lb_params_default": (None, [P]),
            "lb_workspace_size": (C.c_int, [P, C.POINTER(C.c_size_t)]),
            "lb_create": (C.c_int, [P, C.c_void_p, C.POINTER(H)]),
            "lb_create_in": (C.c_int, [P, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(H)]),
            "lb_init_seeded": (C.c_int, [H, C.c_uint64]),
            "lb_init_fields": (C.c_int, [H, dp, dp, dp, dp]),
            "lb_init_populations": (C.c_int, [H, dp, C.c_int64]),
            "lb_checkpoint": (C.c_int, [H, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
            "lb_restore": (C.c_int, [H, dp, C.c_int64, C.c_int32]),
            "lb_step": (C.c_int, [H, C.c_int64]),
            "lb_fields": (C.c_int, [H, dp, dp, dp, dp]),
            "lb_populations": (C.c_int, [H, dp]),
            "lb_stress": (C.c_int, [H, C.POINTER(lb_stress_out)]),
            "lb_sync": (C.c_int, [H]),
            "lb_time": (C.c_int64, [H]),
            "lb_destroy": (C.c_int, [H]),
            "lb_status_string": (C.c_char_p, [C.c_int]),
            "lb_totals_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
            "lb_pool_footprint": (C.c_int, [P, C.POINTER(C.c_size_t)]),
            "lb_pool_create": (C.c_int, [P, C.c_size_t, C.c_int32, C.c_void_p, C.POINTER(H)]),
            "lb_pool_admit": (C.c_int, [H, P, C.c_uint64, C.c_int64, C.POINTER(C.c_int32)]),
            "lb_pool_run": (C.c_int, [H, C.c_int64, C.POINTER(C.c_int32)]),
            "lb_pool_prepare": (C.c_int, [H]),
            "lb_pool_poll": (C.c_int, [H, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
            "lb_pool_fields": (C.c_int, [H, C.c_int32, dp, dp, dp, dp]),
            "lb_pool_init_fields": (C.c_int, [H, C.c_int32, dp, dp, dp, dp]),
            "lb_pool_stress": (C.c_int, [H, C.c_int32, C.POINTER(lb_stress_out)]),
            "lb_pool_release": (C.c_int, [H, C.c_int32]),
            "lb_pool_segment": (C.c_int32, [H]),
            "lb_selftest_wait": (C.c_int, [H, C.c_int32]),
            "lb_selftest_math": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
            "lb_pool_set_partition": (C.c_int, [H, C.c_int32]),
            "lb_pool_set_tile_rows": (C.c_int, [H, C.c_int32]),
            "lb_pool_tile_rows": (C.c_int32, [H]),
            "lb_pool_destroy": (C.c_int, [H]),
            "lb_plan_partition": (C.c_int, [C.POINTER(lb_params), C.c_int32, C.c_int32, C.c_int32,
                                            C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int, where: str):
    if status != LB_OK:
        raise LbError(status, where)


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------- C ABI names
def lb_status_string(status: int) -> str:
    return load().lb_status_string(status).decode()


def lb_params_default() -> lb_params:
    p = lb_params()
    load().lb_params_default(C.byref(p))
    return p


def lb_workspace_size(p: lb_params) -> int:
    n = C.c_size_t()
    _check(load().lb_workspace_size(C.byref(p), C.byref(n)), "lb_workspace_size")
    return n.value


def lb_create(p: lb_params, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().lb_create(C.byref(p), C.c_void_p(stream), C.byref(h)), "lb_create")
    return h.value


def lb_create_in(p: lb_params, stream: int, workspace_ptr: int, nbytes: int) -> int:
    h = C.c_void_p()
    _check(load().lb_create_in(C.byref(p), C.c_void_p(stream), C.c_void_p(workspace_ptr),
                               nbytes, C.byref(h)), "lb_create_in")
    return h.value


def lb_init_seeded(h: int, seed: int):
    _check(load().lb_init_seeded(C.c_void_p(h), seed), "lb_init_seeded")


def lb_init_fields(h: int, rho_A, rho_B, ux=None, uy=None):
    _check(load().lb_init_fields(C.c_void_p(h), _dp(rho_A), _dp(rho_B), _dp(ux), _dp(uy)),
           "lb_init_fields")


def lb_init_populations(h: int, f, t: int):
    _check(load().lb_init_populations(C.c_void_p(h), _dp(f), t), "lb_init_populations")


def lb_checkpoint(h: int, state):
    t, pulled = C.c_int64(), C.c_int32()
    _check(load().lb_checkpoint(C.c_void_p(h), _dp(state), C.byref(t), C.byref(pulled)),
           "lb_checkpoint")
    return t.value, pulled.value


def lb_restore(h: int, state, t: int, pulled: int):
    _check(load().lb_restore(C.c_void_p(h), _dp(state), t, pulled), "lb_restore")


def lb_step(h: int, n: int):
    _check(load().lb_step(C.c_void_p(h), n), "lb_step")


def lb_fields(h: int, rho_A=None, rho_B=None, ux=None, uy=None):
    _check(load().lb_fields(C.c_void_p(h), _dp(rho_A), _dp(rho_B), _dp(ux), _dp(uy)), "lb_fields")


def lb_populations(h: int, f):
    _check(load().lb_populations(C.c_void_p(h), _dp(f)), "lb_populations")


def lb_stress(h: int) -> dict:
    out = lb_stress_out()
    _check(load().lb_stress(C.c_void_p(h), C.byref(out)), "lb_stress")
    return {k: getattr(out, k) for k, _ in lb_stress_out._fields_}


def lb_sync(h: int):
    _check(load().lb_sync(C.c_void_p(h)), "lb_sync")


def lb_time(h: int) -> int:
    return load().lb_time(C.c_void_p(h))


def lb_destroy(h: int):
    _check(load().lb_destroy(C.c_void_p(h)), "lb_destroy")


# ------------------------------------------------------------- lattice pool
def lb_pool_footprint(p: lb_params) -> int:
    n = C.c_size_t()
    _check(load().lb_pool_footprint(C.byref(p), C.byref(n)), "lb_pool_footprint")
    return n.value


def lb_pool_create(shared: lb_params, budget: int, max_jobs: int, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().lb_pool_create(C.byref(shared), budget, max_jobs, C.c_void_p(stream),
                                 C.byref(h)), "lb_pool_create")
    return h.value


def lb_pool_admit(pool: int, p: lb_params, seed: int, steps: int) -> int:
    j = C.c_int32()
    _check(load().lb_pool_admit(C.c_void_p(pool), C.byref(p), seed, steps, C.byref(j)),
           "lb_pool_admit")
    return j.value


def lb_pool_run(pool: int, quantum: int) -> int:
    n = C.c_int32()
    _check(load().lb_pool_run(C.c_void_p(pool), quantum, C.byref(n)), "lb_pool_run")
    return n.value


def lb_pool_prepare(pool: int):
    _check(load().lb_pool_prepare(C.c_void_p(pool)), "lb_pool_prepare")


def lb_pool_poll(pool: int, job: int):
    steps, done = C.c_int64(), C.c_int32()
    _check(load().lb_pool_poll(C.c_void_p(pool), job, C.byref(steps), C.byref(done)),
           "lb_pool_poll")
    return steps.value, bool(done.value)


def lb_pool_fields(pool: int, job: int, rho_A=None, rho_B=None, ux=None, uy=None):
    _check(load().lb_pool_fields(C.c_void_p(pool), job, _dp(rho_A), _dp(rho_B), _dp(ux),
                                 _dp(uy)), "lb_pool_fields")


def lb_pool_init_fields(pool: int, job: int, rho_A, rho_B, ux=None, uy=None):
    _check(load().lb_pool_init_fields(C.c_void_p(pool), job, _dp(rho_A), _dp(rho_B), _dp(ux),
                                      _dp(uy)), "lb_pool_init_fields")


def lb_pool_stress(pool: int, job: int) -> dict:
    out = lb_stress_out()
    _check(load().lb_pool_stress(C.c_void_p(pool), job, C.byref(out)), "lb_pool_stress")
    return {k: getattr(out, k) for k, _ in lb_stress_out._fields_}


def lb_pool_release(pool: int, job: int):
    _check(load().lb_pool_release(C.c_void_p(pool), job), "lb_pool_release")


def lb_selftest_wait(limit: int = 1024, stream: int = 0) -> int:
    """Status of the bounded-wait self-test (LB_ERR_TIMEOUT when it works)."""
    return load().lb_selftest_wait(C.c_void_p(stream), limit)


def lb_selftest_math(x_ptr: int, out_ptr: int, n: int, stream: int = 0):
    """Device pointers: n FP32 arguments in, 3 n FP32 values out (see include/lb.h)."""
    _check(load().lb_selftest_math(C.c_void_p(x_ptr), C.c_void_p(out_ptr), n, C.c_void_p(stream)),
           "lb_selftest_math")


def lb_pool_segment(pool: int) -> int:
    return load().lb_pool_segment(C.c_void_p(pool))


def lb_pool_set_partition(pool: int, seg: int):
    _check(load().lb_pool_set_partition(C.c_void_p(pool), seg), "lb_pool_set_partition")


def lb_pool_set_tile_rows(pool: int, rows: int):
    _check(load().lb_pool_set_tile_rows(C.c_void_p(pool), rows), "lb_pool_set_tile_rows")


def lb_pool_tile_rows(pool: int) -> int:
    return load().lb_pool_tile_rows(C.c_void_p(pool))


def lb_pool_destroy(pool: int):
    _check(load().lb_pool_destroy(C.c_void_p(pool)), "lb_pool_destroy")


def lb_plan_partition(params, seg: int = 0, sms: int = 152, tile_rows: int = 8):
    """Host-only work plan of one step launch over the lattices `params`:
    (items int32[n, 4] = lattice, strip, first tile row, end tile row;
    cta int32[grid + 1] offsets into items; the partition applied)."""
    import numpy as np
    L = load()
    arr = (lb_params * len(params))(*params)
    ni, ng, su = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    L.lb_plan_partition(arr, len(params), seg, tile_rows, sms, None, C.byref(ni), None,
                        C.byref(ng), C.byref(su))
    if ni.value < 1 or ng.value < 1:
        raise LbError(LB_ERR_INVALID, "lb_plan_partition")
    items = np.zeros((ni.value, 4), dtype=np.int32)
    cta = np.zeros(ng.value + 1, dtype=np.int32)
    ni.value, ng.value = items.shape[0], cta.shape[0]
    _check(L.lb_plan_partition(arr, len(params), seg, tile_rows, sms,
                               items.ctypes.data_as(C.c_void_p), C.byref(ni),
                               cta.ctypes.data_as(C.c_void_p), C.byref(ng), C.byref(su)),
           "lb_plan_partition")
    return items, cta, su.value


LB_NOALLOC_MAX_SITES = 16777216


def lb_totals_noalloc(nx: int, ny: int, rho_A: int, rho_B: int, ux: int, uy: int,
                      totals: int, stream: int = 0):
    """Device pointers in and out (see include/lb.h); allocates nothing."""
    _check(load().lb_totals_noalloc(nx, ny, C.c_void_p(rho_A), C.c_void_p(rho_B),
                                    C.c_void_p(ux), C.c_void_p(uy), C.c_void_p(totals),
                                    C.c_void_p(stream)), "lb_totals_noalloc")


# ------------------------------------------------------------ convenience
def make_params(nx: int, ny: int, precision="fp32", **kw) -> lb_params:
    """lb_params from keyword arguments (the names of the struct fields);
    unspecified fields keep lb_params_default's values."""
    p = lb_params_default()
    p.nx, p.ny = nx, ny
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Lattice:
    """One resident lattice.  Device memory is a torch uint8 tensor on the
    current CUDA device; work runs on torch's current stream (or `stream`)."""

    def __init__(self, params: lb_params, stream=None, device=None):
        import torch
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
        nbytes = lb_workspace_size(params)
        with torch.cuda.device(dev):
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.workspace_bytes = nbytes
        self.h = lb_create_in(params, self._stream.cuda_stream, ptr, nbytes)

    @property
    def stream(self):
        return self._stream

    def init_seeded(self, seed: int):
        lb_init_seeded(self.h, seed)
        return self

    def init_fields(self, rho_A, rho_B, ux=None, uy=None):
        f = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
             for a in (rho_A, rho_B, ux, uy)]
        lb_init_fields(self.h, *f)
        return self

    def step(self, n: int = 1):
        lb_step(self.h, n)
        return self

    def checkpoint(self):
        """(stored state [2][9][ny][nx] FP64, step, pulled) -- see resume()."""
        f = np.empty((2, 9, self.ny, self.nx))
        t, pulled = lb_checkpoint(self.h, f)
        return f, t, pulled

    def resume(self, state, t: int, pulled: int):
        lb_restore(self.h, np.ascontiguousarray(state, dtype=np.float64), t, pulled)
        return self

    def init_populations(self, f, t: int = 0):
        lb_init_populations(self.h, np.ascontiguousarray(f, dtype=np.float64), t)
        return self

    def fields(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        lb_fields(self.h, *out)
        return out

    def populations(self):
        f = np.empty((2, 9, self.ny, self.nx))
        lb_populations(self.h, f)
        return f

    def stress(self) -> dict:
        return lb_stress(self.h)

    def sync(self):
        lb_sync(self.h)

    @property
    def t(self) -> int:
        return lb_time(self.h)

    def close(self):
        if getattr(self, "h", None):
            lb_destroy(self.h)
            self.h = None
            self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """Resident lattices stepped together (lb_pool_*).  `shared` fixes the
    precision, couplings, tau, psi form and forcing of every member."""

    def __init__(self, shared: lb_params, budget: int, max_jobs: int = 256, stream=None):
        s = 0 if stream is None else stream.cuda_stream
        self.h = lb_pool_create(shared, budget, max_jobs, s)
        self.shared = shared
        self._dims = {}

    @staticmethod
    def footprint(p: lb_params) -> int:
        return lb_pool_footprint(p)

    def admit(self, p: lb_params, seed: int, steps: int) -> int:
        j = lb_pool_admit(self.h, p, seed, steps)
        self._dims[j] = (p.ny, p.nx)
        return j

    def run(self, quantum: int) -> int:
        return lb_pool_run(self.h, quantum)

    def prepare(self):
        """Build the current member set's launch and capture its graph
        without stepping (see lb_pool_prepare)."""
        lb_pool_prepare(self.h)

    def poll(self, job: int):
        return lb_pool_poll(self.h, job)

    def fields(self, job: int):
        ny, nx = self._dims[job]
        out = [np.empty((ny, nx)) for _ in range(4)]
        lb_pool_fields(self.h, job, *out)
        return out

    def init_fields(self, job: int, rho_A, rho_B, ux=None, uy=None):
        """Restart member `job` from FP64 host fields (C-contiguous, ny x nx)."""
        lb_pool_init_fields(self.h, job, rho_A, rho_B, ux, uy)

    def stress(self, job: int) -> dict:
        return lb_pool_stress(self.h, job)

    def release(self, job: int):
        lb_pool_release(self.h, job)
        self._dims.pop(job, None)

    @property
    def segment(self) -> int:
        return lb_pool_segment(self.h)

    def set_partition(self, seg: int):
        """Fix the work partition (seg > 0 segments, -1 contiguous runs, 0 autotune)."""
        lb_pool_set_partition(self.h, seg)

    def set_tile_rows(self, rows: int):
        """Fix the step kernel's tile height (8 or 16; 0 autotune)."""
        lb_pool_set_tile_rows(self.h, rows)

    @property
    def tile_rows(self) -> int:
        return lb_pool_tile_rows(self.h)

    def close(self):
        if getattr(self, "h", None):
            lb_pool_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
