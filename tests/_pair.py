"""Helpers that set up the same model on the FP64 oracle and on the GPU
library from one set of keyword arguments (test infrastructure)."""
import numpy as np

import lbinputs

ORACLE_KEYS = ("boundary", "psi_form", "force_scheme", "u_wall", "init_amp", "init_shear",
               "g_x", "kolmo_amp", "kolmo_k", "stress_every", "stress_t0")


def model(nx, ny, *, Ga=None, Gr=None, GX=None, rho0=None, tau=(1.0, 1.0), psi_form=1, **kw):
    """Caption couplings and, by default, Psi = rho0 (1 - exp(-rho/rho0)), the
    form the plain-method configuration states."""
    c = lbinputs.CAPTION
    Ga = c["Ga"] if Ga is None else Ga
    Gr = c["Gr"] if Gr is None else Gr
    GX = c["GX"] if GX is None else GX
    rho0 = c["rho0"] if rho0 is None else rho0
    return dict(nx=nx, ny=ny, Ga=tuple(Ga), Gr=tuple(Gr), GX=GX, rho0=rho0, tau=tuple(tau),
                psi_form=psi_form, **kw)


def oracle_params(O, m):
    kw = {k: m[k] for k in ORACLE_KEYS if k in m}
    return O.make_params(m["nx"], m["ny"], Ga=m["Ga"], Gr=m["Gr"], GX=m["GX"], rho0=m["rho0"],
                         tau=m["tau"], **kw)


def gpu_params(lb, m, precision):
    kw = {k: m[k] for k in ORACLE_KEYS if k in m}
    return lb.make_params(m["nx"], m["ny"], precision, G_A1=m["Ga"][0], G_A2=m["Gr"][0],
                          G_B1=m["Ga"][1], G_B2=m["Gr"][1], G_X=m["GX"], rho0=m["rho0"],
                          tau_A=m["tau"][0], tau_B=m["tau"][1], **kw)


def gpu_pops_as_oracle(f):
    """[2][9][ny][nx] -> oracle layout (ny, nx, 2, 9)."""
    return np.ascontiguousarray(f.transpose(2, 3, 0, 1))


def rel_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def round_half(x):
    """Round FP64 offsets to the FP16 storage format: binary16 of x * 2^10,
    nearest-even (numpy's conversion), divided back by 2^10."""
    x = np.asarray(x, dtype=np.float64) * 1024.0
    return x.astype(np.float16).astype(np.float64) / 1024.0


def round_bf16(x):
    """Round FP64 values to bfloat16 (7 fraction bits), nearest-even, directly
    from the FP64 bits (values well inside the normal range)."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    b = (b + np.uint64((1 << 44) - 1) + lsb) & ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


def ulp16(x, fmt):
    """Spacing of the 16-bit storage format at |x| (FP16: binary16 of
    x * 2^10, 10 fraction bits, subnormal spacing 2^-34 in x; bfloat16: 7
    fraction bits)."""
    ax = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), 1e-300)
    e = np.floor(np.log2(ax))
    if fmt == "fp16":
        return np.power(2.0, np.maximum(e, -24.0) - 10.0)
    return np.power(2.0, e - 7.0)


def offsets(f, rho_ref):
    """Oracle-layout populations f (ny, nx, 2, 9) -> offsets f - w_i rho_ref."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return f - w * rho_ref
