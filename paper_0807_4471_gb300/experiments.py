"""Observables and experiments of the paper, run on the GPU library.

* structure_factor: radially binned S(k) of phi = rho_A - rho_B (the measure
  used to compare long chaotic runs statistically).
* interface_indicator: I_AB = sum_r grad rho_A . grad rho_B (text before
  Fig. 3), with central differences on the periodic lattice.
* kolmogorov_run: the shear experiment of the paper (forcing that sustains
  U_x = U0 sin(k y) in a Newtonian fluid), returning the response
  R(t) = U(t)/U0 and I_AB(t) (Fig. 3).
* ageing_overlap: C(t_w, tau) of Eq. (6) over an ensemble of realisations,
  stepped together in one lattice pool (Fig. 4).
* laplace_test: surface tension from the pressure jump across the
  interface of circular drops, p_in - p_out = sigma / R (Fig. 2, left).
* couette_study: time-averaged wall stress and effective viscosity of plane
  Couette runs over shear rates and storage precisions.
* sweep_structure_factor: the rho0 sweep at 512^2 with S(k) and the domain
  length every 10^4 steps, for comparing storage precisions statistically.

The host code here only samples fields (lb_fields) and reduces them with
numpy; every time step runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


# ---------------------------------------------------------------- measures
def structure_factor(phi: np.ndarray):
    """S(k) = |FFT(phi - <phi>)|^2 / N, averaged over rings of width 2 pi / L
    (L = min(nx, ny)).  Returns (k centres, S per ring, modes per ring)."""
    ny, nx = phi.shape
    f = np.fft.fft2(phi - phi.mean())
    s = (np.abs(f) ** 2) / phi.size
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kk = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    dk = 2 * np.pi / min(nx, ny)
    idx = np.floor(kk / dk + 0.5).astype(int)
    nb = idx.max() + 1
    tot = np.bincount(idx.ravel(), weights=s.ravel(), minlength=nb)
    cnt = np.bincount(idx.ravel(), minlength=nb)
    with np.errstate(invalid="ignore"):
        avg = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    return np.arange(nb) * dk, avg, cnt


def domain_length(phi: np.ndarray) -> float:
    """Characteristic domain size 2 pi sum S / sum k S (k > 0)."""
    k, s, c = structure_factor(phi)
    w = s * c
    return float(2 * np.pi * w[1:].sum() / (k[1:] * w[1:]).sum())


def interface_indicator(rho_a: np.ndarray, rho_b: np.ndarray) -> float:
    """I_AB = sum grad rho_A . grad rho_B, central differences, periodic."""
    def grad(f):
        return ((np.roll(f, -1, 1) - np.roll(f, 1, 1)) / 2, (np.roll(f, -1, 0) - np.roll(f, 1, 0)) / 2)
    ax, ay = grad(rho_a)
    bx, by = grad(rho_b)
    return float((ax * bx + ay * by).sum())


def sine_projection(ux: np.ndarray, kmode: int = 1) -> float:
    """Amplitude U of u_x = U sin(2 pi kmode y / ny): 2 <u_x sin(k y)>."""
    ny = ux.shape[0]
    s = np.sin(2 * np.pi * kmode * np.arange(ny) / ny)[:, None]
    return float(2 * (ux * s).mean())


def bulk_pressure(rho_a, rho_b, Ga, Gr, GX, rho0, psi_pref):
    """Bulk part of Eq. (3): c_s^2 (rho_A + rho_B) + (c_s^2/2) sum_s
    (G^a_s + G^r_s) Psi_s^2 + c_s^2 (G_X/rho0) rho_A rho_B."""
    pa = psi_pref * (1 - np.exp(-rho_a / rho0))
    pb = psi_pref * (1 - np.exp(-rho_b / rho0))
    return (CS2 * (rho_a + rho_b) + 0.5 * CS2 * ((Ga[0] + Gr[0]) * pa ** 2 + (Ga[1] + Gr[1]) * pb ** 2)
            + CS2 * (GX / rho0) * rho_a * rho_b)


def overlap(phi_w: np.ndarray, phi_t: np.ndarray) -> float:
    """One realisation's numerator and denominator of Eq. (6)."""
    return float((phi_w * phi_t).sum()), float((phi_w * phi_w).sum())


# -------------------------------------------------------------- experiments
def kolmogorov_run(lb, n: int = 128, U0: float = 0.1, steps: int = 2000, every: int = 100,
                   seed: int = 0, precision: str = "fp32", **kw):
    """Shear by the body force a_x(y) = nu0 k^2 U0 sin(k y), k = 2 pi / n,
    which sustains U_x = U0 sin(k y) in a fluid of viscosity nu0 =
    c_s^2 (tau - 1/2).  Returns [(t, R, I_AB)], R = U(t)/U0."""
    tau = kw.pop("tau_A", 1.0)
    nu0 = CS2 * (tau - 0.5)
    k = 2 * np.pi / n
    p = lb.make_params(n, n, precision, tau_A=tau, tau_B=kw.pop("tau_B", tau),
                       kolmo_amp=nu0 * k * k * U0, kolmo_k=1.0, **kw)
    out = []
    with lb.Lattice(p) as g:
        g.init_seeded(seed)
        for t in range(0, steps + 1, every):
            if t:
                g.step(every)
            ra, rb, ux, _ = g.fields()
            out.append((t, sine_projection(ux) / U0, interface_indicator(ra, rb)))
    return out


def ageing_overlap(lb, n: int, seeds, t_w, taus, precision: str = "fp16", U0: float = 0.0,
                   **kw):
    """C(t_w, tau) of Eq. (6): ensemble averages over `seeds` of
    sum phi(t_w) phi(t_w + tau) over the average of sum phi(t_w)^2, with
    the realisations stepped together in one pool.  `t_w` is one waiting
    time or a sequence of them (one pool run serves all); U0 > 0 adds the
    Kolmogorov forcing.  Returns (taus, C), C of shape (len(taus),) for a
    single t_w, else (len(t_w), len(taus))."""
    nu0 = CS2 * (kw.get("tau_A", 1.0) - 0.5)
    k = 2 * np.pi / n
    extra = dict(kolmo_amp=nu0 * k * k * U0, kolmo_k=1.0) if U0 else {}
    p = lb.make_params(n, n, precision, **kw, **extra)
    single = np.ndim(t_w) == 0
    t_ws = [int(t_w)] if single else sorted(int(v) for v in t_w)
    taus = sorted(int(v) for v in taus)
    total = t_ws[-1] + taus[-1]
    budget = lb.Pool.footprint(p) * len(seeds) + (64 << 20)
    num = np.zeros((len(t_ws), len(taus)))
    den = np.zeros(len(t_ws))
    # every time at which the fields are read, with what to do there
    events = {}
    for a, w in enumerate(t_ws):
        events.setdefault(w, []).append(("w", a, 0))
        for b, tau in enumerate(taus):
            events.setdefault(w + tau, []).append(("t", a, b))
    with lb.Pool(p, budget, max_jobs=len(seeds)) as pool:
        jobs = [pool.admit(p, int(s), total) for s in seeds]
        phi_w = [[None] * len(jobs) for _ in t_ws]
        t = 0
        for when in sorted(events):
            if when > t:
                pool.run(when - t)
                t = when
            phis = []
            for j in jobs:
                ra, rb, _, _ = pool.fields(j)
                phis.append(ra - rb)
            # waiting-time snapshots first: tau = 0 reads the same fields
            for kind, a, b in sorted(events[when], key=lambda e: e[0] != "w"):
                if kind == "w":
                    phi_w[a] = phis
                    den[a] = sum(float((q * q).sum()) for q in phis)
                else:
                    num[a, b] = sum(float((q * r).sum()) for q, r in zip(phi_w[a], phis))
    C = num / den[:, None]
    return taus, (C[0] if single else C)


def drop_fields(n: int, radius: float, rho_in, rho_out):
    """A circular drop of species A (densities rho_in = (A, B) inside,
    rho_out outside) centred on an n x n lattice, with a tanh profile."""
    y, x = np.mgrid[0:n, 0:n]
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    s = 0.5 * (1 - np.tanh((r - radius) / 2.0))
    ra = rho_out[0] + (rho_in[0] - rho_out[0]) * s
    rb = rho_out[1] + (rho_in[1] - rho_out[1]) * s
    return ra, rb


def laplace_test(lb, rho0: float, radii=(12, 18, 26), n: int = 128, steps: int = 30000,
                 avg_from: int = 20000, every: int = 1000, precision: str = "fp32",
                 psi_form: int = 1, rho_dense: float = 1.12, rho_light: float = 0.07, **kw):
    """Laplace test on drops of A in B: p_in - p_out = sigma / R in 2-D, with
    the bulk pressure of Eq. (3) averaged over the drop interior
    (r < R - 4) and the exterior (r > R + 6), and over the samples taken
    every `every` steps from `avg_from` on.  The drop densities (rho_dense,
    rho_light) are held fixed while rho0 varies: with Psi = sqrt(rho0)
    (1 - exp(-rho/rho0)), drops whose densities scale with rho0 are exact
    rescalings of one another, so sigma would only scale with rho0.
    Returns dict(sigma, rows=[dict(R, dp, interior_cv)], uniform): sigma
    from the least-squares fit dp = sigma / R, interior_cv the relative
    spread of rho_A inside the drop (a drop whose dense phase breaks into
    micro-domains has no single bulk pressure; uniform is False then)."""
    p = lb.make_params(n, n, precision, rho0=rho0, psi_form=psi_form, **kw)
    Ga, Gr = (p.G_A1, p.G_B1), (p.G_A2, p.G_B2)
    pref = rho0 if psi_form == 1 else math.sqrt(rho0)
    y, x = np.mgrid[0:n, 0:n]
    rr = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    rows = []
    for R in radii:
        ra, rb = drop_fields(n, R, (rho_dense, rho_light), (rho_light, rho_dense))
        acc = []
        with lb.Lattice(p) as g:
            g.init_fields(ra, rb)
            g.step(avg_from)
            t = avg_from
            while True:
                fa, fb, _, _ = g.fields()
                Rm = math.sqrt(float((fa - fb > 0).sum()) / math.pi)
                inner, outer = rr < Rm - 4, rr > Rm + 6
                if inner.sum() < 4 or outer.sum() < 4:
                    acc.append((Rm, float("nan"), float("inf")))
                else:
                    pr = bulk_pressure(fa, fb, Ga, Gr, p.G_X, rho0, pref)
                    cv = float(fa[inner].std() / fa[inner].mean())
                    acc.append((Rm, float(pr[inner].mean() - pr[outer].mean()), cv))
                if t + every > steps:
                    break
                g.step(every)
                t += every
        a = np.array(acc)
        rows.append(dict(R=float(a[:, 0].mean()), dp=float(a[:, 1].mean()),
                         interior_cv=float(a[:, 2].max())))
    # drops that dissolved or lost a uniform interior carry no Laplace jump
    ok = [r for r in rows if r["R"] > 0 and np.isfinite(r["dp"])]
    xs = np.array([1.0 / r["R"] for r in ok])
    ys = np.array([r["dp"] for r in ok])
    sigma = float((xs * ys).sum() / (xs * xs).sum()) if ok else float("nan")
    return dict(sigma=sigma, rows=rows,
                uniform=len(ok) == len(rows) and all(r["interior_cv"] < 0.05 for r in rows))


def couette_study(lb, rates, precisions=("fp32", "fp16", "bf16"), n: int = 512,
                  steps: int = 200_000, avg_from: int = 100_000, rho0: float = 0.70,
                  seed: int = 2, **kw):
    """Time-averaged wall stress and effective viscosity of plane Couette
    runs (walls at +-U, shear rate 2U/n) for each storage precision; the
    lattices of one precision run together in one pool.  Returns
    {precision: [dict(rate, sigma, nu_eff, R)]}."""
    out = {}
    for prec in precisions:
        ps = [lb.make_params(n, n, prec, boundary=1, u_wall=r * n / 2.0, init_shear=1,
                             rho0=rho0, stress_t0=avg_from, **kw) for r in rates]
        budget = sum(lb.Pool.footprint(p) for p in ps) + (64 << 20)
        with lb.Pool(ps[0], budget, max_jobs=len(ps)) as pool:
            jobs = [pool.admit(p, seed, steps) for p in ps]
            while pool.run(10_000):
                pass
            rows = []
            for r, j in zip(rates, jobs):
                st = pool.stress(j)
                rows.append(dict(rate=r, sigma=st["sigma_mean"], nu_eff=st["nu_eff"],
                                 R=st["response_R"], samples=st["samples"]))
        out[prec] = rows
    return out


def couette_ensemble(lb, rate: float, seeds, precision: str = "fp32", n: int = 256,
                     steps: int = 100_000, avg_from: int = 20_000, rho0: float = 0.70, **kw):
    """Time-averaged wall stress of plane Couette runs at one shear rate over
    an ensemble of seeds (one pool).  Returns the per-seed sigma_mean list,
    in seed order, for paired comparisons between storage precisions."""
    p = lb.make_params(n, n, precision, boundary=1, u_wall=rate * n / 2.0, init_shear=1,
                       rho0=rho0, stress_t0=avg_from, **kw)
    budget = lb.Pool.footprint(p) * len(seeds) + (64 << 20)
    with lb.Pool(p, budget, max_jobs=len(seeds)) as pool:
        jobs = [pool.admit(p, int(s), steps) for s in seeds]
        while pool.run(10_000):
            pass
        return [float(pool.stress(j)["sigma_mean"]) for j in jobs]


def sweep_structure_factor(lb, rho0s=(0.55, 0.65, 0.70, 0.75, 0.83), precision: str = "fp32",
                           n: int = 512, steps: int = 100_000, every: int = 10_000, seed: int = 1,
                           psi_form: int = 1, **kw):
    """The rho0 sweep at the paper's resolution: one periodic n x n lattice
    per rho0 (seeded, all stepped together in one pool), the radially binned
    structure factor S(k) of phi = rho_A - rho_B and its domain length every
    `every` steps.  Returns {"k": ring centres, "t": sample times,
    "rho0": {rho0: {"S": [S(k) per sample], "L": [domain length per sample]}}}."""
    ps = [lb.make_params(n, n, precision, rho0=r0, psi_form=psi_form, **kw) for r0 in rho0s]
    budget = sum(lb.Pool.footprint(p) for p in ps) + (64 << 20)
    out = {"t": [], "rho0": {float(r0): {"S": [], "L": []} for r0 in rho0s}}
    with lb.Pool(ps[0], budget, max_jobs=len(ps)) as pool:
        jobs = [pool.admit(p, seed, steps) for p in ps]
        t = 0
        while True:
            if t > 0:
                out["t"].append(t)
                for r0, j in zip(rho0s, jobs):
                    ra, rb, _, _ = pool.fields(j)
                    k, S, _ = structure_factor(ra - rb)
                    rec = out["rho0"][float(r0)]
                    rec["S"].append(S.tolist())
                    rec["L"].append(domain_length(ra - rb))
                    out["k"] = k.tolist()
            if t >= steps:
                break
            step = min(every, steps - t)
            pool.run(step)
            t += step
    return out


def ensemble_statistics(lb, precision: str, seeds, n: int = 128, steps: int = 2000, **kw):
    """Per-seed domain length and phi variance after `steps` steps of seeded
    periodic lattices stepped together in one pool."""
    p = lb.make_params(n, n, precision, **kw)
    budget = lb.Pool.footprint(p) * len(seeds) + (64 << 20)
    L, var = [], []
    with lb.Pool(p, budget, max_jobs=len(seeds)) as pool:
        jobs = [pool.admit(p, int(s), steps) for s in seeds]
        pool.run(steps)
        for j in jobs:
            ra, rb, _, _ = pool.fields(j)
            phi = ra - rb
            L.append(domain_length(phi))
            k, s, c = structure_factor(phi)
            var.append(float((s * c).sum()))
    return dict(L=L, var=var)


# ------------------------------------------------------------ command line
def main(argv=None):
    """Run one study on the GPU and print its result as JSON:

        python -m paper_0807_4471_gb300.experiments kolmogorov --psi-form 1
        python -m paper_0807_4471_gb300.experiments ageing
        python -m paper_0807_4471_gb300.experiments laplace
        python -m paper_0807_4471_gb300.experiments couette --precisions fp64,fp32,fp16,bf16
        python -m paper_0807_4471_gb300.experiments couette-ensemble --rate 1e-4
        python -m paper_0807_4471_gb300.experiments statistics --steps 2000
        python -m paper_0807_4471_gb300.experiments sweep --precisions fp64,fp32,fp16,bf16
    """
    import argparse
    import json

    import paper_0807_4471_gb300 as lb

    ap = argparse.ArgumentParser(prog="python -m paper_0807_4471_gb300.experiments")
    ap.add_argument("study", choices=["kolmogorov", "ageing", "laplace", "couette",
                                      "couette-ensemble", "statistics", "sweep"])
    ap.add_argument("--psi-form", type=int, default=1)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--precisions", default="fp64,fp32,fp16,bf16")
    ap.add_argument("--rounding", type=int, default=1)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--every", type=int, default=20_000)
    ap.add_argument("--U0", type=float, default=None)
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--rate", type=float, default=1e-4)
    ap.add_argument("--rho0s", default="0.55,0.60,0.65,0.70,0.75,0.80")
    ap.add_argument("--passive", action="store_true", help="all couplings zero")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    lb.load()
    kw = dict(psi_form=a.psi_form, rounding=a.rounding)
    if a.passive:
        kw.update(G_A1=0.0, G_A2=0.0, G_B1=0.0, G_B2=0.0, G_X=0.0, init_amp=0.0)
    precs = a.precisions.split(",")
    if a.study == "kolmogorov":
        res = kolmogorov_run(lb, n=a.n or 128, U0=0.1 if a.U0 is None else a.U0,
                             steps=a.steps or 2_000_000, every=a.every, precision=a.precision, **kw)
    elif a.study == "ageing":
        taus = [0, 1000, 3000, 10_000, 30_000, 100_000, 200_000]
        out = {}
        for U0 in ((0.02, 0.03) if a.U0 is None else (a.U0,)):
            t, C = ageing_overlap(lb, a.n or 128, range(a.seeds), [50_000, 200_000, 300_000], taus,
                                  precision=a.precision, U0=U0, **kw)
            out[str(U0)] = dict(t_w=[50_000, 200_000, 300_000], taus=t, C=C.tolist())
        res = out
    elif a.study == "laplace":
        res = {r0: laplace_test(lb, float(r0), precision=a.precision, **kw)
               for r0 in a.rho0s.split(",")}
    elif a.study == "couette":
        rates = [float(v) for v in np.logspace(-6, -4, 8)]
        res = couette_study(lb, rates, precisions=tuple(precs), n=a.n or 512,
                            steps=a.steps or 200_000, avg_from=(a.steps or 200_000) // 2, **kw)
    elif a.study == "sweep":
        res = {p: sweep_structure_factor(lb, precision=p, n=a.n or 512, steps=a.steps or 100_000,
                                         every=a.every if a.every != 20_000 else 10_000, **kw)
               for p in precs}
    elif a.study == "couette-ensemble":
        res = {p: couette_ensemble(lb, a.rate, range(a.seeds), precision=p, n=a.n or 256,
                                   steps=a.steps or 100_000, **kw) for p in precs}
    else:
        res = {p: ensemble_statistics(lb, p, range(32 if a.seeds == 16 else a.seeds),
                                      n=a.n or 128, steps=a.steps or 2000, **kw) for p in precs}
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    print(text)


if __name__ == "__main__":
    main()
