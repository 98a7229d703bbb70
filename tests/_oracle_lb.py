"""The slice of the library's Python API that the experiment drivers use
(make_params, Lattice, Pool), backed by the FP64 CPU oracle, so that the
drivers run unchanged on the oracle (test infrastructure)."""


class OracleLb:
    """The slice of the library's Python API that the experiment drivers
    use (make_params, Lattice), run on the oracle so the drivers' host
    logic is exercised on the CPU."""

    def __init__(self, O, caption):
        self.O, self.caption = O, caption

    def make_params(self, nx, ny, precision="fp64", *, rho0=None, psi_form=0, **kw):
        from types import SimpleNamespace
        c = dict(self.caption)
        if rho0 is not None:
            c["rho0"] = rho0
        P = self.O.make_params(nx, ny, psi_form=psi_form, **c, **kw)
        return SimpleNamespace(P=P, G_A1=c["Ga"][0], G_B1=c["Ga"][1], G_A2=c["Gr"][0],
                               G_B2=c["Gr"][1], G_X=c["GX"])

    def Lattice(self, p):
        O = self.O

        class _L:
            def __enter__(s):
                s.t = 0
                return s

            def __exit__(s, *a):
                return False

            def init_fields(s, ra, rb):
                s.f = O.init_fields(p.P, ra, rb)

            def step(s, n):
                assert O.run(p.P, s.f, n, t0=s.t) == 0
                s.t += n

            def fields(s):
                return O.fields(p.P, s.f)

        return _L()

    @property
    def Pool(self):
        O = self.O

        class _Pool:
            @staticmethod
            def footprint(p):
                return 1

            def __init__(s, p, budget, max_jobs):
                s.jobs = []

            def __enter__(s):
                return s

            def __exit__(s, *a):
                return False

            def admit(s, p, seed, steps):
                s.jobs.append([p.P, O.init_seeded(p.P, seed), 0])
                return len(s.jobs) - 1

            def run(s, n):
                for j in s.jobs:
                    assert O.run(j[0], j[1], n, t0=j[2]) == 0
                    j[2] += n
                return len(s.jobs)

            def fields(s, j):
                return O.fields(s.jobs[j][0], s.jobs[j][1])

        return _Pool
