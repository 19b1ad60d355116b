"""The pins catch plausible mistakes: each mutant below is a copy of the
oracle with one deliberate error (dropped term, flipped sign, wrong index,
transposed operand, wrong normalisation).  Mutants of the C evaluator are
compiled on the CPU; mutants of the Python sampler are executed as a copy of
the oracle package whose functions stand in for the originals.  Every mutant
must fail at least one pin of test_oracle_pins.py or test_oracle_mcmc.py.
Nothing here touches a GPU."""
import inspect
import types

import pytest

import oracle
from tests import test_oracle_mcmc as mcmc_pins
from tests import test_oracle_pins as pins

# (description, exact text in lens_oracle.c, replacement)
MUTANTS = [
    ("Hessian xy sign", "out[4] = -f * x * y;", "out[4] = f * x * y;"),
    ("dropped s*psi in psi_xx", "out[2] = f * (q * q * s * s + y * y + s * psi);", "out[2] = f * (q * q * s * s + y * y);"),
    ("atanh denominator", "atanh_over_u(u, y / (psi + q * q * s))", "atanh_over_u(u, y / (psi + s))"),
    ("axis ratio inverted", "*q = (1.0 - e) / (1.0 + e);", "*q = (1.0 + e) / (1.0 - e);"),
    ("strength not scaled", "*b = h->b0 * (1.0 + e);", "*b = h->b0;"),
    ("rotation sign", "y = -s * dX + c * dY; /* halo frame */", "y = s * dX + c * dY; /* halo frame */"),
    ("back-rotation sign", "out[0] = c * p[0] - s * p[1];", "out[0] = c * p[0] + s * p[1];"),
    ("Hessian rotation transposed", "out[4] = c * s * (p[2] - p[3]) + (c * c - s * s) * p[4];",
     "out[4] = c * s * (p[3] - p[2]) + (c * c - s * s) * p[4];"),
    ("core + cut", "p[k] = core[k] - cut[k];", "p[k] = core[k] + cut[k];"),
    ("SIS Hessian index", "out[2] = b * dY * dY / r3;", "out[2] = b * dX * dX / r3;"),
    ("point-mass shear factor", "out[4] = -2.0 * te2 * dX * dY / r4;", "out[4] = -te2 * dX * dY / r4;"),
    ("kappa without 1/2", "double kappa = 0.5 * (v[2] + v[3]);", "double kappa = (v[2] + v[3]);"),
    ("det sign (the Eq. 9 typo)", "double det = (1.0 - kappa) * (1.0 - kappa) - g1 * g1 - g2 * g2;",
     "double det = (1.0 - kappa) * (1.0 - kappa) + g1 * g1 + g2 * g2;"),
    ("mapped residual transposed", "double rx = (a22 * dbx - a12 * dby) / det;", "double rx = (a11 * dbx - a12 * dby) / det;"),
    ("barycentre count", "bary[2 * i] = m > 0 ? sx / m : 0.0;", "bary[2 * i] = m > 0 ? sx / (m + 1) : 0.0;"),
    ("Newton step sign", "    x += dx;\n    y += dy;", "    x -= dx;\n    y -= dy;"),
    ("distance ratio dropped", "for (int k = 0; k < 5; ++k) out[k] = dls_ds * acc[k];",
     "for (int k = 0; k < 5; ++k) out[k] = acc[k];"),
    ("magnification weight is det, not |mu|", "chi2 += (dbx * dbx + dby * dby) * fabs(1.0 / det) / s2;",
     "chi2 += (dbx * dbx + dby * dby) * fabs(det) / s2;"),
    ("magnification weight without its absolute value", "chi2 += (dbx * dbx + dby * dby) * fabs(1.0 / det) / s2;",
     "chi2 += (dbx * dbx + dby * dby) * (1.0 / det) / s2;"),
    ("chi2 sigma not squared", "ci += bd / (c->sigma[j] * c->sigma[j]);", "ci += bd / c->sigma[j];"),
    ("grid spacing", "return g->nx > 1 ? g->xmin + i * ((g->xmax - g->xmin) / (g->nx - 1)) : g->xmin;",
     "return g->nx > 1 ? g->xmin + i * ((g->xmax - g->xmin) / g->nx) : g->xmin;"),
    ("potential log term", "return x * ax + y * ay - b * q * s * 0.5 * log(w);", "return x * ax + y * ay - b * q * 0.5 * log(w);"),
    ("point-mass potential ln r^2 for ln r", "return r2 > 0.0 ? h->b0 * h->b0 * 0.5 * log(r2) : 0.0;",
     "return r2 > 0.0 ? h->b0 * h->b0 * log(r2) : 0.0;"),
    ("SIS potential with the strength halved", "if (h->type == OR_SIS) return h->b0 * sqrt(r2);",
     "if (h->type == OR_SIS) return 0.5 * h->b0 * sqrt(r2);"),
    ("series used outside its range", "static double atan_over_u(double u, double t) {\n  if (u < 1e-4) {",
     "static double atan_over_u(double u, double t) {\n  if (u < 0.5) {"),
]


# (description, exact text in oracle/__init__.py, replacement)
PY_MUTANTS = [
    ("acceptance without the 1/2 of the likelihood exp(-chi2/2)",
     "(np.log(u) < -(chi2p - chi2) / (2.0 * temperature))", "(np.log(u) < -(chi2p - chi2) / temperature)"),
    ("acceptance with the chi2 difference reversed",
     "(np.log(u) < -(chi2p - chi2) / (2.0 * temperature))", "(np.log(u) < -(chi2 - chi2p) / (2.0 * temperature))"),
    ("Box-Muller radius without the factor 2", "rad = np.sqrt(-2.0 * np.log(u[:, 2 * i]))",
     "rad = np.sqrt(-np.log(u[:, 2 * i]))"),
]


def pin_functions():
    out = []
    for mod in (pins, mcmc_pins):
        fixtures = getattr(mod, "FIXTURES", {})
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_"):
                continue
            marks = getattr(fn, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            args = list(inspect.signature(fn).parameters)
            if params:
                for v in params[0].args[1]:
                    out.append((f"{name}[{v}]", lambda fn=fn, v=v: fn(v)))
            elif args:
                out.append((name, lambda fn=fn, args=args, fx=fixtures: fn(*[fx[a]() for a in args])))
            else:
                out.append((name, fn))
    return out


def first_failing_pin():
    for name, fn in pin_functions():
        try:
            fn()
        except Exception:
            return name
    return None


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(desc, old, new, workdir):
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site not found: {desc}"
    path = oracle.build_variant(src.replace(old, new), str(workdir / f"m{abs(hash(desc))}.so"))
    oracle.use_library(path)
    try:
        assert first_failing_pin() is not None, f"no pin caught mutant: {desc}"
    finally:
        oracle.use_library(None)


@pytest.mark.parametrize("desc,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_fails_a_pin(desc, old, new):
    with open(oracle.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not found: {desc}"
    mutant = types.ModuleType("oracle_mutant")
    mutant.__file__ = oracle.__file__
    exec(compile(src.replace(old, new), oracle.__file__, "exec"), mutant.__dict__)
    names = [n for n, v in vars(oracle).items() if inspect.isfunction(v) and not n.startswith("_")]
    saved = {n: getattr(oracle, n) for n in names}
    try:
        for n in names:
            setattr(oracle, n, getattr(mutant, n))
        assert first_failing_pin() is not None, f"no pin caught mutant: {desc}"
    finally:
        for n, v in saved.items():
            setattr(oracle, n, v)
