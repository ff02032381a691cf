"""The oracle's pins catch plausible mistakes.

Each case copies the oracle (and the pin tests) into a temporary directory,
plants one mistake in the copy by a text patch, and runs the pin tests
against that copy in a subprocess: at least one pin must fail. The
committed oracle holds none of the mistakes; they live only in the table
below. They are the kinds the pins exist to catch: a wrong sampling law, a
dropped or transposed term, a sign error, an index error, a wrong constant.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/sas_oracle.c"
PY = "oracle/__init__.py"
MSA = "oracle/msa.py"

# k: (mistake, -k selector, pin file, patched file, [(clean text, mistaken text), ...])
MUTATIONS = {
    1: ("uniform instead of triangular wavelength spread", "triangular or finite_beam", "test_oracle_pins.py", C,
        [("double T = (u < 0.5) ? sqrt(2.0 * u) - 1.0 : 1.0 - sqrt(2.0 * (1.0 - u));",
          "double T = 2.0 * u - 1.0;")]),
    2: ("sphere amplitude sin x - cos x (dropped factor x)", "sphere", "test_oracle_pins.py", C,
        [("return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);", "return 3.0 * (sin(x) - cos(x)) / (x * x * x);")]),
    3: ("Percus-Yevick beta with the wrong sign", "percus", "test_oracle_pins.py", C,
        [("double beta = -6.0 * phi", "double beta = 6.0 * phi")]),
    4: ("Eq. 8 as printed: sinc on Q_AB, J1 on Q_C", "cylinder", "test_oracle_pins.py", C,
        [("oracle_sinc(0.5 * qc * m->length)", "oracle_sinc(0.5 * qab * m->length)"),
         ("double F = drho * V * s * oracle_cyl_a(qab * r);", "double F = drho * V * s * oracle_cyl_a(qc * r);")]),
    5: ("orientation weights without sin(gamma)", "orientation or isotropic", "test_oracle_pins.py", PY,
        [("wgam = 0.5 * gmax * wg * np.sin(gam)", "wgam = 0.5 * gmax * wg * 1.0")]),
    6: ("Schulz nodes scaled by z instead of z + 1", "schulz or polydisperse", "test_oracle_pins.py", PY,
        [("return mean * x / (z + 1.0), w", "return mean * x / z, w")]),
    7: ("detector pixel index off by one", "ideal_beam or finite_beam", "test_oracle_pins.py", C,
        [("*pixel = iy * in->nx + ix;", "*pixel = iy * in->nx + ix + (ix + 1 < in->nx ? 1 : 0);")]),
    8: ("solid angle with 1/r instead of 1/r^2", "ideal_beam or finite_beam", "test_oracle_pins.py", C,
        [("double domega = area * k_out[2] / (rr * rr);", "double domega = area * k_out[2] / rr;")]),
    10: ("Philox multiplier typo", "philox", "test_oracle_pins.py", C,
         [("(uint64_t)0xCD9E8D57u * (uint64_t)c2", "(uint64_t)0xCD9E8D55u * (uint64_t)c2")]),
    11: ("core-shell outer term with the core volume", "core_shell", "test_oracle_pins.py", C,
         [("(m->sld_shell - m->sld_solvent) * Vo * oracle_sphere_f(qq * ro)",
           "(m->sld_shell - m->sld_solvent) * Vc * oracle_sphere_f(qq * ro)")]),
    12: ("per-event radius drawn without the positivity restriction", "restricted_gaussian",
         "test_event_oracle.py", C,
         [("else z = sqrt(2.0) * oracle_erfcinv(2.0 * uc * (1.0 - lo));",
           "else z = sqrt(2.0) * oracle_erfcinv(2.0 * uc * (1.0 - lo));\n"
           "    z = -sqrt(2.0) * oracle_erfcinv(2.0 * u);")]),
    13: ("parallelepiped with Q_B and Q_C swapped", "eq1_volume", "test_triaxial_oracle.py", C,
         [("F = drho * V * oracle_sinc(s * a0 * qa) * oracle_sinc(s * b0 * qb)\n"
           "                      * oracle_sinc(s * c0 * qc);",
           "F = drho * V * oracle_sinc(s * a0 * qa) * oracle_sinc(s * b0 * qc)\n"
           "                      * oracle_sinc(s * c0 * qb);")]),
    14: ("total cross section over a flat Ewald sphere (Q_z dropped)", "ewald_direction",
         "test_attenuation_oracle.py", C,
         [("double qz = -Q * Q / (2.0 * k);", "double qz = 0.0;")]),
    15: ("total cross section without the |Q| of dOmega = Q dQ dphi / k^2", "sphere_large_k",
         "test_attenuation_oracle.py", C,
         [("panel += wq * Q * ring", "panel += wq * 1.0 * ring")]),
    16: ("per-event axis uniform on the sphere where the angles are asked for", "event_axis_definitions",
         "test_event_oracle.py", C,
         [("ct = cos(th); st = sin(th);", "ct = 1.0 - 2.0 * u01(xa); st = sqrt(fmax(0.0, 1.0 - ct * ct));")]),
    17: ("Chebyshev interpolant with the constant term not halved", "chebyshev_table",
         "test_attenuation_oracle.py", C,
         [("a->c[i] = (i == 0 ? 1.0 : 2.0) * c / n;", "a->c[i] = 2.0 * c / n;")]),
    18: ("particle frame rotated by -psi instead of psi", "frame_definition", "test_triaxial_oracle.py", C,
         [("f[k] = cq * et[k] + sq * ep[k];", "f[k] = cq * et[k] - sq * ep[k];"),
          ("f[3 + k] = -sq * et[k] + cq * ep[k];", "f[3 + k] = sq * et[k] + cq * ep[k];")]),
    19: ("capped cylinder with the sphere centres outside the cylinder", "forward_scattering",
         "test_capped_oracle.py", C,
         [("double H0 = m->kind == 6 ? r0 * r0 / (R0 + h0) : R0 + h0;",
           "double H0 = m->kind != 6 ? r0 * r0 / (R0 + h0) : R0 + h0;")]),
    20: ("cap slices without their area factor rho^2 / R^2", "forward_scattering", "test_capped_oracle.py", C,
         [("cos(qc * (0.5 * L + H - R * uj[j])) * v\n", "cos(qc * (0.5 * L + H - R * uj[j])) * 1.0\n")]),
    21: ("cap slices with the sphere's radius instead of the slice's", "eq1_shells", "test_capped_oracle.py", C,
         [("oracle_cyl_a(qab * R * sqrt(v))", "oracle_cyl_a(qab * R)")]),
    22: ("core-shell cylinder shell term without its face thickness", "rectangles",
         "test_shell_models_oracle.py", C,
         [("oracle_sinc(qc * (0.5 * L + tf))", "oracle_sinc(qc * (0.5 * L))")]),
    23: ("hollow cylinder with the hollow core added instead of removed", "hollow or rectangles",
         "test_shell_models_oracle.py", C,
         [("-(m->sld - m->sld_solvent)", "(m->sld - m->sld_solvent)")]),
    24: ("core-shell ellipsoid shell without its polar thickness", "ellipsoid", "test_shell_models_oracle.py", C,
         [("double rpo = rp + m->thickness_face;", "double rpo = rp;")]),
    25: ("bicelle rim over the core's length only", "bicelle", "test_shell_models_oracle.py", C,
         [("Lo * s2 * ao", "Lo * s1 * ao")]),
    26: ("elliptical cylinder with one semi-axis for both", "new_bodies_against", "test_triaxial_oracle.py", C,
         [("xb = s * b0 * qb;", "xb = s * a0 * qb;")]),
    27: ("hollow prism normalised by its outer volume", "new_bodies_against", "test_triaxial_oracle.py", C,
         [("double v0 = vo - vi;", "double v0 = vo;")]),
    28: ("Gaussian coil without the -1 of Debye's function", "coil", "test_shape_independent_oracle.py", C,
         [("f = u < 1e-3 ? 1.0 - u / 3.0 + u * u / 12.0 : 2.0 * (expm1(-u) + u) / (u * u);",
           "f = u < 1e-3 ? 1.0 : 2.0 * (exp(-u) + u) / (u * u);")]),
    29: ("star polymer with f instead of f - 1 arm pairs", "star", "test_shape_independent_oracle.py", C,
         [("f = (deb + (fa - 1.0) * g * g) / fa;", "f = (deb + fa * g * g) / fa;")]),
    30: ("polydisperse coil with the weight-average instead of the z-average radius", "poly_coil",
         "test_shape_independent_oracle.py", C,
         [("x = q2 * m->f_p0 * m->f_p0 / (1.0 + 2.0 * U);", "x = q2 * m->f_p0 * m->f_p0 / (1.0 + U);")]),
    31: ("Guinier-Porod join without the Guinier factor", "guinier_porod", "test_shape_independent_oracle.py", C,
         [("else f = pow(q1, mp - sd) * exp(-(mp - sd) / 2.0) * pow(q, -mp);",
           "else f = pow(q1, mp - sd) * pow(q, -mp);")]),
    32: ("screened Coulomb potential with the wrong sign", "low_density", "test_msa_oracle.py", MSA,
         [("tail[1:] = -gamma_c * np.exp(-k * (x[1:] - 1.0)) / x[1:]",
           "tail[1:] = gamma_c * np.exp(-k * (x[1:] - 1.0)) / x[1:]")]),
    33: ("Bjerrum length without the relative permittivity", "textbook", "test_msa_oracle.py", MSA,
         [("/ (4.0 * math.pi * EPS0 * dielectric * K_B * temperature)", "/ (4.0 * math.pi * EPS0 * K_B * temperature)")]),
    34: ("MSA closure with h = 0 in the core instead of -1", "percus", "test_msa_oracle.py", MSA,
         [("    inner = -1.0\n", "    inner = 0.0\n")]),
    35: ("fractal factor with D instead of D - 1 in the sine", "mass_fractal", "test_shape_independent_oracle.py",
         C, [("sin(e * atan(y)) / (e * y * pow(1.0 + y * y, 0.5 * e))",
              "sin(D * atan(y)) / (D * y * pow(1.0 + y * y, 0.5 * e))")]),
    36: ("Teixeira's aggregate with Gamma(D) instead of Gamma(D + 1)", "fractal_aggregate",
         "test_shape_independent_oracle.py", C,
         [("1.0 + tgamma(D + 1.0) * pow(m->f_p2 / m->f_p0, D) * M", "1.0 + tgamma(D) * pow(m->f_p2 / m->f_p0, D) * M")]),
    38: ("excluded-volume chain with U = (Q Rg)^2 (the Rg factor dropped)", "excluded_volume",
         "test_shape_independent_oracle.py", C,
         [("double U = q2 * m->f_p0 * m->f_p0 * (2.0 * nu + 1.0) * (2.0 * nu + 2.0) / 6.0;",
           "double U = q2 * m->f_p0 * m->f_p0;")]),
    39: ("linear pearls with N instead of N - k pairs at distance k d", "linear_pearls",
         "test_shape_independent_oracle.py", C,
         [("pairs += 2.0 * (double)(N - k) * (y < 1e-8 ? 1.0 : sin(y) / y);",
           "pairs += 2.0 * (double)N * (y < 1e-8 ? 1.0 : sin(y) / y);")]),
    40: ("fuzzy sphere blurred by exp(-(Q sigma)^2) in the amplitude instead of its square root",
         "fuzzy_sphere", "test_oracle_pins.py", C,
         [("blur = exp(-0.5 * qq * qq * m->fuzz * m->fuzz);", "blur = exp(-qq * qq * m->fuzz * m->fuzz);")]),
    37: ("spinodal peak without its normalisation 1 + g/2", "spinodal", "test_shape_independent_oracle.py", C,
         [("f = (1.0 + g / 2.0) * x * x / (g / 2.0 + pow(x, 2.0 + g));", "f = x * x / (g / 2.0 + pow(x, 2.0 + g));")]),
}


def _copy_tree(dst):
    """The oracle sources, the pin tests and the workloads, without builds."""
    os.makedirs(os.path.join(dst, "oracle"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f.endswith(".py") and (f.endswith("_oracle.py") or f in ("conftest.py", "test_oracle_pins.py")):
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    for f in ("sas_workloads.py", "pytest.ini"):
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))


def _cached_build(dst, save=False):
    """Compiled copies of the oracle are kept under oracle/_build/mutants,
    keyed by the hash of the C source, so a rerun does not recompile them
    (build output only; the patched sources are rebuilt from the table)."""
    import hashlib
    src = os.path.join(dst, "oracle", "sas_oracle.c")
    key = hashlib.sha1(open(src, "rb").read()).hexdigest()[:16]
    cache = os.path.join(ROOT, "oracle", "_build", "mutants", key + ".so")
    lib = os.path.join(dst, "oracle", "_build", "libsas_oracle.so")
    if save:
        if os.path.exists(lib) and not os.path.exists(cache):
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            tmp = cache + f".tmp{os.getpid()}"
            shutil.copy(lib, tmp)
            os.replace(tmp, cache)
    elif os.path.exists(cache):
        os.makedirs(os.path.dirname(lib), exist_ok=True)
        shutil.copy(cache, lib)
        os.utime(lib)          # newer than the copied source: the loader keeps it


def test_patches_apply_to_the_clean_oracle():
    """Every clean text occurs exactly once, so each patch plants exactly
    the mistake it names (and the committed oracle is the clean form)."""
    for k, (desc, _, _, rel, hunks) in MUTATIONS.items():
        src = open(os.path.join(ROOT, rel)).read()
        for old, new in hunks:
            assert src.count(old) == 1, (k, desc, old)


@pytest.mark.parametrize("k", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(k, tmp_path):
    desc, sel, pins, rel, hunks = MUTATIONS[k]
    dst = str(tmp_path / "tree")
    _copy_tree(dst)
    path = os.path.join(dst, rel)
    src = open(path).read()
    for old, new in hunks:
        assert src.count(old) == 1, (k, old)
        src = src.replace(old, new)
    open(path, "w").write(src)
    _cached_build(dst)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(dst, "tests", pins), "-k", sel],
                       cwd=dst, capture_output=True, text=True, timeout=900)
    _cached_build(dst, save=True)
    assert r.returncode == 1, f"mutation {k} ({desc}) was not caught:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
