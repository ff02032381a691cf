"""The oracle's pins catch plausible mistakes.

Each case builds a copy of the oracle with one planted mistake
(SAS_ORACLE_MUTATION=k; the default build has none) and runs the pin tests
in a subprocess: at least one pin must fail. The mistakes are the kinds the
pins exist to catch: a wrong sampling law, a dropped or transposed term, a
sign error, an index error, a wrong constant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    1: ("uniform instead of triangular wavelength spread", "triangular or finite_beam"),
    2: ("sphere amplitude sin x - cos x (dropped factor x)", "sphere"),
    3: ("Percus-Yevick beta with the wrong sign", "percus"),
    4: ("Eq. 8 as printed: sinc on Q_AB, J1 on Q_C", "cylinder"),
    5: ("orientation weights without sin(gamma)", "orientation or isotropic"),
    6: ("Schulz nodes scaled by z instead of z + 1", "schulz or polydisperse"),
    7: ("detector pixel index off by one", "ideal_beam or finite_beam"),
    8: ("solid angle with 1/r instead of 1/r^2", "ideal_beam or finite_beam"),
    10: ("Philox multiplier typo", "philox"),
    11: ("core-shell outer term with the core volume", "core_shell"),
    12: ("per-event radius drawn without the positivity restriction", "restricted_gaussian",
         "test_event_oracle.py"),
    13: ("parallelepiped with Q_B and Q_C swapped", "eq1_volume", "test_triaxial_oracle.py"),
    14: ("total cross section over a flat Ewald sphere (Q_z dropped)", "ewald_direction",
         "test_attenuation_oracle.py"),
    15: ("total cross section without the |Q| of dOmega = Q dQ dphi / k^2", "sphere_large_k",
         "test_attenuation_oracle.py"),
    16: ("per-event axis uniform on the sphere where the angles are asked for", "event_axis_definitions",
         "test_event_oracle.py"),
    17: ("Chebyshev interpolant with the constant term not halved", "chebyshev_table",
         "test_attenuation_oracle.py"),
    18: ("particle frame rotated by -psi instead of psi", "frame_definition", "test_triaxial_oracle.py"),
    19: ("capped cylinder with the sphere centres outside the cylinder", "forward_scattering",
         "test_capped_oracle.py"),
    20: ("cap slices without their area factor rho^2 / R^2", "forward_scattering", "test_capped_oracle.py"),
    21: ("cap slices with the sphere's radius instead of the slice's", "eq1_shells", "test_capped_oracle.py"),
    22: ("core-shell cylinder shell term without its face thickness", "rectangles", "test_shell_models_oracle.py"),
    23: ("hollow cylinder with the hollow core added instead of removed", "hollow or rectangles",
         "test_shell_models_oracle.py"),
    24: ("core-shell ellipsoid shell without its polar thickness", "ellipsoid", "test_shell_models_oracle.py"),
    25: ("bicelle rim over the core's length only", "bicelle", "test_shell_models_oracle.py"),
    26: ("elliptical cylinder with one semi-axis for both", "new_bodies_against", "test_triaxial_oracle.py"),
    27: ("hollow prism normalised by its outer volume", "new_bodies_against", "test_triaxial_oracle.py"),
    28: ("Gaussian coil without the -1 of Debye's function", "coil", "test_shape_independent_oracle.py"),
}


@pytest.mark.parametrize("k", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(k):
    desc, sel = MUTATIONS[k][:2]
    pins = MUTATIONS[k][2] if len(MUTATIONS[k]) > 2 else "test_oracle_pins.py"
    env = dict(os.environ, SAS_ORACLE_MUTATION=str(k))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins), "-k", sel],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, f"mutation {k} ({desc}) was not caught:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
