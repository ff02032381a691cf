"""The nominal FLOP table behind the roofline lines (CPU): per-history totals
of the workloads the benchmark reports, built from the per-term counts the
table's docstring derives, and the FP32 peak it divides by."""
import pytest

import sas_workloads as W
from paper_2501_06054_gb300 import flops as F


def test_workload_totals():
    cs = W.core_shell_config()["model"]
    assert F.flops_per_history(cs.kind, cs.n_poly, 1, sq=True) == 40 * F.CS_NODE + F.CS_HISTORY + F.GEOMETRY + F.PY
    assert F.flops_per_history(cs.kind, cs.n_poly, 1, sq=True) == 2690
    cyl = W.cylinder_config()["model"]
    n_orient = cyl.n_gamma * cyl.n_psi
    assert F.flops_per_history(cyl.kind, cyl.n_poly, n_orient) == n_orient * (F.ORIENT_NODE + 40 * F.CYL_TERM) + F.GEOMETRY
    assert F.flops_per_history(cyl.kind, cyl.n_poly, n_orient) == 6353750


@pytest.mark.parametrize("cfg", W.shelled_configs(), ids=lambda c: c["name"])
def test_shelled_totals(cfg):
    m = cfg["model"]
    no = m.n_gamma * m.n_psi
    if m.kind == W.CORE_SHELL_ELLIPSOID:
        per = no * (F.ORIENT_NODE + m.n_poly * F.CS_ELL_TERM)
    else:
        per = no * (F.CS_CYL_ORIENT + m.n_poly * F.CS_CYL_TERM)
    assert F.flops_per_history(m.kind, m.n_poly, no) == per + F.GEOMETRY


def test_capped_totals():
    for cfg in (W.capped_cylinder_config(), W.barbell_config()):
        m = cfg["model"]
        no = m.n_gamma * m.n_psi
        per = no * (F.ORIENT_NODE + m.n_poly * (F.CAP_NODE + m.n_cap * F.CAP_SLICE))
        assert F.flops_per_history(m.kind, m.n_poly, no, n_cap=m.n_cap) == per + F.GEOMETRY


def test_fp32_peak():
    # 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2.07 GHz
    assert F.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784, rel=1e-12)
