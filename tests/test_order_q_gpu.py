"""The |Q|-ordered trace pass (launch option order_q) against the plain loop.

Ordering a CTA's histories by |Q|^2 only changes which lane evaluates which
history, and in the closed-form run of the radius nodes the order in which
the common factor 1/q^6 is applied; every history keeps its pixel and a
weight equal to within FP32 rounding. So on the same Philox streams:
counts are bit-exact, per-bin sums agree to the FP32 tally precision
(6e-6 relative on bins above 1e-6 of the maximum, the
bound on one history's rounding difference derived below), the transmitted weight
to 1e-12, and the ordered run matches the FP64 oracle as the plain run does.
Cases: the core-shell workload and a polydisperse sphere; ragged history
counts (not a multiple of the CTA), fewer histories than one CTA, several
block sizes; the option is ignored (same result as plain) where it does not
apply: per-event sampling, FP64, monodisperse.
"""
import numpy as np
import pytest

import oracle
import paper_2501_06054_gb300 as sas
import sas_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    yield


def _sphere():
    return W.Model(kind=W.SPHERE, precision=W.FP32, radius=60.0, sld=2.0e-6, sld_solvent=0.0,
                   volume_fraction=0.01, poly=0.15, n_poly=30)


def _run(inst, model, n, seed, order_q, block=1024, tally=1):
    ex = sas.Experiment(inst, model, stream=torch.cuda.current_stream())
    c = sas.sas_launch_config(block=block, tally=tally, agg=0, ctas_per_sm=0, stage_orient=0, order_q=order_q)
    sas.sas_set_launch_config(ex.h, c)
    ex.trace(n, seed)
    d = ex.read()
    ex.close()
    return d


# Per history the two paths differ only in the rounding of the closed-form
# run: there the plain loop rounds (q^-3 c_k) once per node and squares, the
# ordered one applies q^-6 to the run's sum; each of the <= 40 positive terms
# moves by at most about 6 ulps and the sum's own rounding by <= 40 ulps, so
# a history's value moves by less than 2 x 46 x 2^-24 = 5.5e-6 relative. Bins
# of many histories average these; single-history bins do not.
REL = 6e-6


def _same(a, b, rel=REL):
    assert np.array_equal(a["count"], b["count"])
    so = b["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(a["sum_w"] - so)[big] <= rel * so[big])
    s2 = b["sum_w2"]
    big2 = s2 > 1e-6 * s2.max()
    assert np.all(np.abs(a["sum_w2"] - s2)[big2] <= 2 * rel * s2[big2])
    assert abs(a["trans"] / b["trans"] - 1) < 1e-12


@pytest.mark.parametrize("which", ["core_shell", "sphere"])
@pytest.mark.parametrize("n,block", [(1_000_003, 1024), (300_001, 512), (777, 1024), (2_049, 256)])
def test_ordered_equals_plain(which, n, block):
    inst = W.instrument()
    model = W.core_shell_config()["model"] if which == "core_shell" else _sphere()
    _same(_run(inst, model, n, 5, 1, block), _run(inst, model, n, 5, 0, block))


def test_ordered_matches_the_oracle():
    cfg = W.core_shell_config()
    n = 200_003
    d = _run(cfg["instrument"], cfg["model"], n, 11, 1)
    ref = oracle.trace(cfg["instrument"], cfg["model"], n, seed=11)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
    so = ref["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    assert abs(d["sum_w"].sum() / so.sum() - 1) < 1e-4


def test_default_configuration_orders_the_headline_workload():
    # a detector size no autotuning in this process has cached a configuration for
    cfg = W.core_shell_config()
    ex = sas.Experiment(W.instrument(nx=126, ny=126), cfg["model"])
    c = sas.sas_get_launch_config(ex.h)
    assert c.order_q == 1 and c.tally == 1
    ex.close()


@pytest.mark.parametrize("variant", ["per_event", "fp64", "mono"])
def test_option_is_ignored_where_it_does_not_apply(variant):
    inst = W.instrument()
    m = _sphere()
    if variant == "per_event":
        m.sampling, m.poly_dist = W.PER_EVENT, W.GAUSSIAN
    elif variant == "fp64":
        m.precision = W.FP64
    else:
        m.poly, m.n_poly = 0.0, 1
    tally = 0 if variant == "fp64" else 1
    a = _run(inst, m, 100_003, 3, 1, 256, tally)
    b = _run(inst, m, 100_003, 3, 0, 256, tally)
    assert np.array_equal(a["count"], b["count"])
    so = b["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(a["sum_w"] - so)[big] <= REL * so[big])
