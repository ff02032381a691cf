"""The Hayter-Penfold S(Q) on the GPU against the oracle.

* model evaluations (sas_eval_model) of a sphere and a core-shell sphere
  with the charged-sphere S(Q), a plain and a rescaled case, FP32 at T1
  (1e-5 relative + 1e-7 of the largest) and FP64 at 1e-6 relative (both
  sides interpolate their own tables: the library's within 2.2e-7 of the
  direct transform, the oracle's within 1e-8);
* traced detectors against the oracle's trace on the same Philox streams:
  counts bit-exact, per-bin sums 1e-4 relative where they hold >= 1e-6 of
  the largest (FP32 tallies);
* the ordered FP32 sphere pass with this S(Q) against the plain loop;
* refusals: a batch, parameters out of range.
"""
import numpy as np
import pytest

import oracle
import paper_2501_06054_gb300 as sas
import sas_workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

CASES = {
    "plain": dict(sq_radius=40.0, sq_fraction=0.2, sq_charge=15.0, sq_salt=0.05, sq_temperature=310.0,
                  sq_dielectric=70.0),
    "rescaled": dict(sq_radius=22.0, sq_fraction=0.1, sq_charge=20.0, sq_salt=0.01),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    yield


def _model(kind, case, precision):
    if kind == "sphere":
        m = W.Model(kind=W.SPHERE, precision=precision, radius=20.0, sld=2.0e-6, sld_solvent=0.0,
                    volume_fraction=0.1, poly=0.1, n_poly=20)
    else:
        m = W.Model(kind=W.CORE_SHELL, precision=precision, radius=15.0, thickness=5.0, sld=1.0e-6,
                    sld_shell=3.0e-6, sld_solvent=6.0e-6, volume_fraction=0.1, poly=0.1, n_poly=20)
    m.sq_kind = W.SQ_HAYTER_MSA
    for k, v in CASES[case].items():
        setattr(m, k, v)
    return m


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["sphere", "core_shell"])
def test_eval_parity(kind, case, precision):
    m = _model(kind, case, precision)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    q = d * rng.uniform(1e-4, 0.4, 3000)[:, None]
    e = sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
    dt = torch.float64 if precision == W.FP64 else torch.float32
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, torch.tensor(q, dtype=dt, device="cuda"), len(q), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    e.close()
    qd = torch.tensor(q, dtype=dt).double().numpy()
    ref = oracle.dsigma(oracle.Prepared(m), qd)
    rel, ab = (1e-6, 0.0) if precision == W.FP64 else (1e-5, 1e-7)
    err = np.abs(got - ref)
    assert np.all(err <= rel * np.abs(ref) + ab * ref.max()), np.max(err / (rel * np.abs(ref) + ab * ref.max()))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["sphere", "core_shell"])
def test_trace_against_the_oracle(kind, case):
    m = _model(kind, case, W.FP32)
    inst = W.instrument()
    n = 300_007
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    e.trace(n, 6)
    d = e.read()
    e.close()
    ref = oracle.trace(inst, m, n, seed=6)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
    so = ref["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    assert abs(d["trans"] / ref["trans"] - 1) < 1e-6


def test_ordered_pass_with_the_charged_sphere_s_of_q():
    m = _model("sphere", "rescaled", W.FP32)
    inst = W.instrument()
    res = []
    for oq in (1, 0):
        e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
        c = sas.sas_launch_config(block=1024, tally=1, agg=0, ctas_per_sm=0, stage_orient=0, order_q=oq)
        sas.sas_set_launch_config(e.h, c)
        e.trace(500_003, 2)
        res.append(e.read())
        e.close()
    assert np.array_equal(res[0]["count"], res[1]["count"])
    so = res[1]["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(res[0]["sum_w"] - so)[big] <= 6e-6 * so[big])


def test_refusals():
    m = _model("sphere", "plain", W.FP32)
    with pytest.raises(sas.SasError):
        sas.sas_create_batch(W.instrument(), [m], np.array([1000], dtype=np.uint64),
                             stream=torch.cuda.current_stream())
    bad = _model("sphere", "plain", W.FP32)
    bad.sq_fraction = 0.5
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), bad)
    bad = _model("sphere", "plain", W.FP32)
    bad.sq_salt = -1.0
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), bad)
