"""Ablations on a synthetic tomographic series (the paper's Figs. S3-S5,
qualitatively): PWF on every projection, FBP, scores against the phantom."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ablation():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import ablation as A
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return A


@pytest.fixture(scope="module")
def series(ablation):
    return ablation.make_series(n_angles=32, n=128)


def by_name(A, name):
    return next(s for s in A.SETTINGS if s.name == name)


def test_gamma_zero_and_alpha_zero_both_switch_the_regularizer_off(ablation, series):
    _, p_g0, _ = ablation.run_setting(series, by_name(ablation, "gamma_0"), 20)
    _, p_a0, _ = ablation.run_setting(series, by_name(ablation, "alpha_0"), 20)
    assert torch.equal(p_g0, p_a0)


def test_without_the_preconditioner_delta_is_underestimated(ablation, series):
    paper, _, _ = ablation.run_setting(series, by_name(ablation, "paper"), 150)
    noprec, _, _ = ablation.run_setting(series, by_name(ablation, "no_precond"), 150)
    assert noprec["delta_ratio"] < 0.7 * paper["delta_ratio"], (paper, noprec)
    assert paper["delta_rel_err"] < noprec["delta_rel_err"], (paper, noprec)


def test_ablation_table_runs_every_setting(ablation, series):
    rows = ablation.run_ablation(series, iters=30)
    assert [r["setting"] for r in rows] == [s.name for s in ablation.SETTINGS]
    for r in rows:
        assert all(v == v for v in (r["delta_rel_err"], r["beta_rel_err"], r["delta_ratio"], r["rmse_image_pct"]))
    print(ablation.summary_table(rows))
