"""GPU regularisation selection (Algorithm 3) against the oracle's selection on the same snapshots."""
import numpy as np
import pytest

from oracle import fit as OF
from oracle import oracle as O
from paper_2511_20687_gb300 import osam
from paper_2511_20687_gb300 import workloads as W

from .test_oracle_fit_adjoint import _known_quadratic_trajectory

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20687_gb300 import build_lib
    build_lib.build()
    osam.load()
    return torch


def _compare(errs_gpu, errs_ref):
    for eg, er in zip(errs_gpu, errs_ref):
        if np.isfinite(er):
            assert np.isfinite(eg)
            assert abs(eg - er) <= 1e-6 * er + 1e-9, (eg, er)
        else:
            assert not np.isfinite(eg) or eg >= 1e300


def test_selection_on_a_generating_model_matches_oracle(gpu):
    U, A, S, v0 = _known_quadratic_trajectory()
    lams = OF.lambda_grid()
    ref_err, ref_best, _ = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.02, k=1, r_s=2)
    got = osam.opinf_select(U.T, A.T, S.T, v0, r=5, lambdas=lams, dt=0.02, substeps=1, r_s=2)
    _compare(got["errors"], ref_err)
    assert got["errors"][got["best"]] < 1e-6 and got["lambda"] <= 1e-4


def test_selection_on_fom_training_snapshots_matches_oracle(gpu):
    """Snapshots of the ROM-side subdomain of a small Neo-Hookean FOM-FOM run (one per controller
    step of 3 substeps), 11 candidates, rollouts with the online step and the interpolated boundary."""
    spec = W.bar_chain("sel", 3, [6, 6], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 3)
    prob = O.Problem(spec)
    free, sdof = prob.free_dofs(1), prob.schwarz_dofs(1)
    U, A, S = [], [], []
    u, v, a = prob.state(1)
    U.append(u.reshape(-1)[free]); A.append(a.reshape(-1)[free]); S.append(u.reshape(-1)[sdof])
    v0 = v.reshape(-1)[free].copy()
    for _ in range(80):
        prob.step()
        u, _, a = prob.state(1)
        U.append(u.reshape(-1)[free]); A.append(a.reshape(-1)[free]); S.append(u.reshape(-1)[sdof])
    U, A, S = np.array(U), np.array(A), np.array(S)
    lams = OF.lambda_grid()
    ref_err, ref_best, ref_ops = OF.select_lambda(U.T, A.T, S.T, v0, r=6, lambdas=lams, dt=spec.dt, k=3, r_s=4)
    got = osam.opinf_select(U, A, S, v0, r=6, lambdas=lams, dt=spec.dt, substeps=3, r_s=4)
    _compare(got["errors"], ref_err)
    assert got["best"] == ref_best
    # the returned operators are the fit at the selected lambda
    fit = osam.opinf_fit(U, A, S, r=6, lam=float(lams[ref_best]), r_s=4)
    for key in ("K", "c"):
        assert np.allclose(np.abs(got[key]), np.abs(fit[key]), rtol=1e-10, atol=1e-12 * np.abs(fit[key]).max())


def test_selection_penalises_non_finite_rollouts(gpu):
    """A rollout step above the oscillators' stability limit (omega dt up to 2.4) overflows for every
    weakly regularised candidate; an overwhelmingly regularised one (operators ~ 0) stays finite and
    wins; with no finite candidate the call reports ENONFINITE."""
    U, A, S, v0 = _known_quadratic_trajectory()
    lams = np.array([1e-10, 1e-6, 1e15])
    ref_err, ref_best, _ = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.6, k=1, r_s=2)
    got = osam.opinf_select(U.T, A.T, S.T, v0, r=5, lambdas=lams, dt=0.6, substeps=1, r_s=2)
    assert not np.isfinite(ref_err[0]) and got["errors"][0] >= 1e300
    assert got["best"] == ref_best == 2
    with pytest.raises(osam.OsamError) as ei:
        osam.opinf_select(U.T, A.T, S.T, v0, r=5, lambdas=lams[:2], dt=0.6, substeps=1, r_s=2)
    assert ei.value.code == osam.ENONFINITE


def test_single_candidate_selection_is_the_fit_at_that_lambda(gpu):
    """One candidate: it is selected, its E(lambda) matches the oracle's, and the returned operators
    are the plain fit at that lambda."""
    U, A, S, v0 = _known_quadratic_trajectory()
    ref_err, ref_best, _ = OF.select_lambda(U, A, S, v0, r=5, lambdas=[1e-6], dt=0.02, k=1, r_s=2)
    got = osam.opinf_select(U.T, A.T, S.T, v0, r=5, lambdas=[1e-6], dt=0.02, substeps=1, r_s=2)
    assert got["best"] == ref_best == 0 and got["lambda"] == 1e-6
    _compare(got["errors"], ref_err)
    fit = osam.opinf_fit(U.T, A.T, S.T, r=5, lam=1e-6, r_s=2)
    for key in ("K", "H", "B", "c"):
        assert np.array_equal(got[key], fit[key]), key


def test_cubic_selection_on_a_duffing_model_matches_oracle(gpu):
    """Algorithm 3 with cubic candidates on the oracle-pinned model with Duffing-type cubic terms."""
    from .test_oracle_fit_adjoint import CUBIC_SCALE
    U, A, S, v0 = _known_quadratic_trajectory(cubic=CUBIC_SCALE, seed=4)
    lams = OF.lambda_grid()
    ref_err, ref_best, _ = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.02, k=1, r_s=2, cubic=True)
    got = osam.opinf_select(U.T, A.T, S.T, v0, r=5, lambdas=lams, dt=0.02, substeps=1, r_s=2, cubic=True)
    _compare(got["errors"], ref_err)
    assert got["best"] == ref_best and got["errors"][got["best"]] < 1e-6
