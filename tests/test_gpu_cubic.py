"""GPU parity of cubic OpInf (COpInf: qdd = K q + H kron_c(q) + C kron3_c(q) + B ghat + c) against the
oracle: the GPU fit with the compressed Kronecker cube, the cubic ROM step in FOM-COpInf and
COpInf-COpInf couplings (the paper's pairing with Saint Venant-Kirchhoff FOMs), batches of cubic
instances, and the regularisation selection of Algorithm 3 with cubic candidates.
"""
import numpy as np
import pytest

from oracle import fit as OF
from oracle import oracle as O
from paper_2511_20687_gb300 import osam
from paper_2511_20687_gb300 import workloads as W

from .helpers import rel_l2

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


def _cubic_data(seed=41, n=700, ns=120, nsd=40, r=4, rs=3):
    rng = np.random.default_rng(seed)
    nq, nc = r * (r + 1) // 2, r * (r + 1) * (r + 2) // 6
    Q = np.diag(np.linspace(5.0, 1.0, r)) @ rng.standard_normal((r, ns))
    Phi_t, _ = np.linalg.qr(rng.standard_normal((n, r)))
    PhiS_t, _ = np.linalg.qr(rng.standard_normal((nsd, rs)))
    G = np.diag(np.linspace(3.0, 1.0, rs)) @ rng.standard_normal((rs, ns))
    K = rng.standard_normal((r, r))
    H = 0.1 * rng.standard_normal((r, nq))
    Cc = 0.05 * rng.standard_normal((r, nc))
    B = rng.standard_normal((r, rs))
    c = rng.standard_normal(r)
    Qdd = K @ Q + H @ OF.kron_c(Q) + Cc @ OF.kron3_c(Q) + B @ G + c[:, None]
    U = (Phi_t @ Q).T + 1e-3 * rng.standard_normal((ns, n))
    A = (Phi_t @ Qdd).T
    S = (PhiS_t @ G).T + 1e-3 * rng.standard_normal((ns, nsd))
    return U, A, S, r, rs, rng


def test_cubic_fit_matches_oracle(gpu):
    """Same snapshots: sign-aligned bases agree, and so do the full-space accelerations of the fitted
    cubic models at fresh reduced states (both primal-size and dual-size regressions)."""
    for ns in (120, 40):   # d = r + nq + nc + rs + 1 = 38: primal at 120 snapshots, dual at 40
        U, A, S, r, rs, rng = _cubic_data(ns=ns)
        ref = OF.opinf_fit(U.T, A.T, S.T, r=r, lam=1e-6, r_s=rs, cubic=True)
        got = osam.opinf_fit(U, A, S, r=r, lam=1e-6, r_s=rs, cubic=True)
        sg = np.sign(np.sum(got["Phi"] * ref["Phi"], axis=0))
        ss = np.sign(np.sum(got["Phi_S"] * ref["Phi_S"], axis=0))
        assert np.abs(got["Phi"] * sg - ref["Phi"]).max() < 1e-9
        qs = rng.standard_normal((r, 8))
        gs = rng.standard_normal((rs, 8))
        for k in range(8):
            want = ref["Phi"] @ OF.rom_rhs(ref["K"], ref["H"], ref["B"], ref["c"], qs[:, k], gs[:, k], ref["C"])
            have = got["Phi"] @ OF.rom_rhs(got["K"], got["H"], got["B"], got["c"], sg * qs[:, k], ss * gs[:, k],
                                           got["C"])
            assert np.linalg.norm(have - want) < 1e-7 * np.linalg.norm(want)


def _svk_training(spec_ff, i, n_ctrl):
    prob = O.Problem(spec_ff)
    free, sdof = prob.free_dofs(i), prob.schwarz_dofs(i)
    U, A, S = [], [], []
    for _ in range(n_ctrl):
        prob.step()
        u, _, a = prob.state(i)
        U.append(u.reshape(-1)[free]); A.append(a.reshape(-1)[free]); S.append(u.reshape(-1)[sdof])
    return np.array(U), np.array(A), np.array(S)


def _compare(spec, n_ctrl, rom_ops, tol=1e-9, **kw):
    gpu = osam.Problem(spec, rom_ops=rom_ops, **kw)
    ref = O.Problem(spec, rom_ops=rom_ops)
    hg = {i: [] for i in range(len(spec.subdomains))}
    hr = {i: [] for i in range(len(spec.subdomains))}
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] in (osam.OK, osam.MAXITER) and rr["status"] in (O.OK, O.MAXITER)
        assert abs(rg["iterations"] - rr["iterations"]) <= 1
        for i, sd in enumerate(spec.subdomains):
            if sd.kind == "fom":
                hg[i].append(gpu.state(i)[0].copy())
                hr[i].append(ref.state(i)[0].copy())
            else:
                hg[i].append(gpu.reduced_state(i)[0].copy())
                hr[i].append(ref.rom_state(i)[0].copy())
    gpu.close()
    for i in hg:
        assert rel_l2(hg[i], hr[i]) < tol, (i, rel_l2(hg[i], hr[i]))


@pytest.fixture(scope="module")
def svk_cubic_ops(gpu):
    """COpInf ROMs of both halves of a Saint Venant-Kirchhoff bar, fitted by the oracle on a FOM-FOM
    run (the paper's bolted-joint pairing of the material and the model)."""
    pf = W.bar_chain("svkff", 3, [6, 6], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 4)
    ops = {}
    for i in (0, 1):
        U, A, S = _svk_training(pf, i, 60)
        ops[i] = OF.opinf_fit(U.T, A.T, S.T, r=5, lam=1e-6, r_s=4, cubic=True)
    return ops


@pytest.mark.parametrize("kinds", [("fom", "rom"), ("rom", "fom"), ("rom", "rom")])
def test_svk_copinf_couplings(gpu, svk_cubic_ops, kinds):
    spec = W.bar_chain("svkc", 3, [6, 6], list(kinds), "svk", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 4, max_iters=12)
    ops = {i: svk_cubic_ops[i] for i, k in enumerate(kinds) if k == "rom"}
    _compare(spec, 4, ops)


def test_cubic_rom_batch_equals_single_runs(gpu, svk_cubic_ops):
    specs = []
    for amp in (1e-3, 2e-3, 1.5e-3):
        s = W.bar_chain("svkb", 3, [6, 6], ["fom", "rom"], "svk", 1e9, 0.3, 1000.0, amp, 1e-6, 4, max_iters=10)
        specs.append(s)
    ops = [{1: svk_cubic_ops[1]} for _ in specs]
    batch = osam.Batch(specs, rom_ops=ops, scatter=osam.SCATTER_GATHER)
    singles = [osam.Problem(s, rom_ops=o, scatter=osam.SCATTER_GATHER) for s, o in zip(specs, ops)]
    for _ in range(3):
        per, _ = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
    for n, p in enumerate(singles):
        assert np.array_equal(batch.state(0, inst=n)[0], p.state(0)[0])
        assert np.array_equal(batch.reduced_state(1, inst=n)[0], p.reduced_state(1)[0])


def test_cubic_selection_matches_oracle(gpu):
    """Algorithm 3 with cubic candidates on Saint Venant-Kirchhoff training snapshots."""
    pf = W.bar_chain("svks", 3, [6, 6], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 3)
    prob = O.Problem(pf)
    free, sdof = prob.free_dofs(1), prob.schwarz_dofs(1)
    u, v, a = prob.state(1)
    U, A, S = [u.reshape(-1)[free]], [a.reshape(-1)[free]], [u.reshape(-1)[sdof]]
    v0 = v.reshape(-1)[free].copy()
    for _ in range(50):
        prob.step()
        u, _, a = prob.state(1)
        U.append(u.reshape(-1)[free]); A.append(a.reshape(-1)[free]); S.append(u.reshape(-1)[sdof])
    U, A, S = np.array(U), np.array(A), np.array(S)
    lams = OF.lambda_grid()
    ref_err, ref_best, _ = OF.select_lambda(U.T, A.T, S.T, v0, r=4, lambdas=lams, dt=pf.dt, k=3, r_s=3, cubic=True)
    got = osam.opinf_select(U, A, S, v0, r=4, lambdas=lams, dt=pf.dt, substeps=3, r_s=3, cubic=True)
    for eg, er in zip(got["errors"], ref_err):
        if np.isfinite(er):
            assert abs(eg - er) <= 1e-6 * er + 1e-9, (eg, er)
        else:
            assert not np.isfinite(eg) or eg >= 1e300
    assert got["best"] == ref_best
    assert "C" in got and got["C"].shape == (4, 20)


def test_cubic_rom_with_its_own_time_step(gpu, svk_cubic_ops):
    """FOM-COpInf with the cubic ROM taking half as many substeps (twice the step) as the SVK FOM:
    the ROM's boundary data pass through the temporal interpolant, its trace back to the FOM too."""
    spec = W.bar_chain("svkm", 3, [6, 6], ["fom", "rom"], "svk", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 4, max_iters=12)
    spec.subdomains[1].n_substeps = 2
    _compare(spec, 3, {1: svk_cubic_ops[1]})


def test_cubic_rom_at_the_maximum_rank(gpu):
    """COpInf at r = 128, the largest cubic rank the library takes (C has 357,760 columns, 366 MB):
    seeded stand-in operators with a cubic part that moves the reduced state by ~1e-5 relative,
    four orders of magnitude above the parity bar, coupled to an SVK FOM; r = 129 is rejected."""
    from .test_gpu_additive import _rom_ops
    r, rs = 128, 16
    spec = W.bar_chain("c128", 6, [8, 8], ["fom", "rom"], "svk", 1e9, 0.3, 1000.0, 1e-3, 1e-6, 10, max_iters=8)
    ops = _rom_ops(spec, 1, r, rs, 12)
    nc = r * (r + 1) * (r + 2) // 6
    ops["C"] = 1e12 * np.random.default_rng(13).standard_normal((r, nc)) / np.sqrt(nc)
    _compare(spec, 2, {1: ops})
    big = _rom_ops(spec, 1, r + 1, rs, 12)
    big["C"] = np.zeros((r + 1, (r + 1) * (r + 2) * (r + 3) // 6))
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec, rom_ops={1: big})
    assert ei.value.code == osam.EINVAL
