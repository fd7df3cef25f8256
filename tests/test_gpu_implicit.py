"""GPU parity of implicit Newmark subdomains (average acceleration, beta = 1/4, gamma = 1/2) against
the oracle, which solves each substep's Newton systems with an assembled tangent and a dense Cholesky
factorisation; the GPU applies the tangent matrix-free inside conjugate gradients.  Both stop Newton at
|R| <= 1e-12 |R(u~)|, so the states agree to the solver tolerance (well inside the 1e-9 relative L2 bar).

Meshes span several element and node blocks with ragged tails; couplings cover implicit-implicit,
explicit-implicit and FOM(implicit)-ROM, time steps up to five times the explicit stability limit,
batches of instances, and the failure path (a non-finite state reported as OSAM_ENONFINITE).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_20687_gb300 import osam
from paper_2511_20687_gb300 import workloads as W

from .helpers import oracle_rom_ops, rel_l2

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


def _implicit(spec, which=None):
    for i, sd in enumerate(spec.subdomains):
        if which is None or i in which:
            sd.integrator = "implicit"
    return spec


def _compare(spec, n_ctrl, rom_ops=None, tol=1e-9, **kw):
    gpu = osam.Problem(spec, rom_ops=rom_ops, **kw)
    ref = O.Problem(spec, rom_ops=rom_ops)
    n_sd = len(spec.subdomains)
    hg = {i: [] for i in range(n_sd)}
    hr = {i: [] for i in range(n_sd)}
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] == osam.OK and rr["status"] == O.OK
        assert abs(rg["iterations"] - rr["iterations"]) <= 1
        for i, sd in enumerate(spec.subdomains):
            if sd.kind == "fom":
                hg[i].append(np.concatenate([f.reshape(-1) for f in gpu.state(i)]))
                hr[i].append(np.concatenate([f.reshape(-1) for f in ref.state(i)]))
            else:
                hg[i].append(gpu.reduced_state(i)[0].copy())
                hr[i].append(ref.rom_state(i)[0].copy())
    gpu.close()
    for i in range(n_sd):
        err = rel_l2(hg[i], hr[i])
        assert err < tol, (i, err)


# OSAM_FP64_TANGENT32 (the Neo-Hookean Newton tangent in FP32, residual and CG vectors in FP64) meets
# the same FP64 Newton test, so it is held to the same bar; linear elastic runs it as FP64
PRECISIONS = [osam.FP64, osam.FP64_TANGENT32]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("material", ["le", "nh"])
def test_single_implicit_fom(gpu, material, precision):
    """5x5x13 bar (325 elements, 504 nodes: several blocks and a ragged tail), displacement, velocity
    and acceleration over 3 controller steps of 6 substeps."""
    spec = _implicit(W.single_bar("imp1", 5, 13, material, 1e9, 0.25, 1000.0, 2e-3, 2e-6, 6))
    _compare(spec, 3, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("material", ["le", "nh"])
def test_implicit_above_explicit_limit(gpu, material, precision):
    """dt = 5x the explicit stability limit: accepted for an implicit subdomain (the explicit one is
    refused with OSAM_ECFL) and still equal to the oracle.  (At twice this pulse amplitude the
    Neo-Hookean Newton solve from the predictor fails on both sides at this step.)"""
    spec = _implicit(W.single_bar("imp5", 4, 9, material, 1e9, 0.25, 1000.0, 1e-3, 1e-6, 4))
    sd = spec.subdomains[0]
    spec.dt = 5.0 * O.stable_dt(sd.dims, sd.h, sd.origin, sd.lam, sd.mu, sd.rho)
    _compare(spec, 3, precision=precision)
    sd.integrator = "explicit"
    with pytest.raises(osam.OsamError) as e:
        osam.Problem(spec)
    assert e.value.code == osam.ECFL


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("material", ["le", "nh"])
def test_implicit_implicit_schwarz(gpu, material, precision):
    spec = _implicit(W.bar_chain("imp2", 3, [8, 8], ["fom", "fom"], material, 1e9, 0.25, 1000.0, 2e-3, 2e-6, 5,
                                 max_iters=40))
    _compare(spec, 3, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("which", [{0}, {1}])
def test_explicit_implicit_schwarz(gpu, which, precision):
    """Neo-Hookean chain with one implicit and one explicit FOM at a common time step."""
    spec = _implicit(W.bar_chain("mix", 4, [9, 7], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 2e-6, 5,
                                 max_iters=40), which)
    _compare(spec, 3, precision=precision)


def test_three_subdomain_chain_mixed(gpu):
    spec = _implicit(W.bar_chain("mix3", 3, [6, 6, 6], ["fom", "fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3,
                                 2e-6, 4, max_iters=40), {1})
    _compare(spec, 2)


def test_implicit_fom_with_rom(gpu):
    """Implicit FOM coupled to a quadratic OpInf ROM trained on an oracle FOM-FOM run."""
    pf = W.bar_chain("fr", 3, [8, 8], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    ops, _ = oracle_rom_ops(pf, 1, 40, r=6, lam=1e-6, r_s=4)
    spec = _implicit(W.bar_chain("fr", 3, [8, 8], ["fom", "rom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5,
                                 max_iters=20), {0})
    _compare(spec, 3, rom_ops={1: ops})


@pytest.mark.parametrize("precision", PRECISIONS)
def test_implicit_batch_equals_single_runs(gpu, precision):
    """Instances with different meshes and materials in one batch follow their own runs bit for bit
    (per-instance Newton / CG masks, fixed-order reductions)."""
    specs = W.batched_samples(n_samples=3, n_min=3, n_max=6, rom=False)
    for s in specs:
        s.max_iters = 20
        _implicit(s, {1})
    batch = osam.Batch(specs, scatter=osam.SCATTER_GATHER, precision=precision)
    singles = [osam.Problem(s, scatter=osam.SCATTER_GATHER, precision=precision) for s in specs]
    for _ in range(2):
        per, _ = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
    for n, p in enumerate(singles):
        for i in range(2):
            for f in range(3):
                assert np.array_equal(batch.state(i, inst=n)[f], p.state(i)[f])


def test_implicit_needs_fp64(gpu):
    spec = _implicit(W.single_bar("imp32", 3, 6, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 2))
    for prec in (osam.FP32_FORCE, osam.F32X2_FORCE):
        with pytest.raises(osam.OsamError) as e:
            osam.Problem(spec, precision=prec)
        assert e.value.code == osam.EINVAL
    osam.Problem(spec, precision=osam.FP64_TANGENT32).close()


def test_fp32_tangent_converges_to_the_fp64_tangent_state(gpu):
    """The FP32 tangent changes only how each Newton system is solved, not the FP64 residual test that
    ends a substep: two implicit Neo-Hookean FOMs at three times the explicit limit agree between the
    two precisions to well inside the effect of the Newton tolerance on the state, within one Schwarz
    iteration per controller step, and the FP32 run does solve Newton systems by CG."""
    spec = _implicit(W.bar_chain("t32", 5, [12, 10], ["fom", "fom"], "nh", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 4,
                                 max_iters=40))
    sd = spec.subdomains[0]
    spec.dt = 3.0 * O.stable_dt(sd.dims, sd.h, sd.origin, sd.lam, sd.mu, sd.rho)
    runs = {}
    for prec in PRECISIONS:
        p = osam.Problem(spec, precision=prec, scatter=osam.SCATTER_GATHER)
        p.profile(False)
        its = [p.step()["iterations"] for _ in range(3)]
        runs[prec] = (its, [p.state(i) for i in range(2)], p.implicit_profile())
        p.close()
    (i64, s64, _), (i32, s32, p32) = runs[osam.FP64], runs[osam.FP64_TANGENT32]
    assert all(abs(a - b) <= 1 for a, b in zip(i64, i32))
    for i in range(2):
        for f in range(3):
            assert rel_l2([s32[i][f]], [s64[i][f]]) < 1e-10
    assert p32["newton_steps"] > 0 and p32["cg_iterations"] >= p32["newton_steps"]


def test_implicit_nonfinite_state_reported(gpu):
    """A non-finite initial displacement makes the Newton residual non-finite: the solve stops, the
    state is marked non-finite and the step returns OSAM_ENONFINITE (as the oracle does)."""
    spec = _implicit(W.single_bar("impnan", 3, 6, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 2))
    sd = spec.subdomains[0]
    sd.u0 = sd.u0.copy()
    sd.u0[sd.n_nodes // 2, 0] = np.nan
    p = osam.Problem(spec)
    with pytest.raises(osam.OsamError) as e:
        p.step()
    assert e.value.code == osam.ENONFINITE
    ref = O.Problem(spec)
    with pytest.raises(O.OracleError) as e:
        ref.step()
    assert e.value.code == O.ENONFINITE


@pytest.mark.parametrize("precision", PRECISIONS)
def test_device_loops_equal_host_loop(gpu, precision):
    """The implicit interval as a graph (Newton and CG as device-side WHILE nodes, inside the captured
    controller step or as a per-interval graph) follows the host-driven Newton / CG loop bit for bit:
    same kernels, same per-instance masks, only the trailing masked CG passes and the host round trips
    are gone.  The explicit subdomain's scatter is pinned to the deterministic gather: left to the
    autotuner, each problem may pick atomics on a mesh this small, whose order of additions varies."""
    spec = _implicit(W.bar_chain("dl", 3, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 2e-6, 5,
                                 max_iters=40), {1})
    a = osam.Problem(spec, graph=True, scatter=osam.SCATTER_GATHER, precision=precision)
    b = osam.Problem(spec, graph=False, scatter=osam.SCATTER_GATHER, precision=precision)
    c = osam.Problem(spec, graph=False, scatter=osam.SCATTER_GATHER, precision=precision)
    c.profile(True)   # kernel-level profiling drives the Newton / CG loops from the host
    for _ in range(3):
        ra, rb, rc = a.step(), b.step(), c.step()
        assert ra["iterations"] == rb["iterations"] == rc["iterations"]
    for i in range(2):
        for f in range(3):
            assert np.array_equal(a.state(i)[f], b.state(i)[f])
            assert np.array_equal(a.state(i)[f], c.state(i)[f])
