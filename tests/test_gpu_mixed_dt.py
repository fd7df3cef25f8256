"""GPU parity with a different time step on each subdomain (n_i substeps per controller step, Delta
t_i = T / n_i) against the oracle: Schwarz data pass through the temporal interpolant Xi, linear in
time between the source levels that bracket each destination level (Sec. 4.1).

Covers FOM-FOM (explicit / explicit, explicit / implicit), FOM-ROM in both directions of refinement,
counts that do not divide one another, the graph-captured step against the host loop, batches, the
rigid-translation invariant on the GPU alone, and the validation of the counts.
"""
import numpy as np
import pytest

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


def _setup(spec, counts, integrators=None):
    for i, sd in enumerate(spec.subdomains):
        sd.n_substeps = counts[i]
        if integrators:
            sd.integrator = integrators[i]
    return spec


def _synthetic_rom(spec, i, r, rs, seed):
    sd = spec.subdomains[i]
    n_sdof = 3 * (sd.dims[0] + 1) ** 2
    return W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof, n_sdof, r, rs, seed)


def _compare(spec, n_ctrl, rom_ops=None, tol=1e-9, its_slack=1, **kw):
    gpu = osam.Problem(spec, rom_ops=rom_ops, **kw)
    ref = O.Problem(spec, rom_ops=rom_ops)
    n_sd = len(spec.subdomains)
    hg = {i: [] for i in range(n_sd)}
    hr = {i: [] for i in range(n_sd)}
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] in (osam.OK, osam.MAXITER) and rr["status"] in (O.OK, O.MAXITER)
        assert its_slack is None or abs(rg["iterations"] - rr["iterations"]) <= its_slack
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


@pytest.mark.parametrize("counts", [(6, 4), (5, 3), (3, 7), (2, 6)])
def test_fom_fom_explicit_mixed_steps(gpu, counts):
    spec = _setup(W.bar_chain("mx", 3, [7, 6], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                              max_iters=40), counts)
    _compare(spec, 3)


@pytest.mark.parametrize("counts", [(6, 3), (4, 8)])
def test_fom_fom_explicit_implicit_mixed_steps(gpu, counts):
    """The paper's explicit / implicit pairing with different steps on the two subdomains."""
    spec = _setup(W.bar_chain("mxi", 3, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                              max_iters=40), counts, ("explicit", "implicit"))
    _compare(spec, 3)


@pytest.mark.parametrize("counts", [(6, 3), (3, 6), (4, 6)])
def test_fom_rom_mixed_steps(gpu, counts):
    """FOM -> ROM (publish into the ROM's boundary snapshots) and ROM -> FOM (reconstruction of the
    interpolated reduced state) across different levels."""
    spec = _setup(W.bar_chain("mxr", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 6,
                              max_iters=6), counts)
    ops = {1: _synthetic_rom(spec, 1, 5, 4, 7)}
    _compare(spec, 3, rom_ops=ops)


def test_three_subdomains_three_steps(gpu):
    spec = _setup(W.bar_chain("mx3", 3, [6, 6, 6], ["fom", "fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                              max_iters=40), (6, 4, 3), ("explicit", "implicit", "explicit"))
    _compare(spec, 2)


@pytest.mark.parametrize("graph", [True, False])
def test_rigid_translation_stays_exact(gpu, graph):
    """Rigid motion at constant velocity with counts 5 and 3: u = V t to rounding on both subdomains."""
    p = W.bar_chain("tr", 3, [6, 6], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 0.0, 1e-6, 6, max_iters=10)
    V = np.array([0.3, -0.2, 0.5])
    for sd, n in zip(p.subdomains, (5, 3)):
        sd.dirichlet = np.zeros(sd.n_nodes, np.uint8)
        sd.u0 = np.zeros((sd.n_nodes, 3))
        sd.v0 = np.tile(V, (sd.n_nodes, 1))
        sd.n_substeps = n
    g = osam.Problem(p, graph=graph)
    t = 0.0
    for _ in range(3):
        g.step()
        t += p.dt * p.n_substeps
    for i in range(2):
        u, v, _ = g.state(i)
        assert np.abs(u - V * t).max() < 1e-13 * np.abs(V).max() * t
        assert np.abs(v - V).max() < 1e-12 * np.abs(V).max()
    g.close()


def test_graph_equals_host_loop_with_mixed_steps(gpu):
    spec = _setup(W.bar_chain("mg", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 6,
                              max_iters=6), (6, 4))
    ops = {1: _synthetic_rom(spec, 1, 5, 4, 8)}
    a = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=True)
    b = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(3):
        ra, rb = a.step(), b.step()
        assert ra["iterations"] == rb["iterations"]
    assert np.array_equal(a.state(0)[0], b.state(0)[0])
    assert np.array_equal(a.reduced_state(1)[0], b.reduced_state(1)[0])


def test_batch_with_mixed_steps_equals_single_runs(gpu):
    specs = W.batched_samples(n_samples=3, n_min=3, n_max=6, rom=False)
    for s in specs:
        s.max_iters = 20
        _setup(s, (20, 8))
    batch = osam.Batch(specs, scatter=osam.SCATTER_GATHER)
    singles = [osam.Problem(s, scatter=osam.SCATTER_GATHER) for s in specs]
    for _ in range(2):
        per, tot = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
        assert tot["element_updates"] == sum(r["element_updates"] for r in reps)
    for n, p in enumerate(singles):
        for i in range(2):
            for f in range(3):
                assert np.array_equal(batch.state(i, inst=n)[f], p.state(i)[f])


def test_element_updates_count_each_subdomains_substeps(gpu):
    spec = _setup(W.bar_chain("cnt", 3, [6, 6], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 6,
                              max_iters=5), (6, 3))
    g = osam.Problem(spec)
    r = g.step()
    ne = spec.subdomains[0].n_elements
    assert r["element_updates"] == r["iterations"] * (6 + 3) * ne
    g.close()


def test_substep_counts_must_agree_across_instances(gpu):
    specs = W.batched_samples(n_samples=2, n_min=3, n_max=4, rom=False)
    _setup(specs[0], (20, 10))
    _setup(specs[1], (20, 5))
    with pytest.raises(osam.OsamError) as e:
        osam.Batch(specs)
    assert e.value.code == osam.EINVAL


@pytest.mark.parametrize("steppers,counts", [(("implicit", "implicit"), (10, 10)), (("explicit", "implicit"), (10, 10)),
                                             (("explicit", "explicit"), (10, 10)), (("explicit", "implicit"), (10, 5))])
def test_wave1d_stepper_matrix_matches_dalembert(gpu, steppers, counts):
    """The 1D bar of Sec. 5.1 on the paper's decomposition and mesh (dz = 1e-3 m) with each time-stepper
    pairing of its table of steppers (implicit / implicit, explicit / implicit, explicit / explicit at
    dt = 1e-7 s, and explicit 1e-7 s / implicit 2e-7 s), controller intervals of 1e-6 s: after the
    pulse has crossed both Schwarz boundaries (t = 3e-4 s) the FOM-FOM solution matches the exact
    solution Eq. disp_exact to the discretisation error (the explicit / explicit run of the oracle at
    this resolution: 2.1e-3 relative L2)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wave1d_symmetric_gaussian.json")))
    a, b, s = g["initial_condition"]["a"], g["initial_condition"]["b"], g["initial_condition"]["s"]
    c = (g["E"] / g["rho"]) ** 0.5
    T = g["T"]

    def exact(z, t):
        f = lambda x: a * np.exp(-((x - b) ** 2) / (2 * s * s))  # noqa: E731
        return 0.5 * f(z - c * t) + 0.5 * f(z + c * t) - 0.5 * f(z - c * (T - t)) - 0.5 * f(z + c * (T - t))

    p = W.wave1d(n_elem=1000, dt=1e-7, subdomains=True, n_substeps=10)
    _setup(p, counts, steppers)
    prob = osam.Problem(p)
    t = 0.0
    for _ in range(300):
        assert prob.step()["status"] == osam.OK
        t += p.dt * p.n_substeps
    num = den = 0.0
    for i in range(2):
        u = prob.state(i)[0][:, 2]
        ex = exact(p.subdomains[i].node_coords()[:, 2], t)
        num += np.sum((u - ex) ** 2)
        den += np.sum(ex ** 2)
    prob.close()
    assert np.sqrt(num / den) < 5e-3


@pytest.mark.parametrize("precision,tol,slack", [(osam.F32X2_FORCE, 1e-9, 1), (osam.FP32_FORCE, 1e-5, None)])
def test_mixed_steps_with_reduced_force_precision(gpu, precision, tol, slack):
    """The double-float and FP32 force paths under different substep counts (their node kernels take
    the per-subdomain time steps and history levels). FP32 force rounding sits above the Schwarz
    tolerance, so that run may stop on the iteration cap: its iteration count is not compared."""
    spec = _setup(W.bar_chain("mxp", 4, [8, 7], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                              max_iters=8), (6, 4))
    _compare(spec, 3, tol=tol, its_slack=slack, precision=precision)


def test_additive_with_mixed_steps_graph_equals_host(gpu):
    spec = _setup(W.bar_chain("mxa", 3, [6, 6, 6], ["fom", "rom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 6,
                              max_iters=8), (6, 4, 3))
    spec.schwarz = "additive"
    from .test_gpu_additive import _rom_ops
    ops = {1: _rom_ops(spec, 1, 5, 4, 9)}
    _compare(spec, 2, rom_ops=ops)
    a = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=True)
    b = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(2):
        assert a.step()["iterations"] == b.step()["iterations"]
    for i in (0, 2):
        assert np.array_equal(a.state(i)[0], b.state(i)[0])
    assert np.array_equal(a.reduced_state(1)[0], b.reduced_state(1)[0])


def test_single_substep_implicit_subdomain(gpu):
    """The degenerate count: an implicit subdomain taking the whole controller interval as one step
    (levels 0 and 1 only) against an explicit one with six substeps."""
    spec = _setup(W.bar_chain("one", 3, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                              max_iters=40), (6, 1), ("explicit", "implicit"))
    _compare(spec, 3)


@pytest.mark.parametrize("graph", [True, False])
def test_criterion_sums_match_oracle(gpu, graph):
    """The c_num, c_den of Eq. conv_criterion after two sweeps (per-subdomain steps 1.5 us and 2 us, a
    FOM and a ROM) against the oracle's, whose sums are pinned to the written-out formula."""
    from .test_oracle_pins import _free_mask
    spec = W.bar_chain("crit", 3, [7, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6, max_iters=2)
    spec.subdomains[0].n_substeps, spec.subdomains[1].n_substeps = 4, 3
    n_sdof = 3 * int(np.asarray(spec.couplings[[c.dst for c in spec.couplings].index(1)].nodes, bool).sum())
    ops = {1: W.synthetic_rom_operators(int(_free_mask(spec, 1).sum()), n_sdof, 5, 4, 31)}
    g = osam.Problem(spec, rom_ops=ops, graph=graph)
    ref = O.Problem(spec, rom_ops=ops)
    for _ in range(2):
        rg, rr = g.step(), ref.step()
        assert rg["iterations"] == rr["iterations"] == 2
        assert abs(rg["cden"] - rr["cden"]) <= 1e-12 * rr["cden"]
        assert abs(rg["cnum"] - rr["cnum"]) <= 1e-6 * rr["cnum"]
    g.close()
