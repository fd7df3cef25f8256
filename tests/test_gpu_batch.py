"""Batched contexts and the graph-captured controller step.

Every instance of a batch must follow exactly its own single-instance run (same kernels, same
fixed-order reductions, converged instances frozen), and the CUDA-graph step (Schwarz iterations in
a while node) must reproduce the host-driven loop.  Also: batch instances against the CPU oracle.
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


def _synthetic_rom(spec, i, r, rs, seed):
    sd = spec.subdomains[i]
    nxy = sd.dims[0]
    n_sdof = 3 * (nxy + 1) ** 2
    n_free = 3 * sd.n_nodes - n_sdof
    return W.synthetic_rom_operators(n_free, n_sdof, r, rs, seed)


def test_graph_step_equals_host_loop(gpu):
    spec = W.fom_fom_plain()
    a = osam.Problem(spec, scatter=osam.SCATTER_GATHER, graph=True)
    b = osam.Problem(spec, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(4):
        ra, rb = a.step(), b.step()
        assert ra["iterations"] == rb["iterations"] and ra["cnum"] == rb["cnum"]
    for i in range(2):
        for f in range(3):
            assert np.array_equal(a.state(i)[f], b.state(i)[f])


def test_graph_step_hybrid_equals_host_loop(gpu):
    spec = W.bar_chain("h", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=6)
    ops = {1: _synthetic_rom(spec, 1, 5, 4, 1)}
    a = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=True)
    b = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(3):
        ra, rb = a.step(), b.step()
        assert ra["iterations"] == rb["iterations"]
    assert np.array_equal(a.state(0)[0], b.state(0)[0])
    assert np.array_equal(a.reduced_state(1)[0], b.reduced_state(1)[0])


@pytest.mark.parametrize("graph", [True, False])
def test_batch_instances_equal_single_runs(gpu, graph):
    """Uneven FOM-FOM pairs (different n, E, nu, amplitude): each batch instance equals its own run."""
    specs = W.batched_samples(n_samples=5, n_min=3, n_max=7, rom=False)
    for s in specs:
        s.max_iters = 20
    batch = osam.Batch(specs, scatter=osam.SCATTER_GATHER, graph=graph)
    singles = [osam.Problem(s, scatter=osam.SCATTER_GATHER, graph=graph) for s in specs]
    for _ in range(3):
        per, tot = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
        assert tot["element_updates"] == sum(r["element_updates"] for r in reps)
    for n, p in enumerate(singles):
        for i in range(2):
            for f in range(3):
                assert np.array_equal(batch.state(i, inst=n)[f], p.state(i)[f])


def test_batch_fom_rom_instances_equal_single_runs(gpu):
    specs = W.batched_samples(n_samples=4, n_min=3, n_max=6, rom=True)
    ops = []
    for k, s in enumerate(specs):
        s.max_iters = 8
        ops.append({1: _synthetic_rom(s, 1, 4 + k, 3, 100 + k)})
    batch = osam.Batch(specs, rom_ops=ops, scatter=osam.SCATTER_GATHER)
    singles = [osam.Problem(s, rom_ops=o, scatter=osam.SCATTER_GATHER) for s, o in zip(specs, ops)]
    for _ in range(2):
        per, _ = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
    for n, p in enumerate(singles):
        assert np.array_equal(batch.state(0, inst=n)[0], p.state(0)[0])
        assert np.array_equal(batch.reduced_state(1, inst=n)[0], p.reduced_state(1)[0])


def test_batch_instances_match_oracle(gpu):
    specs = W.batched_samples(n_samples=3, n_min=3, n_max=5, rom=False)
    batch = osam.Batch(specs)
    refs = [O.Problem(s) for s in specs]
    hist = {(n, i): ([], []) for n in range(3) for i in range(2)}
    for _ in range(3):
        batch.step()
        for n, ref in enumerate(refs):
            ref.step()
            for i in range(2):
                hist[(n, i)][0].append(batch.state(i, inst=n)[0])
                hist[(n, i)][1].append(ref.state(i)[0])
    for key, (g, r) in hist.items():
        assert rel_l2(g, r) < 1e-9, key


def test_batch_rejects_mixed_topology(gpu):
    a = W.fom_fom_plain()
    b = W.bar_chain("x", 6, [12, 12, 12], ["fom", "fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20)
    with pytest.raises(osam.OsamError) as ei:
        osam.Batch([a, b])
    assert ei.value.code == osam.EINVAL


def test_autotuner_reports_a_valid_configuration(gpu):
    p = osam.Problem(W.fom_opinf_hybrid(8, 16, rom=False))
    t = p.tuning()
    assert t["scatter"] in ("gather", "atomic") and t["element_block"] in (64, 128, 256)


def _manual_step(p, spec, iterations):
    """One controller step through the manual ABI: subdomains advanced one after another in chain
    order, every transfer after its source's advance (no overlap of subdomains)."""
    p.begin_interval()
    n_sd = len(spec.subdomains)
    for n in range(1, iterations + 1):
        if n > 1:
            p.restore_interval()
        for s in range(n_sd):
            p.advance(s)
            for c in spec.couplings:
                if c.src == s:
                    p.transfer(c.src, c.dst)
        cnum, cden = p.criterion()
    return cnum, cden


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("kinds", [["fom", "rom"], ["fom", "rom", "fom"]])
def test_rom_pipelined_behind_fom_equals_sequential_order(gpu, graph, kinds):
    """schwarz_step advances a ROM that follows its FOM source one substep behind it on a second
    stream; the result must equal the strictly sequential manual sequence bit for bit."""
    nz = [6] * len(kinds)
    spec = W.bar_chain("pipe", 3, nz, kinds, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 7, max_iters=6)
    ops = {1: _synthetic_rom(spec, 1, 5, 4, 11)} if len(kinds) == 2 else {1: _chain_rom(spec, 5, 6, 12)}
    a = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=graph)
    b = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(3):
        rep = a.step()
        cnum, cden = _manual_step(b, spec, rep["iterations"])
        assert cnum == rep["cnum"] and cden == rep["cden"]
    for i, sd in enumerate(spec.subdomains):
        if sd.kind == "fom":
            assert np.array_equal(a.state(i)[0], b.state(i)[0])
        else:
            assert np.array_equal(a.reduced_state(i)[0], b.reduced_state(i)[0])


def _chain_rom(spec, r, rs, seed):
    """Stand-in operators for the middle subdomain of a chain (Schwarz faces at both ends)."""
    sd = spec.subdomains[1]
    n_sdof = 2 * 3 * (sd.dims[0] + 1) ** 2
    return W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof, n_sdof, r, rs, seed)


@pytest.mark.parametrize("tiled", ["tiled", "tiled_lowreg"])
@pytest.mark.parametrize("material", ["le", "nh", "svk"])
def test_tiled_force_equals_untiled(gpu, material, tiled):
    """The tiled FP64 force shares the edge interpolation between neighbouring elements with the same
    per-value arithmetic: states equal the untiled gather path bit for bit (ragged tiles included),
    also for its build capped at 128 registers."""
    spec = W.bar_chain("tile", 11, [13, 9], ["fom", "fom"], material, 1e9, 0.3, 1000.0, 2e-3, 1e-6, 5)
    mode = osam.SCATTER_GATHER_TILED if tiled == "tiled" else osam.SCATTER_GATHER_TILED_LOWREG
    a = osam.Problem(spec, scatter=mode)
    b = osam.Problem(spec, scatter=osam.SCATTER_GATHER)
    assert a.tuning()["tiled"] and not b.tuning()["tiled"]
    assert a.tuning()["register_cap"] == (128 if tiled == "tiled_lowreg" else 0)
    for _ in range(3):
        ra, rb = a.step(), b.step()
        assert ra["iterations"] == rb["iterations"] and ra["cnum"] == rb["cnum"]
    for i in range(2):
        for f in range(3):
            assert np.array_equal(a.state(i)[f], b.state(i)[f])


def test_tiled_batch_equals_untiled_single_runs(gpu):
    specs = W.batched_samples(n_samples=4, n_min=3, n_max=9, rom=False)
    batch = osam.Batch(specs, scatter=osam.SCATTER_GATHER_TILED)
    singles = [osam.Problem(s, scatter=osam.SCATTER_GATHER) for s in specs]
    for _ in range(2):
        per, _ = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
    for n, p in enumerate(singles):
        for i in range(2):
            assert np.array_equal(batch.state(i, inst=n)[0], p.state(i)[0])
