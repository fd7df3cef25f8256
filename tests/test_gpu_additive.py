"""GPU parity of the additive Schwarz variant (Remark additive_sam: every subdomain advances from the
previous iteration's data, concurrently on its own stream) and of OpInf-OpInf coupling, against the
oracle; graph-captured step against the host loop; batches against single runs.
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


def _rom_ops(spec, i, r, rs, seed):
    """Seeded stand-in operators sized for subdomain i: free dofs exclude its Schwarz nodes and its
    clamped components."""
    sd = spec.subdomains[i]
    snodes = np.zeros(sd.n_nodes, bool)
    for c in spec.couplings:
        if c.dst == i:
            snodes |= np.asarray(c.nodes, bool)
    dm = np.zeros(sd.n_nodes, np.uint8) if sd.dirichlet is None else np.asarray(sd.dirichlet)
    clamped = sum(int(((dm[~snodes] >> b) & 1).sum()) for b in range(3))
    n_sdof = 3 * int(snodes.sum())
    return W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof - clamped, n_sdof, r, rs, seed)


def _compare(spec, n_ctrl, rom_ops=None, tol=1e-9, **kw):
    gpu = osam.Problem(spec, rom_ops=rom_ops, **kw)
    ref = O.Problem(spec, rom_ops=rom_ops)
    n_sd = len(spec.subdomains)
    hg = {i: [] for i in range(n_sd)}
    hr = {i: [] for i in range(n_sd)}
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] in (osam.OK, osam.MAXITER) and rr["status"] in (O.OK, O.MAXITER)
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


@pytest.mark.parametrize("material", ["le", "nh"])
def test_additive_fom_fom(gpu, material):
    spec = W.bar_chain("af", 3, [7, 6], ["fom", "fom"], material, 1e9, 0.25, 1000.0, 2e-3, 1e-6, 5, max_iters=60)
    spec.schwarz = "additive"
    _compare(spec, 3)


def test_additive_fom_rom(gpu):
    spec = W.bar_chain("ar", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=8)
    spec.schwarz = "additive"
    _compare(spec, 3, rom_ops={1: _rom_ops(spec, 1, 5, 4, 21)})


@pytest.mark.parametrize("schwarz", ["multiplicative", "additive"])
def test_rom_rom(gpu, schwarz):
    """OpInf-OpInf coupling: ROM -> ROM reconstruction into the other ROM's boundary snapshots."""
    spec = W.bar_chain("rr", 3, [6, 6], ["rom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=8)
    spec.schwarz = schwarz
    ops = {0: _rom_ops(spec, 0, 6, 4, 22), 1: _rom_ops(spec, 1, 5, 4, 23)}
    _compare(spec, 3, rom_ops=ops)


def test_additive_three_subdomains_mixed(gpu):
    """Three subdomains, an implicit middle one and different substep counts, additive sweeps (the
    implicit subdomain's host-driven Newton loop runs while the explicit ones are in flight)."""
    spec = W.bar_chain("a3", 3, [6, 6, 6], ["fom", "fom", "rom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                       max_iters=12)
    spec.schwarz = "additive"
    spec.subdomains[1].integrator = "implicit"
    spec.subdomains[1].n_substeps = 3
    spec.subdomains[2].n_substeps = 4
    _compare(spec, 2, rom_ops={2: _rom_ops(spec, 2, 5, 4, 24)})


def test_additive_graph_equals_host_loop(gpu):
    spec = W.bar_chain("ag", 3, [6, 6, 6], ["fom", "rom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5,
                       max_iters=8)
    spec.schwarz = "additive"
    ops = {1: _rom_ops(spec, 1, 5, 4, 25)}
    a = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=True)
    b = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER, graph=False)
    for _ in range(3):
        ra, rb = a.step(), b.step()
        assert ra["iterations"] == rb["iterations"] and ra["cnum"] == rb["cnum"]
    for i in (0, 2):
        for f in range(3):
            assert np.array_equal(a.state(i)[f], b.state(i)[f])
    assert np.array_equal(a.reduced_state(1)[0], b.reduced_state(1)[0])


def test_additive_batch_equals_single_runs(gpu):
    specs = W.batched_samples(n_samples=3, n_min=3, n_max=6, rom=False)
    for s in specs:
        s.max_iters = 30
        s.schwarz = "additive"
    batch = osam.Batch(specs, scatter=osam.SCATTER_GATHER)
    singles = [osam.Problem(s, scatter=osam.SCATTER_GATHER) for s in specs]
    for _ in range(2):
        per, _ = batch.step()
        reps = [p.step() for p in singles]
        assert [p["iterations"] for p in per] == [r["iterations"] for r in reps]
    for n, p in enumerate(singles):
        for i in range(2):
            for f in range(3):
                assert np.array_equal(batch.state(i, inst=n)[f], p.state(i)[f])


def test_additive_needs_more_iterations_than_multiplicative(gpu):
    """Same fixed point, slower information exchange: additive sweeps take more iterations."""
    spec = W.bar_chain("cmp", 3, [7, 6], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 5, max_iters=60)
    m = osam.Problem(spec)
    spec.schwarz = "additive"
    a = osam.Problem(spec)
    ia = sum(a.step()["iterations"] for _ in range(3))
    im = sum(m.step()["iterations"] for _ in range(3))
    assert ia > im
    u_a, u_m = a.state(1)[0], m.state(1)[0]
    assert np.abs(u_a - u_m).max() < 1e-8 * np.abs(u_m).max()
