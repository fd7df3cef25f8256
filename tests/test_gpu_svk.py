"""GPU parity of the Saint Venant-Kirchhoff material (Appendix A.2) against the oracle: the element
force in every kernel variant (stand-alone, batched gather / atomic / tiled / 128-register, FP32
and double-float), coupled explicit and implicit runs, and the entry points that reject it (the
adjoint covers linear elastic and Neo-Hookean only).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_20687_gb300 import osam
from paper_2511_20687_gb300 import workloads as W

from .helpers import rel_l2

pytestmark = pytest.mark.gpu

LAM, MU = W.lame(1e9, 0.3)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20687_gb300 import build_lib
    build_lib.build()
    osam.load()
    return torch


@pytest.mark.parametrize("per_element", [False, True])
def test_svk_force_matches_oracle(gpu, per_element):
    """Large strains (~10%) so that the quadratic and cubic terms of the force matter; 13x9x11 mesh
    (several blocks and a ragged tail)."""
    torch = gpu
    dims, h = (13, 9, 11), 0.01
    sd = W.Subdomain(kind="fom", dims=dims, h=h, origin=(0.0, 0.0, 0.0))
    X = sd.node_coords()
    rng = np.random.default_rng(31)
    u = np.ascontiguousarray(0.1 * h * np.sin(40.0 * X[:, [2, 0, 1]]) + 1e-4 * rng.standard_normal(X.shape))
    ne = sd.n_elements
    le = LAM * (1 + 0.1 * rng.uniform(-1, 1, ne)) if per_element else None
    me = MU * (1 + 0.1 * rng.uniform(-1, 1, ne)) if per_element else None
    ref = O.internal_force(dims, h, (0.0, 0.0, 0.0), "svk", LAM, MU, u, lam_e=le, mu_e=me).reshape(-1, 3)
    ud = torch.tensor(u, device="cuda")
    fd = torch.empty_like(ud)
    le_d = None if le is None else torch.tensor(le, device="cuda")
    me_d = None if me is None else torch.tensor(me, device="cuda")
    osam.hex8_force(dims, h, "svk", LAM, MU, ud, fd, lam_e=le_d, mu_e=me_d)
    torch.cuda.synchronize()
    assert np.abs(fd.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    # the same force through the allocation-free entry point
    f2 = torch.empty_like(ud)
    L = osam.load()
    if ne <= 32768:
        rc = L.osam_hex8_force_noalloc(dims[0], dims[1], dims[2], h, osam.SAINT_VENANT_KIRCHHOFF, LAM, MU,
                                       None if le_d is None else le_d.data_ptr(),
                                       None if me_d is None else me_d.data_ptr(), ud.data_ptr(), f2.data_ptr(), None)
        torch.cuda.synchronize()
        assert rc == osam.OK
        assert np.abs(f2.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


def _pair(spec, n_ctrl, tol, **kw):
    gpu = osam.Problem(spec, **kw)
    ref = O.Problem(spec)
    hg = {i: [] for i in range(len(spec.subdomains))}
    hr = {i: [] for i in range(len(spec.subdomains))}
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] in (osam.OK, osam.MAXITER) and rr["status"] in (O.OK, O.MAXITER)
        for i in range(len(spec.subdomains)):
            hg[i].append(gpu.state(i)[0].copy())
            hr[i].append(ref.state(i)[0].copy())
    gpu.close()
    for i in hg:
        assert rel_l2(hg[i], hr[i]) < tol, (i, rel_l2(hg[i], hr[i]))


@pytest.mark.parametrize("scatter", [osam.SCATTER_GATHER, osam.SCATTER_ATOMIC, osam.SCATTER_GATHER_TILED,
                                     osam.SCATTER_GATHER_LOWREG])
def test_svk_fom_fom_explicit(gpu, scatter):
    spec = W.bar_chain("svk", 4, [9, 7], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 3e-3, 1e-6, 6, max_iters=40)
    _pair(spec, 3, 1e-9, scatter=scatter)


@pytest.mark.parametrize("precision,tol", [(osam.F32X2_FORCE, 1e-9), (osam.FP32_FORCE, 1e-5)])
def test_svk_precision_variants(gpu, precision, tol):
    spec = W.bar_chain("svkp", 4, [9, 7], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 3e-3, 1e-6, 6, max_iters=6)
    _pair(spec, 3, tol, precision=precision)


def test_svk_implicit_and_mixed_steps(gpu):
    """Implicit Saint Venant-Kirchhoff subdomain (Newton on the A.2 tangent) coupled to an explicit one
    with twice as many substeps."""
    spec = W.bar_chain("svki", 3, [8, 8], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 3e-3, 1e-6, 6, max_iters=40)
    spec.subdomains[1].integrator = "implicit"
    spec.subdomains[1].n_substeps = 3
    _pair(spec, 3, 1e-9)


def test_svk_adjoint_is_rejected(gpu):
    p, w = W.adjoint_bar(n=3, nz=4, n_steps=2)
    sd = p.subdomains[0]
    with pytest.raises(osam.OsamError) as e:
        osam.adjoint(sd.dims, sd.h, "svk", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, sd.u0, None, p.dt, 2, w)
    assert e.value.code == osam.EINVAL
