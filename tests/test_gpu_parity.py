"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded inputs.

Tolerances: FP64 paths 1e-9 relative L2 displacement error (the paper's error measure, Eq. mse,
over the saved controller steps); single force / VJP evaluations are compared element by element
at 1e-12 of the field's scale; the FP32-force variant at 1e-5.
"""
import numpy as np
import pytest

from oracle import fit as OF
from oracle import oracle as O
from paper_2511_20687_gb300 import osam
from paper_2511_20687_gb300 import workloads as W

from .helpers import oracle_rom_ops, rel_l2

pytestmark = pytest.mark.gpu

LAM, MU = W.lame(1e9, 0.25)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20687_gb300 import build_lib
    build_lib.build()
    osam.load()
    return torch


def _run_pair(spec, n_ctrl, rom_ops=None, **kw):
    gpu = osam.Problem(spec, rom_ops=rom_ops, **kw)
    ref = O.Problem(spec, rom_ops=rom_ops)
    hist = {i: ([], []) for i in range(len(spec.subdomains))}
    its = []
    for _ in range(n_ctrl):
        rg, rr = gpu.step(), ref.step()
        its.append((rg["iterations"], rr["iterations"]))
        assert rg["status"] in (osam.OK, osam.MAXITER) and rr["status"] in (O.OK, O.MAXITER)
        for i in range(len(spec.subdomains)):
            hist[i][0].append(gpu.state(i)[0].copy())
            hist[i][1].append(ref.state(i)[0].copy())
    gpu_final = [gpu.state(i) for i in range(len(spec.subdomains))]
    ref_final = [ref.state(i) for i in range(len(spec.subdomains))]
    gpu.close()
    return hist, its, gpu_final, ref_final


# ---------------------------------------------------------------------------------------------
# element level
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("material", ["le", "nh"])
@pytest.mark.parametrize("per_element", [False, True])
def test_hex8_force_matches_oracle(torch_cuda, material, per_element):
    torch = torch_cuda
    dims, h = (13, 9, 11), 0.01          # 1287 elements: several blocks and a ragged tail
    nn = 14 * 10 * 12
    rng = np.random.default_rng(10)
    u = 1e-4 * rng.standard_normal((nn, 3))
    le = LAM * (1 + 0.1 * rng.uniform(-1, 1, 13 * 9 * 11)) if per_element else None
    me = MU * (1 + 0.1 * rng.uniform(-1, 1, 13 * 9 * 11)) if per_element else None
    f_ref = O.internal_force(dims, h, (0.0, 0.0, 0.0), material, LAM, MU, u, lam_e=le, mu_e=me).reshape(nn, 3)
    ud = torch.tensor(u, device="cuda")
    fd = torch.empty_like(ud)
    osam.hex8_force(dims, h, material, LAM, MU, ud, fd,
                    lam_e=None if le is None else torch.tensor(le, device="cuda"),
                    mu_e=None if me is None else torch.tensor(me, device="cuda"))
    torch.cuda.synchronize()
    f = fd.cpu().numpy()
    assert np.abs(f - f_ref).max() < 1e-12 * np.abs(f_ref).max()


@pytest.mark.parametrize("material", ["le", "nh"])
def test_hex8_vjp_matches_oracle(torch_cuda, material):
    torch = torch_cuda
    dims, h = (7, 5, 9), 0.02
    nn, ne = 8 * 6 * 10, 7 * 5 * 9
    rng = np.random.default_rng(11)
    u = 2e-4 * rng.standard_normal((nn, 3))
    y = rng.standard_normal((nn, 3))
    le = LAM * (1 + 0.1 * rng.uniform(-1, 1, ne))
    me = MU * (1 + 0.1 * rng.uniform(-1, 1, ne))
    ub_r, lb_r, mb_r = O.force_vjp(dims, h, (0, 0, 0), material, le, me, u, y)
    t = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    ub, lb, mb = torch.empty((nn, 3), dtype=torch.float64, device="cuda"), t(np.zeros(ne)), t(np.zeros(ne))
    osam.hex8_force_vjp(dims, h, material, 0.0, 0.0, t(u), t(y), ub, lb, mb, lam_e=t(le), mu_e=t(me))
    torch.cuda.synchronize()
    assert np.abs(ub.cpu().numpy().reshape(-1) - ub_r).max() < 1e-12 * np.abs(ub_r).max()
    assert np.abs(lb.cpu().numpy() - lb_r).max() < 1e-10 * np.abs(lb_r).max()
    assert np.abs(mb.cpu().numpy() - mb_r).max() < 1e-10 * np.abs(mb_r).max()


def test_hex8_force_degenerate_single_element(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(12)
    u = 1e-3 * rng.standard_normal((8, 3))
    f_ref = O.internal_force((1, 1, 1), 0.05, (0, 0, 0), "nh", LAM, MU, u).reshape(8, 3)
    ud = torch.tensor(u, device="cuda")
    fd = torch.empty_like(ud)
    osam.hex8_force((1, 1, 1), 0.05, "nh", LAM, MU, ud, fd)
    torch.cuda.synchronize()
    assert np.abs(fd.cpu().numpy() - f_ref).max() < 1e-12 * np.abs(f_ref).max()


def test_autograd_function_matches_oracle_vjp(torch_cuda):
    torch = torch_cuda
    from paper_2511_20687_gb300.autograd import hex8_force
    dims, h = (4, 3, 5), 0.01
    nn, ne = 5 * 4 * 6, 4 * 3 * 5
    rng = np.random.default_rng(13)
    u = 1e-4 * rng.standard_normal((nn, 3))
    y = rng.standard_normal((nn, 3))
    le = LAM * (1 + 0.1 * rng.uniform(-1, 1, ne))
    me = MU * (1 + 0.1 * rng.uniform(-1, 1, ne))
    ut = torch.tensor(u, device="cuda", requires_grad=True)
    lt = torch.tensor(le, device="cuda", requires_grad=True)
    mt = torch.tensor(me, device="cuda", requires_grad=True)
    f = hex8_force(ut, lt, mt, dims, h, "nh")
    (f * torch.tensor(y, device="cuda")).sum().backward()
    ub_r, lb_r, mb_r = O.force_vjp(dims, h, (0, 0, 0), "nh", le, me, u, y)
    assert np.abs(ut.grad.cpu().numpy().reshape(-1) - ub_r).max() < 1e-12 * np.abs(ub_r).max()
    assert np.abs(lt.grad.cpu().numpy() - lb_r).max() < 1e-10 * np.abs(lb_r).max()
    assert np.abs(mt.grad.cpu().numpy() - mb_r).max() < 1e-10 * np.abs(mb_r).max()


# ---------------------------------------------------------------------------------------------
# coupled problems
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("scatter", [osam.SCATTER_GATHER, osam.SCATTER_ATOMIC, osam.SCATTER_GATHER_LOWREG,
                                     osam.SCATTER_GATHER_TILED])
def test_fom_fom_plain_config_matches_oracle(torch_cuda, scatter):
    """Two 6x6x12 linear-elastic FOMs, 10 controller steps of 20 (the whole 200-step run)."""
    spec = W.fom_fom_plain()
    hist, its, gf, rf = _run_pair(spec, spec.n_controller_steps, scatter=scatter)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9
        for f in range(3):
            assert np.abs(gf[i][f] - rf[i][f]).max() <= 1e-9 * np.abs(rf[i][f]).max()
    assert all(abs(a - b) <= 1 for a, b in its)


@pytest.mark.parametrize("scatter", [osam.SCATTER_AUTO, osam.SCATTER_GATHER_LOWREG, osam.SCATTER_GATHER_TILED])
def test_neo_hookean_fom_fom_odd_substeps(torch_cuda, scatter):
    """Neo-Hookean, unequal subdomain lengths, odd substep count (state ping-pong ends on buffer 1)."""
    spec = W.bar_chain("nh_odd", 5, [9, 7], ["fom", "fom"], "nh", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 7)
    hist, its, _, _ = _run_pair(spec, 4, scatter=scatter)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9


def test_single_subdomain_no_coupling(torch_cuda):
    spec = W.single_bar("single", 4, 10, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10)
    hist, its, _, _ = _run_pair(spec, 3)
    assert rel_l2(*hist[0]) < 1e-9
    assert all(a == 1 for a, _ in its)


def test_three_subdomain_chain_fom(torch_cuda):
    spec = W.bar_chain("chain3", 3, [6, 6, 6], ["fom", "fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 8)
    hist, its, _, _ = _run_pair(spec, 3)
    for i in range(3):
        assert rel_l2(*hist[i]) < 1e-9


def _exact_rom_ops(spec_ff, i):
    prob = O.Problem(spec_ff)
    free, sdof = prob.free_dofs(i), prob.schwarz_dofs(i)
    sd = spec_ff.subdomains[i]
    m = O.lumped_mass(sd.dims, sd.h, sd.origin, sd.rho)
    n3 = 3 * sd.n_nodes

    def col(d):
        e = np.zeros(n3)
        e[d] = 1.0
        return -O.internal_force(sd.dims, sd.h, sd.origin, "le", sd.lam, sd.mu, e)[free] / m[free // 3]

    K = np.stack([col(d) for d in free], axis=1)
    B = np.stack([col(d) for d in sdof], axis=1)
    r = len(free)
    return {"Phi": np.eye(r), "Phi_S": np.eye(len(sdof)), "K": K, "H": np.zeros((r, r * (r + 1) // 2)), "B": B,
            "c": np.zeros(r)}


def test_full_basis_rom_hybrid(torch_cuda):
    """Exact full-basis linear ROM: GPU FOM-ROM equals the oracle FOM-ROM and the GPU FOM-FOM."""
    pf = W.bar_chain("ff", 2, [4, 4], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    pr = W.bar_chain("fr", 2, [4, 4], ["fom", "rom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    ops = {1: _exact_rom_ops(pf, 1)}
    hist, its, gf, rf = _run_pair(pr, 4, rom_ops=ops)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9
    ff = osam.Problem(pf)
    for _ in range(4):
        ff.step()
    for i in range(2):
        assert np.abs(ff.state(i)[0] - gf[i][0]).max() < 1e-11 * np.abs(gf[i][0]).max()


@pytest.mark.parametrize("n_sub", [1, 2, 3])
@pytest.mark.parametrize("kinds", [["fom", "fom"], ["fom", "rom"], ["fom", "rom", "fom"]])
def test_short_controller_intervals(torch_cuda, n_sub, kinds):
    """1-3 substeps per controller step: the trace of the last substep has no force launch to ride in,
    and with one substep none is folded at all; the ROM side stream then runs only after it."""
    spec = W.bar_chain("short", 3, [6] * len(kinds), kinds, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, n_sub,
                       max_iters=8)
    ops = None
    if "rom" in kinds:
        sd = spec.subdomains[1]
        faces = 2 if len(kinds) == 3 else 1
        n_sdof = faces * 3 * (sd.dims[0] + 1) ** 2
        ops = {1: W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof, n_sdof, 5, 4, 21)}
    hist, its, _, _ = _run_pair(spec, 5, rom_ops=ops)
    for i in range(len(spec.subdomains)):
        assert rel_l2(*hist[i]) < 1e-9, i
    assert all(abs(a - b) <= 1 for a, b in its)


@pytest.fixture(scope="module")
def fitted_hybrid():
    """Small NH FOM-ROM hybrid with operators fitted by the oracle on a FOM-FOM training run."""
    pf = W.bar_chain("train", 3, [6, 6], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 4,
                     n_controller_steps=60)
    ops, _ = oracle_rom_ops(pf, 1, 60, r=6, lam=1e-6, r_s=4)
    pr = W.bar_chain("hyb", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 4)
    rom = {k: ops[k] for k in ("Phi", "Phi_S", "K", "H", "B", "c")}
    return pr, {1: rom}


def test_fitted_rom_hybrid_matches_oracle(torch_cuda, fitted_hybrid):
    pr, ops = fitted_hybrid
    pr.max_iters = 16
    hist, its, gf, rf = _run_pair(pr, 5, rom_ops=ops)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9
    assert all(abs(a - b) <= 1 for a, b in its)


@pytest.mark.parametrize("r,r_s", [(1, 1), (128, 64), (256, 64)])
def test_rom_rank_extremes_match_oracle(torch_cuda, r, r_s):
    """FOM-ROM with the smallest ROM rank, the large chain's r = 128 and the largest rank the ROM
    kernels take (256; H has 32,896 columns), seeded stand-in operators on a 6x6x8 + 6x6x8 bar."""
    from .test_gpu_additive import _rom_ops
    spec = W.bar_chain("rk", 6, [8, 8], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10, max_iters=8)
    ops = {1: _rom_ops(spec, 1, r, r_s, 11)}
    gpu = osam.Problem(spec, rom_ops=ops)
    ref = O.Problem(spec, rom_ops=ops)
    hu, hq = ([], []), ([], [])
    for _ in range(2):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] == osam.OK and rr["status"] == O.OK
        assert abs(rg["iterations"] - rr["iterations"]) <= 1
        hu[0].append(gpu.state(0)[0].copy()); hu[1].append(ref.state(0)[0].copy())
        hq[0].append(gpu.reduced_state(1)[0].copy()); hq[1].append(ref.rom_state(1)[0].copy())
    gpu.close()
    assert rel_l2(*hu) < 1e-9
    assert rel_l2(*hq) < 1e-9


def test_five_subdomain_chain_with_two_roms(torch_cuda):
    """FOM-ROM-FOM-FOM-ROM: five subdomains, eight couplings, a ROM at the free end."""
    from .test_gpu_additive import _rom_ops
    spec = W.bar_chain("five", 3, [6, 6, 6, 6, 6], ["fom", "rom", "fom", "fom", "rom"], "nh", 1e9, 0.25, 1000.0,
                       1e-3, 1e-6, 6, max_iters=12)
    ops = {1: _rom_ops(spec, 1, 6, 4, 21), 4: _rom_ops(spec, 4, 5, 3, 22)}
    gpu = osam.Problem(spec, rom_ops=ops)
    ref = O.Problem(spec, rom_ops=ops)
    hist = {i: ([], []) for i in range(5)}
    for _ in range(2):
        rg, rr = gpu.step(), ref.step()
        assert rg["status"] == osam.OK and rr["status"] == O.OK
        assert abs(rg["iterations"] - rr["iterations"]) <= 1
        for i, sd in enumerate(spec.subdomains):
            if sd.kind == "fom":
                hist[i][0].append(gpu.state(i)[0].copy()); hist[i][1].append(ref.state(i)[0].copy())
            else:
                hist[i][0].append(gpu.reduced_state(i)[0].copy()); hist[i][1].append(ref.rom_state(i)[0].copy())
    gpu.close()
    for i in range(5):
        assert rel_l2(*hist[i]) < 1e-9, i


def test_rom_rank_above_the_kernel_limit_is_rejected(torch_cuda):
    from .test_gpu_additive import _rom_ops
    spec = W.bar_chain("rk", 6, [8, 8], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10, max_iters=8)
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec, rom_ops={1: _rom_ops(spec, 1, 257, 4, 11)})
    assert ei.value.code == osam.EINVAL


def test_three_subdomain_chain_fom_rom_fom(torch_cuda):
    pf = W.bar_chain("c", 2, [4, 4, 4], ["fom", "fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    pr = W.bar_chain("c", 2, [4, 4, 4], ["fom", "rom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    ops = {1: _exact_rom_ops(pf, 1)}
    hist, its, _, _ = _run_pair(pr, 3, rom_ops=ops)
    for i in range(3):
        assert rel_l2(*hist[i]) < 1e-9


def test_fp32_force_variant(torch_cuda):
    spec = W.bar_chain("fp32", 4, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10)
    for scatter in (osam.SCATTER_GATHER, osam.SCATTER_ATOMIC):
        hist, _, _, _ = _run_pair(spec, 4, precision=osam.FP32_FORCE, scatter=scatter)
        for i in range(2):
            assert rel_l2(*hist[i]) < 1e-5


def test_manual_abi_sequence_equals_schwarz_step(torch_cuda):
    """begin_interval / advance / transfer / criterion reproduce schwarz_step."""
    spec = W.fom_fom_plain()
    a = osam.Problem(spec, scatter=osam.SCATTER_GATHER)
    b = osam.Problem(spec, scatter=osam.SCATTER_GATHER)
    rep = a.step()
    b.begin_interval()
    for n in range(1, rep["iterations"] + 1):
        if n > 1:
            b.restore_interval()
        b.advance(0)
        b.transfer(0, 1)
        b.advance(1)
        b.transfer(1, 0)
        cnum, cden = b.criterion()
    assert cnum == rep["cnum"] and cden == rep["cden"]
    for i in range(2):
        assert np.array_equal(a.state(i)[0], b.state(i)[0])


def test_set_state_roundtrip(torch_cuda):
    spec = W.fom_fom_plain()
    g = osam.Problem(spec)
    u, v, a = g.state(0)
    rng = np.random.default_rng(3)
    u2 = u + 1e-6 * rng.standard_normal(u.shape)
    g.set_state(0, u2, v, a)
    u3, v3, a3 = g.state(0)
    clamped = np.repeat(spec.subdomains[0].dirichlet > 0, 3).reshape(-1, 3)
    assert np.array_equal(u3[~clamped], u2[~clamped]) and np.all(u3[clamped] == 0)


def test_state_calls_agree_for_pageable_pinned_and_device_buffers(torch_cuda):
    """Pageable host arrays go through the staging buffer; pinned host and device tensors are read and
    written in place by the layout kernels.  All three give the same states, for a FOM and for the
    reconstructed field of a ROM, and a state set from any of them steps identically."""
    torch = torch_cuda
    spec = W.bar_chain("views", 3, [6, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=6)
    sd = spec.subdomains[1]
    n_sdof = 3 * (sd.dims[0] + 1) ** 2
    ops = {1: W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof, n_sdof, 5, 4, 21)}
    g = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER)
    g.step()
    for i in range(2):
        n = g.sizes(i)["n_nodes"]
        ref = g.state(i)
        pinned = tuple(torch.full((n, 3), np.nan, dtype=torch.float64).pin_memory() for _ in range(3))
        device = tuple(torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda") for _ in range(3))
        g.state(i, out=pinned)
        g.state(i, out=device)
        for f in range(3):
            assert np.array_equal(pinned[f].numpy(), ref[f])
            assert np.array_equal(device[f].cpu().numpy(), ref[f])
    u, v, a = g.state(0)
    rng = np.random.default_rng(5)
    u2 = u + 1e-6 * rng.standard_normal(u.shape)
    runs = []
    for kind in ("pageable", "pinned", "device"):
        p = osam.Problem(spec, rom_ops=ops, scatter=osam.SCATTER_GATHER)
        p.step()
        if kind == "pageable":
            p.set_state(0, u2, v, a)
        else:
            ts = [torch.from_numpy(np.ascontiguousarray(x)) for x in (u2, v, a)]
            ts = [t.pin_memory() if kind == "pinned" else t.cuda() for t in ts]
            p.set_state(0, *ts)
        p.step()
        runs.append((p.state(0), p.reduced_state(1)))
    for (s, q) in runs[1:]:
        for f in range(3):
            assert np.array_equal(s[f], runs[0][0][f])
            assert np.array_equal(q[f], runs[0][1][f])


@pytest.mark.parametrize("graph", [True, False])
def test_single_iteration_cap_matches_oracle(torch_cuda, graph):
    """max_iters = 1: the criterion needs two iterates, so every controller step commits after one
    sweep with MAXITER, on both sides (graph-captured and host-driven)."""
    spec = W.fom_fom_plain()
    spec.max_iters = 1
    hist, its, _, _ = _run_pair(spec, 3, graph=graph)
    assert all(a == 1 and b == 1 for a, b in its)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9


def test_empty_mesh_is_rejected(torch_cuda):
    torch = torch_cuda
    u = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(u)
    for dims in ((0, 3, 3), (3, 0, 3), (3, 3, 0)):
        with pytest.raises(osam.OsamError) as ei:
            osam.hex8_force(dims, 0.01, "nh", LAM, MU, u, f)
        assert ei.value.code == osam.EINVAL
        with pytest.raises(osam.OsamError) as ei:
            osam.hex8_force_vjp(dims, 0.01, "nh", LAM, MU, u, u, f)
        assert ei.value.code == osam.EINVAL


def test_donor_failure_is_reported(torch_cuda):
    spec = W.fom_fom_plain()
    # move subdomain 1 away so its Schwarz nodes fall outside subdomain 0
    spec.subdomains[1].origin = (0.0, 0.0, 5.0)
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec)
    assert ei.value.code == osam.EDONOR


def test_invalid_description_is_rejected(torch_cuda):
    spec = W.fom_fom_plain()
    spec.dt = -1.0
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec)
    assert ei.value.code == osam.EINVAL


@pytest.mark.parametrize("per_element", [False, True])
def test_stability_check_agrees_with_oracle(torch_cuda, per_element):
    """Both sides reject a time step 1% above the explicit stability limit (ECFL) and accept one 1%
    below it; with per-element materials the stiffest element sets the limit."""
    spec = W.fom_fom_plain()
    sd = spec.subdomains[0]
    le = me = None
    if per_element:
        rng = np.random.default_rng(12)
        for k, s in enumerate(spec.subdomains):
            s.lam_e = LAM * (1.0 + 0.5 * rng.uniform(-1, 1, s.n_elements))
            s.mu_e = MU * (1.0 + 0.5 * rng.uniform(-1, 1, s.n_elements))
        le, me = sd.lam_e, sd.mu_e
    lim = min(O.stable_dt(s.dims, s.h, s.origin, s.lam, s.mu, s.rho, lam_e=s.lam_e, mu_e=s.mu_e)
              for s in spec.subdomains)
    assert lim > 0 and (le is None or lim < O.stable_dt(sd.dims, sd.h, sd.origin, LAM, MU, sd.rho))
    spec.dt = 1.01 * lim
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec)
    assert ei.value.code == osam.ECFL
    with pytest.raises(O.OracleError) as eo:
        O.Problem(spec)
    assert eo.value.code == O.ECFL
    spec.dt = 0.99 * lim
    osam.Problem(spec).close()
    O.Problem(spec)


def test_stability_check_accepts_the_bar_at_courant_one(torch_cuda):
    spec = W.wave1d(n_elem=40)
    osam.Problem(spec).close()
    O.Problem(spec)


def test_non_positive_definite_material_is_rejected(torch_cuda):
    spec = W.fom_fom_plain()
    spec.subdomains[1].lam = -0.7 * spec.subdomains[1].mu  # 3 lambda + 2 mu < 0
    with pytest.raises(osam.OsamError) as ei:
        osam.Problem(spec)
    assert ei.value.code == osam.EINVAL


@pytest.mark.parametrize("rom", [False, True])
def test_non_finite_state_is_reported(torch_cuda, rom):
    """A NaN in the coupled state ends the controller step with ENONFINITE on both sides."""
    if rom:
        spec = W.bar_chain("nf", 3, [6, 6], ["fom", "rom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=6)
        sd = spec.subdomains[1]
        n_sdof = 3 * (sd.dims[0] + 1) ** 2
        ops = {1: W.synthetic_rom_operators(3 * sd.n_nodes - n_sdof, n_sdof, 5, 4, 3)}
    else:
        spec, ops = W.fom_fom_plain(), None
    spec.subdomains[0].u0 = spec.subdomains[0].u0.copy()
    spec.subdomains[0].u0[spec.subdomains[0].n_nodes // 2, 2] = np.nan
    gpu = osam.Problem(spec, rom_ops=ops)
    with pytest.raises(osam.OsamError) as ei:
        gpu.step()
    assert ei.value.code == osam.ENONFINITE
    with pytest.raises(O.OracleError) as eo:
        O.Problem(spec, rom_ops=ops).step()
    assert eo.value.code == O.ENONFINITE
    gpu.close()


# ---------------------------------------------------------------------------------------------
# offline fit and adjoint
# ---------------------------------------------------------------------------------------------
def _fit_case(n, ns, nsd, seed):
    """Snapshots of a known quadratic model (r = 5, r_s = 3) in random orthonormal bases, with noise."""
    rng = np.random.default_rng(seed)
    r, rs = 5, 3
    Q = np.diag([6.0, 4.5, 3.0, 2.0, 1.0]) @ rng.standard_normal((r, ns))
    Phi_t, _ = np.linalg.qr(rng.standard_normal((n, r)))
    PhiS_t, _ = np.linalg.qr(rng.standard_normal((nsd, rs)))
    G = np.diag([3.0, 2.0, 1.0]) @ rng.standard_normal((rs, ns))
    K = rng.standard_normal((r, r))
    H = 0.1 * rng.standard_normal((r, r * (r + 1) // 2))
    B = rng.standard_normal((r, rs))
    c = rng.standard_normal(r)
    Qdd = K @ Q + H @ OF.kron_c(Q) + B @ G + c[:, None]
    U = (Phi_t @ Q).T + 1e-3 * rng.standard_normal((ns, n))
    A = (Phi_t @ Qdd).T
    S = (PhiS_t @ G).T + 1e-3 * rng.standard_normal((ns, nsd))
    return U, A, S, r, rs, rng


def _check_fit(U, A, S, r, rs, rng):
    ref = OF.opinf_fit(U.T, A.T, S.T, r=r, lam=1e-6, r_s=rs)
    got = osam.opinf_fit(U, A, S, r=r, lam=1e-6, r_s=rs)
    assert got["r_s"] == rs
    assert np.abs(got["sigma"][:r] - ref["sigma"][:r]).max() < 1e-10 * ref["sigma"][0]
    sg = np.sign(np.sum(got["Phi"] * ref["Phi"], axis=0))
    ss = np.sign(np.sum(got["Phi_S"] * ref["Phi_S"], axis=0))
    assert np.abs(got["Phi"] * sg - ref["Phi"]).max() < 1e-9
    assert np.abs(got["Phi_S"] * ss - ref["Phi_S"]).max() < 1e-9
    # operators in the sign-aligned basis
    Kg = sg[:, None] * got["K"] * sg[None, :]
    assert np.abs(Kg - ref["K"]).max() < 1e-7 * np.abs(ref["K"]).max()
    qs = rng.standard_normal((r, 8))
    gs = rng.standard_normal((rs, 8))
    for k in range(8):
        want = ref["Phi"] @ OF.rom_rhs(ref["K"], ref["H"], ref["B"], ref["c"], qs[:, k], gs[:, k])
        qg, gg = sg * qs[:, k], ss * gs[:, k]
        have = got["Phi"] @ OF.rom_rhs(got["K"], got["H"], got["B"], got["c"], qg, gg)
        assert np.linalg.norm(have - want) < 1e-7 * np.linalg.norm(want)


def test_opinf_fit_matches_oracle_fit(torch_cuda):
    """Same snapshots: bases agree up to column signs, singular values and fitted operators (after
    aligning signs) agree; full-space predicted accelerations agree."""
    _check_fit(*_fit_case(900, 60, 45, 21))


def test_opinf_fit_long_reductions_match_oracle_fit(torch_cuda):
    """40,000 dofs and 3,000 Schwarz dofs against 60 snapshots: the Gram, Phi^T Phi, the projections
    and the boundary projection reduce over thousands of entries into outputs of one tile or less, so
    the GEMM splits the reduction (76 chunks of 528 and a ragged last chunk of 400 for the dof sums)
    and sums the partials in a second kernel; the transposed-operand loaders serve Phi = U^T W."""
    _check_fit(*_fit_case(40000, 60, 3000, 22))


def test_adjoint_matches_oracle_and_fd(torch_cuda):
    p, w = W.adjoint_bar(n=3, nz=6, n_steps=120)
    sd = p.subdomains[0]
    u0 = 3.0 * sd.u0
    args = (sd.dims, sd.h, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, u0, None, p.dt, 120, w)
    got = osam.adjoint(*args, checkpoint_every=50)
    J, gu, gv, gl, gm = O.adjoint(sd.dims, sd.h, sd.origin, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, u0, None,
                                  p.dt, 120, w)
    assert abs(got["J"] - J) < 1e-12 * abs(J)
    for a, b in ((got["grad_u0"].reshape(-1), gu), (got["grad_v0"].reshape(-1), gv), (got["grad_lambda"], gl),
                 (got["grad_mu"], gm)):
        assert np.abs(a - b).max() < 1e-9 * np.abs(b).max()
    # central differences of the GPU rollout's J along a random lambda direction
    rng = np.random.default_rng(5)
    dl = rng.standard_normal(sd.n_elements)
    hl = 1e-6 * sd.lam

    def J_of(le):
        return osam.adjoint(sd.dims, sd.h, "nh", le, sd.mu_e, sd.rho, sd.dirichlet, u0, None, p.dt, 120, w)["J"]

    fd = (J_of(sd.lam_e + hl * dl) - J_of(sd.lam_e - hl * dl)) / (2 * hl)
    assert abs(fd - got["grad_lambda"] @ dl) < 1e-6 * abs(fd)


def test_adjoint_with_no_steps_is_the_identity(torch_cuda):
    """T = 0: J = w . u0 over the free dofs, dJ/du0 = w there and zero at clamped dofs, every other
    gradient zero -- GPU and oracle alike."""
    p, w = W.adjoint_bar(n=3, nz=4, n_steps=0)
    sd = p.subdomains[0]
    got = osam.adjoint(sd.dims, sd.h, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, sd.u0, None, p.dt, 0, w)
    J, gu, gv, gl, gm = O.adjoint(sd.dims, sd.h, sd.origin, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, sd.u0,
                                  None, p.dt, 0, w)
    wm = np.array(w, dtype=np.float64).reshape(-1, 3)
    wm[sd.dirichlet.astype(bool)] = 0.0
    assert abs(got["J"] - J) <= 1e-14 * abs(J)
    assert np.abs(got["grad_u0"].reshape(-1) - wm.reshape(-1)).max() <= 1e-15 * np.abs(wm).max()
    assert np.abs(gu - wm.reshape(-1)).max() == 0.0
    for a in (got["grad_v0"], got["grad_lambda"], got["grad_mu"], gv, gl, gm):
        assert np.abs(a).max() == 0.0


def test_profile_counters(torch_cuda):
    spec = W.fom_fom_plain()
    g = osam.Problem(spec)
    g.profile(True)
    r = g.step()
    p = g.profile_read()
    assert p["force_launches"] == r["iterations"] * spec.n_substeps * 2
    assert p["force_elements"] == r["element_updates"]
    assert p["force_ms"] > 0.0 and p["kernel_launches"] > p["force_launches"]
    assert osam.fp64_peak_gflops(0) > 0.0


def test_fp64_probes_are_consistent(torch_cuda):
    """The throughput probe gives rates within a factor of the nominal 1.25 TFLOP/s; the issue probe's
    per-warp interval is no shorter with eight warps on the SM than with one (the SM's FP64 share is
    fixed), and it rejects block shapes outside 1..32 warps of 1..32 lanes."""
    t, ms = osam.fp64_probe(0, 2, 0)
    assert np.all(t > 0.1) and np.all(t < 5.0) and np.all(ms > 0.0)
    one = osam.fp64_issue_probe(1, 32, 0)
    eight = osam.fp64_issue_probe(8, 32, 0)
    assert one > 0.0 and eight >= 0.9 * one
    with pytest.raises(osam.OsamError):
        osam.fp64_issue_probe(0, 32, 0)
    with pytest.raises(osam.OsamError):
        osam.fp64_issue_probe(1, 33, 0)


# ---------------------------------------------------------------------------------------------
# double-float force (f32x2): held to the FP64 tolerance
# ---------------------------------------------------------------------------------------------
def test_f32x2_force_fom_fom_plain_config(torch_cuda):
    spec = W.fom_fom_plain()
    hist, its, gf, rf = _run_pair(spec, spec.n_controller_steps, precision=osam.F32X2_FORCE)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9


def test_f32x2_force_neo_hookean_and_hybrid(torch_cuda, fitted_hybrid):
    spec = W.bar_chain("nh_df", 5, [9, 7], ["fom", "fom"], "nh", 1e9, 0.3, 1000.0, 2e-3, 1e-6, 7)
    hist, _, _, _ = _run_pair(spec, 4, precision=osam.F32X2_FORCE)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9
    pr, ops = fitted_hybrid
    pr.max_iters = 16
    hist, _, _, _ = _run_pair(pr, 5, rom_ops=ops, precision=osam.F32X2_FORCE)
    for i in range(2):
        assert rel_l2(*hist[i]) < 1e-9
