"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: a closed form printed in the
paper, an energy whose derivative the stress must be, an invariant of the discretisation or of
the time integrator, or a special case that reduces to a known answer.  A plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

from paper_2511_20687_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LAM, MU = W.lame(1e9, 0.25)


def _rand_disp(dims, scale, seed):
    nx, ny, nz = dims
    return scale * np.random.default_rng(seed).standard_normal(((nx + 1) * (ny + 1) * (nz + 1), 3))


def _coords(dims, h, origin):
    sd = W.Subdomain(kind="fom", dims=dims, h=h, origin=origin)
    return sd.node_coords(), sd.node_grid()


# ---------------------------------------------------------------------------------------------
# constitutive laws (Appendix A)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("material", ["le", "nh", "svk"])
def test_stress_is_derivative_of_energy_density(oracle, material):
    """P = dA/dF for the energies printed in Appendix A (A.1: 1/2 lam tr(eps)^2 + mu tr(eps^2);
    A.2: lam/2 (tr E)^2 + mu tr(E^2); A.3: 1/4 kappa (detC - log detC - 1) + 1/2 mu (detC^-1/3 trC -
    3)).  This pins the deviatoric coefficient 1/3 of S (the printed 1/2 would fail by O(mu)) and
    P = F S with S = lam tr(E) I + 2 mu E for Saint Venant-Kirchhoff."""
    rng = np.random.default_rng(1)
    for trial in range(5):
        H = 0.05 * rng.standard_normal((3, 3))
        P = oracle.stress(material, H, LAM, MU)
        fd = np.zeros((3, 3))
        eps = 1e-6
        for i in range(3):
            for j in range(3):
                Hp, Hm = H.copy(), H.copy()
                Hp[i, j] += eps
                Hm[i, j] -= eps
                fd[i, j] = (oracle.energy_density(material, Hp, LAM, MU)
                            - oracle.energy_density(material, Hm, LAM, MU)) / (2 * eps)
        assert np.abs(P - fd).max() < 1e-6 * np.abs(P).max()


def test_printed_half_coefficient_would_fail(oracle):
    """The stress the oracle uses differs from the variant with the printed 1/2 coefficient, and the
    energy derivative sides with the 1/3 one (reading c7)."""
    H = np.diag([0.02, -0.01, 0.015]) + 0.01
    F = np.eye(3) + H
    C = F.T @ F
    Ci = np.linalg.inv(C)
    kappa = LAM + 2 * MU / 3
    g = np.linalg.det(C) ** (-1 / 3)
    S_half = 0.5 * kappa * (np.linalg.det(C) - 1) * Ci + MU * g * (np.eye(3) - 0.5 * np.trace(C) * Ci)
    P = oracle.stress("nh", H, LAM, MU)
    assert np.abs(P - F @ S_half).max() > 1e-3 * np.abs(P).max()


@pytest.mark.parametrize("material", ["le", "nh", "svk"])
def test_internal_force_is_gradient_of_discrete_energy(oracle, material):
    """f_int = d/du of sum_e sum_gp w detJ A(F): checks quadrature, shape gradients and assembly
    against the energy of Appendix A (central differences)."""
    dims, h, org = (2, 2, 3), 0.01, (0.1, -0.2, 0.3)
    u = _rand_disp(dims, 1e-3, 2)
    f = oracle.internal_force(dims, h, org, material, LAM, MU, u)
    eps = 1e-8
    flat = u.reshape(-1)
    fd = np.zeros_like(flat)
    for d in range(flat.size):
        up, um = flat.copy(), flat.copy()
        up[d] += eps
        um[d] -= eps
        fd[d] = (oracle.strain_energy(dims, h, org, material, LAM, MU, up)
                 - oracle.strain_energy(dims, h, org, material, LAM, MU, um)) / (2 * eps)
    assert np.abs(f - fd).max() < 1e-6 * np.abs(f).max()


@pytest.mark.parametrize("material", ["le", "nh", "svk"])
def test_patch_test_affine_field_has_zero_interior_force(oracle, material):
    """A uniform deformation gradient gives a uniform stress, so the assembled force vanishes at
    every interior node."""
    dims, h, org = (3, 3, 4), 0.01, (0.0, 0.0, 0.0)
    X, (i, j, k) = _coords(dims, h, org)
    G = np.array([[0.01, 0.002, -0.003], [0.001, -0.004, 0.002], [0.003, 0.001, 0.006]])
    u = X @ G.T + np.array([1e-3, -2e-3, 5e-4])
    f = oracle.internal_force(dims, h, org, material, LAM, MU, u).reshape(-1, 3)
    interior = (i > 0) & (i < 3) & (j > 0) & (j < 3) & (k > 0) & (k < 4)
    scale = np.abs(f).max()
    assert scale > 0
    assert np.abs(f[interior]).max() < 1e-10 * scale


def test_rigid_motion_gives_zero_force(oracle):
    """Neo-Hookean is objective: a finite rotation plus translation gives zero force everywhere;
    the linear elastic law gives zero force for a translation."""
    dims, h, org = (2, 3, 2), 0.01, (0.05, 0.0, -0.02)
    X, _ = _coords(dims, h, org)
    th = 0.3
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    ax = np.array([1.0, 2.0, 2.0]) / 3.0
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = R @ (np.eye(3) + np.sin(0.4) * K + (1 - np.cos(0.4)) * K @ K)
    u = X @ (R - np.eye(3)).T + np.array([0.1, -0.3, 0.2])
    f = oracle.internal_force(dims, h, org, "nh", LAM, MU, u)
    # stress scale of a 1% strain for comparison
    u_ref = X @ (0.01 * np.eye(3)).T
    f_ref = oracle.internal_force(dims, h, org, "nh", LAM, MU, u_ref)
    assert np.abs(f).max() < 1e-8 * np.abs(f_ref).max()
    ft = oracle.internal_force(dims, h, org, "le", LAM, MU, np.tile([1e-3, 2e-3, -3e-3], (X.shape[0], 1)))
    assert np.abs(ft).max() < 1e-9 * np.abs(f_ref).max()


def test_neo_hookean_linearises_to_linear_elastic(oracle):
    """At small amplitude eps the NH force approaches the LE force with the same Lame pair
    (kappa = lambda + 2/3 mu), with a relative gap of order eps."""
    dims, h, org = (2, 2, 2), 0.01, (0.0, 0.0, 0.0)
    base = _rand_disp(dims, 1.0, 3)
    gaps = []
    for eps in (1e-4, 1e-5):
        u = eps * h * base
        f_nh = oracle.internal_force(dims, h, org, "nh", LAM, MU, u)
        f_le = oracle.internal_force(dims, h, org, "le", LAM, MU, u)
        gaps.append(np.abs(f_nh - f_le).max() / np.abs(f_le).max())
    assert gaps[0] < 1e-2
    assert 5.0 < gaps[0] / gaps[1] < 20.0  # first order in eps


def test_tangent_stiffness_is_symmetric(oracle):
    """The FD Jacobian of f_int at a deformed NH state is symmetric (hyperelastic potential)."""
    dims, h, org = (1, 2, 2), 0.01, (0.0, 0.0, 0.0)
    u0 = _rand_disp(dims, 2e-4, 4).reshape(-1)
    n = u0.size
    Kt = np.zeros((n, n))
    eps = 1e-9
    for d in range(n):
        up, um = u0.copy(), u0.copy()
        up[d] += eps
        um[d] -= eps
        Kt[:, d] = (oracle.internal_force(dims, h, org, "nh", LAM, MU, up)
                    - oracle.internal_force(dims, h, org, "nh", LAM, MU, um)) / (2 * eps)
    assert np.abs(Kt - Kt.T).max() < 1e-5 * np.abs(Kt).max()


def test_lumped_mass_totals_and_split(oracle):
    dims, h, org = (3, 2, 4), 0.02, (0.0, 0.0, 0.0)
    m = oracle.lumped_mass(dims, h, org, 1000.0)
    assert abs(m.sum() - 1000.0 * 3 * 2 * 4 * h ** 3) < 1e-12 * m.sum()
    # a corner node belongs to one element: rho V / 8
    assert abs(m[0] - 1000.0 * h ** 3 / 8) < 1e-15


# ---------------------------------------------------------------------------------------------
# spatial projector Pi
# ---------------------------------------------------------------------------------------------
def test_projector_reproduces_trilinear_fields_and_injects_at_nodes(oracle):
    dims, h, org = (3, 3, 5), 0.01, (0.0, 0.0, 0.0)
    X, _ = _coords(dims, h, org)
    rng = np.random.default_rng(5)
    coef = rng.standard_normal(8)

    def tri(p):
        x, y, z = p[..., 0], p[..., 1], p[..., 2]
        return (coef[0] + coef[1] * x + coef[2] * y + coef[3] * z + coef[4] * x * y + coef[5] * y * z
                + coef[6] * x * z + coef[7] * x * y * z)

    vals = tri(X)
    for _ in range(20):
        p = rng.uniform([0, 0, 0], [0.03, 0.03, 0.05])
        nodes, w = oracle.donor(dims, h, org, p)
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(w @ vals[nodes] - tri(p)) < 1e-12
    nodes, w = oracle.donor(dims, h, org, X[37])
    assert np.count_nonzero(w) == 1 and nodes[np.argmax(w)] == 37 and w.max() == 1.0
    with pytest.raises(ValueError):
        oracle.donor(dims, h, org, np.array([0.5, 0.0, 0.0]))


# ---------------------------------------------------------------------------------------------
# explicit central difference + Schwarz controller
# ---------------------------------------------------------------------------------------------
def _wave_fixture():
    with open(os.path.join(HERE, "golden", "wave1d_symmetric_gaussian.json")) as fh:
        return json.load(fh)


def _dalembert(g, z, t):
    a, b, s = g["initial_condition"]["a"], g["initial_condition"]["b"], g["initial_condition"]["s"]
    c = (g["E"] / g["rho"]) ** 0.5
    T = g["T"]
    f = lambda x: a * np.exp(-((x - b) ** 2) / (2 * s * s))  # noqa: E731
    return 0.5 * f(z - c * t) + 0.5 * f(z + c * t) - 0.5 * f(z - c * (T - t)) - 0.5 * f(z + c * (T - t))


def test_wave1d_matches_dalembert_at_courant_one(oracle):
    """Sec. 5.1 bar with dt = dz/c: the lumped-mass central-difference scheme is exact at the nodes,
    so the discrete solution equals Eq. disp_exact to rounding."""
    g = _wave_fixture()
    p = W.wave1d()
    sd = p.subdomains[0]
    assert p.dt == pytest.approx(g["dt_cfl"]) and sd.h == pytest.approx(g["dx"])
    assert sd.origin[2] == g["domain"]["z"][0] and sd.origin[0] == g["domain"]["x"][0]
    prob = oracle.Problem(p)
    z = sd.node_coords()[:, 2]
    t = 0.0
    for _ in range(4):
        for _ in range(10):
            prob.step()
            t += p.dt * p.n_substeps
        u, _, _ = prob.state(0)
        ex = _dalembert(g, z, t)
        assert np.abs(u[:, 2] - ex).max() < 1e-11 * g["initial_condition"]["a"]
        assert np.abs(u[:, :2]).max() == 0.0


def test_wave1d_schwarz_fom_fom_matches_dalembert(oracle):
    """FOM-FOM O-SAM on the paper's decomposition Omega_1 = (-0.5, 0.25), Omega_2 = (-0.25, 0.5)
    reproduces the exact solution on both subdomains."""
    g = _wave_fixture()
    p = W.wave1d(subdomains=True, n_substeps=20)
    assert p.subdomains[0].origin[2] + p.subdomains[0].dims[2] * p.subdomains[0].h == pytest.approx(
        g["subdomains"]["Omega_1"][1])
    assert p.subdomains[1].origin[2] == pytest.approx(g["subdomains"]["Omega_2"][0])
    prob = oracle.Problem(p)
    t = 0.0
    for _ in range(12):  # the pulse crosses the overlap boundaries
        r = prob.step()
        assert r["status"] == oracle.OK
        t += p.dt * p.n_substeps
    for i in range(2):
        u, _, _ = prob.state(i)
        z = p.subdomains[i].node_coords()[:, 2]
        assert np.abs(u[:, 2] - _dalembert(g, z, t)).max() < 1e-11 * g["initial_condition"]["a"]


def test_leapfrog_modified_energy_is_conserved(oracle):
    """Velocity-Verlet on M u'' = -K u conserves 1/2 v.Mv + 1/2 u.Ku - dt^2/8 a.Ma exactly; the
    plain total energy only oscillates at O(dt^2)."""
    p = W.single_bar("energy", 3, 8, "le", 1e9, 0.25, 1000.0, 1e-3, 2e-6, 5)
    sd = p.subdomains[0]
    prob = oracle.Problem(p)
    m = oracle.lumped_mass(sd.dims, sd.h, sd.origin, sd.rho)
    free = np.repeat(sd.dirichlet == 0, 3).reshape(-1, 3)

    def energies():
        u, v, a = prob.state(0)
        f = oracle.internal_force(sd.dims, sd.h, sd.origin, "le", sd.lam, sd.mu, u).reshape(-1, 3)
        kin = 0.5 * np.sum((m[:, None] * v * v)[free])
        pot = 0.5 * np.sum((u * f)[free])
        corr = p.dt ** 2 / 8 * np.sum((m[:, None] * a * a)[free])
        return kin + pot - corr, kin + pot

    e0, t0 = energies()
    mods, tots = [], []
    for _ in range(40):
        prob.step()
        e, t = energies()
        mods.append(e)
        tots.append(t)
    assert np.abs(np.array(mods) - e0).max() < 1e-10 * e0
    assert np.abs(np.array(tots) - t0).max() < 0.05 * t0


def test_fom_fom_schwarz_equals_single_domain(oracle):
    """Two conforming 6x6x12 subdomains (2-layer overlap) converge, within each controller step, to
    the single-domain 6x6x22 explicit solution."""
    p = W.fom_fom_plain()
    ps = W.single_bar("single", 6, 22, "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20)
    A, S = oracle.Problem(p), oracle.Problem(ps)
    for _ in range(3):
        r = A.step()
        S.step()
        assert r["status"] == oracle.OK and 2 <= r["iterations"] < p.max_iters
    us, vs, _ = S.state(0)
    nn = 7 * 7
    for i, k0 in ((0, 0), (1, 10)):
        u, v, _ = A.state(i)
        n = u.shape[0]
        assert np.abs(u - us[k0 * nn:k0 * nn + n]).max() < 1e-12 * np.abs(us).max()
        assert np.abs(v - vs[k0 * nn:k0 * nn + n]).max() < 1e-12 * np.abs(vs).max()


# ---------------------------------------------------------------------------------------------
# OpInf ROM subdomain
# ---------------------------------------------------------------------------------------------
def _exact_linear_rom(oracle, p, i):
    """Full-basis ROM of LE subdomain i: Phi = I on its free dofs, Phi_S = I on its Schwarz dofs,
    K = -M^-1 K_ff, B = -M^-1 K_fS, H = 0, c = 0 (exact projection of the FOM)."""
    probe = oracle.Problem(p)
    free = probe.free_dofs(i)
    sdof = probe.schwarz_dofs(i)
    sd = p.subdomains[i]
    m = oracle.lumped_mass(sd.dims, sd.h, sd.origin, sd.rho)
    n3 = 3 * sd.n_nodes

    def col(d):
        e = np.zeros(n3)
        e[d] = 1.0
        f = oracle.internal_force(sd.dims, sd.h, sd.origin, "le", sd.lam, sd.mu, e)
        return -f[free] / m[free // 3]

    K = np.stack([col(d) for d in free], axis=1)
    B = np.stack([col(d) for d in sdof], axis=1)
    r = len(free)
    ops = {"Phi": np.eye(r), "Phi_S": np.eye(len(sdof)), "K": K, "H": np.zeros((r, r * (r + 1) // 2)), "B": B,
           "c": np.zeros(r)}
    return ops, free


def test_full_basis_rom_reproduces_fom_fom(oracle):
    """FOM-ROM coupling with the exact full-basis linear ROM equals FOM-FOM to rounding: checks the
    ROM step, the boundary projection ghat = Phi_S^T s and the reconstruction Pi Phi q."""
    pf = W.bar_chain("ff", 2, [4, 4], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    pr = W.bar_chain("fr", 2, [4, 4], ["fom", "rom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    ops, free = _exact_linear_rom(oracle, pf, 1)
    A = oracle.Problem(pf)
    B = oracle.Problem(pr, rom_ops={1: ops})
    for _ in range(4):
        ra, rb = A.step(), B.step()
        assert rb["status"] == oracle.OK
    ua, va, _ = A.state(0)
    ub, vb, _ = B.state(0)
    assert np.abs(ua - ub).max() < 1e-12 * np.abs(ua).max()
    u1, _, _ = A.state(1)
    q, qd, _ = B.rom_state(1)
    assert np.abs(q - u1.reshape(-1)[free]).max() < 1e-12 * np.abs(u1).max()
    uB, _, _ = B.state(1)
    assert np.abs(uB - u1).max() < 1e-12 * np.abs(u1).max()


@pytest.mark.parametrize("integrator0,counts", [("implicit", (5, 5)), ("explicit", (5, 3)), ("implicit", (2, 5))])
def test_full_basis_rom_reproduces_fom_fom_across_integrators_and_steps(oracle, integrator0, counts):
    """The exact full-basis linear ROM is an explicit FOM on its free dofs under any coupling: next to
    an implicit neighbour, and with its own step through the temporal interpolant, FOM-ROM equals the
    FOM-FOM run with the same integrators and counts to rounding."""
    def spec(kinds):
        p = W.bar_chain("x", 2, [4, 4], kinds, "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
        p.subdomains[0].integrator = integrator0
        p.subdomains[0].n_substeps, p.subdomains[1].n_substeps = counts
        return p
    pf, pr = spec(["fom", "fom"]), spec(["fom", "rom"])
    ops, free = _exact_linear_rom(oracle, pf, 1)
    A = oracle.Problem(pf)
    B = oracle.Problem(pr, rom_ops={1: ops})
    for _ in range(3):
        ra, rb = A.step(), B.step()
        assert ra["status"] == rb["status"] == oracle.OK and ra["iterations"] == rb["iterations"]
    ua, _, _ = A.state(0)
    ub, _, _ = B.state(0)
    assert np.abs(ua - ub).max() < 1e-12 * np.abs(ua).max()
    u1, v1, _ = A.state(1)
    q, qd, _ = B.rom_state(1)
    assert np.abs(q - u1.reshape(-1)[free]).max() < 1e-12 * np.abs(u1).max()
    assert np.abs(qd - v1.reshape(-1)[free]).max() < 1e-12 * np.abs(v1).max()


def _rotated_full_basis_rom(oracle, p, i, seed):
    """The exact full-basis linear ROM of subdomain i written in rotated bases: Phi = Q, Phi_S = Q_S
    (seeded random orthogonal, non-symmetric), K' = Q^T K Q, B' = Q^T B Q_S.  Then Phi q = u on the
    free dofs and B' Phi_S^T s = Q^T B s, so the ROM still reproduces the FOM exactly, but only if
    ghat = Phi_S^T s, the reconstruction Phi q and the initial projection q0 = Phi^T u0 each read
    their basis the right way round (Sec. 4.2.1, Eq. schwarz_opinf_discrete)."""
    ops, free = _exact_linear_rom(oracle, p, i)
    rng = np.random.default_rng(seed)
    r, rs = ops["K"].shape[0], ops["B"].shape[1]
    Q, _ = np.linalg.qr(rng.standard_normal((r, r)))
    QS, _ = np.linalg.qr(rng.standard_normal((rs, rs)))
    rot = {"Phi": Q, "Phi_S": QS, "K": Q.T @ ops["K"] @ Q, "H": np.zeros((r, r * (r + 1) // 2)),
           "B": Q.T @ ops["B"] @ QS, "c": np.zeros(r)}
    return rot, free


def rotated_rom_mismatch(oracle):
    """Largest relative deviation from FOM-FOM of three couplings of rotated full-basis ROMs (a
    FOM-ROM pair, a ROM-ROM pair and a FOM-ROM pair with its own substep count through Xi) over three
    controller steps: displacements of every subdomain (the ROM's reconstructed field) and the
    reduced state against Phi^T u of the FOM-FOM run.  Exact arithmetic gives 0."""
    worst = 0.0

    def spec(kinds, counts):
        sp = W.bar_chain("rot", 2, [4, 4], kinds, "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
        if counts:
            sp.subdomains[0].n_substeps, sp.subdomains[1].n_substeps = counts
        return sp

    for kinds, counts in ((["fom", "rom"], None), (["rom", "rom"], None), (["fom", "rom"], (5, 3))):
        pf = spec(["fom", "fom"], counts)
        rom_ops, frees = {}, {}
        for i, k in enumerate(kinds):
            if k == "rom":
                rom_ops[i], frees[i] = _rotated_full_basis_rom(oracle, pf, i, 100 + i)
        A = oracle.Problem(pf)
        B = oracle.Problem(spec(kinds, counts), rom_ops=rom_ops)
        for _ in range(3):
            ra, rb = A.step(), B.step()
            if rb["status"] != oracle.OK or ra["iterations"] != rb["iterations"]:
                return float("inf")
        for i in range(2):
            u = A.state(i)[0]
            scale = np.abs(u).max()
            worst = max(worst, np.abs(B.state(i)[0] - u).max() / scale)
            if i in rom_ops:
                q = B.rom_state(i)[0]
                worst = max(worst, np.abs(rom_ops[i]["Phi"] @ q - u.reshape(-1)[frees[i]]).max() / scale)
                worst = max(worst, np.abs(q - rom_ops[i]["Phi"].T @ u.reshape(-1)[frees[i]]).max() / scale)
    return worst


def test_rotated_full_basis_rom_reproduces_fom_fom(oracle):
    """Non-identity orthogonal Phi and Phi_S: FOM-ROM, ROM-ROM and FOM-ROM with mixed substep
    counts all equal FOM-FOM to 1e-12 (the identity-basis pins cannot see a transposed basis)."""
    assert rotated_rom_mismatch(oracle) < 1e-12


def test_rom_norm_identity(oracle):
    """The norm identity of an orthonormal basis, ||Phi dq|| = ||dq||, holds for the bases the
    rotated pin uses, and the ROM's reconstruction at the overlap is Phi q (checked through the
    reconstructed field above); this fixes the scale of the pin's tolerance."""
    pf = W.bar_chain("rot", 2, [4, 4], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    rot, _ = _rotated_full_basis_rom(oracle, pf, 1, 5)
    dq = np.random.default_rng(6).standard_normal(rot["Phi"].shape[1])
    assert abs(np.linalg.norm(rot["Phi"] @ dq) - np.linalg.norm(dq)) < 1e-13 * np.linalg.norm(dq)


# Each mutation reads one basis transposed: in the boundary projection ghat = Phi_S^T s, in the
# reconstruction Phi q, and in the initial projection q0 = Phi^T u0 of the set-up.
_BASIS_MUTATIONS = {
    "ghat": ("acc += s->PhiS[i * s->rs + k] * su[i];", "acc += s->PhiS[k * 3 * ns + i] * su[i];"),
    "reconstruction": ("val += s->Phi[(size_t)row * s->r + k] * qv[k];",
                       "val += s->Phi[(size_t)k * s->r + row] * qv[k];"),
    "initial_projection": ("a += s->Phi[(size_t)f * s->r + k] * s->u[s->free_dof[f]];",
                           "a += s->Phi[(size_t)k * s->r + f] * s->u[s->free_dof[f]];"),
}


@pytest.mark.parametrize("site", sorted(_BASIS_MUTATIONS))
def test_rotated_pin_fails_on_a_transposed_basis(tmp_path, site):
    """Plant a transposed basis read in a copy of the oracle (CPU only) and check that the rotated
    full-basis pin rejects it; the unmodified copy passes the same check."""
    import shutil
    import subprocess
    import sys
    root = os.path.dirname(HERE)
    src = open(os.path.join(root, "oracle", "osam_oracle.c")).read()
    before, after = _BASIS_MUTATIONS[site]
    assert src.count(before) == 1, f"mutation site {site} not found exactly once"
    results = {}
    for tag, text in (("planted", src.replace(before, after)), ("unmodified", src)):
        d = tmp_path / tag
        d.mkdir()
        shutil.copy(os.path.join(root, "oracle", "oracle.py"), d / "oracle.py")
        (d / "osam_oracle.c").write_text(text)
        code = ("import importlib.util, sys\n"
                f"sys.path.insert(0, {root!r})\n"
                f"spec = importlib.util.spec_from_file_location('oracle_copy', {str(d / 'oracle.py')!r})\n"
                "O = importlib.util.module_from_spec(spec); spec.loader.exec_module(O)\n"
                "from tests.test_oracle_pins import rotated_rom_mismatch\n"
                "print(rotated_rom_mismatch(O))\n")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        results[tag] = float(out.stdout.strip().splitlines()[-1])
    assert results["unmodified"] < 1e-12
    assert results["planted"] > 1e-6, results


def test_lame_relations_give_uniaxial_stress(oracle):
    """The (lambda, mu) of workloads.lame(E, nu), used by both sides, through the oracle's linear
    elastic force: under the affine field u = eps (x, -nu y, -nu z) of a uniaxial stress state the
    summed nodal force on the +x face is E eps times its area and the +y and +z faces carry no
    normal force.  A wrong nu term in lambda or mu breaks the second condition, a wrong E scale the
    first (Appendix A.1 with the standard isotropic relations)."""
    dims, h = (2, 3, 2), 0.01
    xyz, (ii, jj, kk) = _coords(dims, h, (0.0, 0.0, 0.0))
    X, Y, Z = xyz.T
    eps = 1e-4
    for E, nu in ((1e9, 0.2), (2e9, 0.3), (7e8, 0.25)):
        lam, mu = W.lame(E, nu)
        u = np.stack([eps * X, -nu * eps * Y, -nu * eps * Z], axis=1)
        f = oracle.internal_force(dims, h, (0.0, 0.0, 0.0), "le", lam, mu, u).reshape(-1, 3)
        ax, ay, az = dims[1] * dims[2] * h * h, dims[0] * dims[2] * h * h, dims[0] * dims[1] * h * h
        sxx = f[ii == dims[0], 0].sum() / ax
        syy = f[jj == dims[1], 1].sum() / ay
        szz = f[kk == dims[2], 2].sum() / az
        assert abs(sxx - E * eps) < 1e-10 * E * eps
        assert abs(syy) < 1e-10 * E * eps and abs(szz) < 1e-10 * E * eps
    # the check has teeth: Poisson's ratio in the wrong place of lambda leaves a lateral stress
    E, nu = 1e9, 0.3
    lam_bad, mu = E * nu / ((1 + nu) * (1 - nu)), E / (2 * (1 + nu))
    u = np.stack([eps * X, -nu * eps * Y, -nu * eps * Z], axis=1)
    f = oracle.internal_force(dims, h, (0.0, 0.0, 0.0), "le", lam_bad, mu, u).reshape(-1, 3)
    assert abs(f[jj == dims[1], 1].sum() / (dims[0] * dims[2] * h * h)) > 1e-3 * E * eps


# ---------------------------------------------------------------------------------------------
# stability limit of the explicit scheme (set-up check)
# ---------------------------------------------------------------------------------------------
def _assembled_stiffness(O, dims, h, lam, mu):
    """K of the linear elastic mesh by columns of the force of unit displacements (dense, small meshes)."""
    nx, ny, nz = dims
    ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    K = np.zeros((ndof, ndof))
    for j in range(ndof):
        u = np.zeros(ndof)
        u[j] = 1.0
        K[:, j] = O.internal_force(dims, h, (0.0, 0.0, 0.0), "le", lam, mu, u.reshape(-1, 3)).reshape(-1)
    return 0.5 * (K + K.T)


def _global_omega2(O, dims, h, lam, mu, rho):
    K = _assembled_stiffness(O, dims, h, lam, mu)
    m = np.repeat(O.lumped_mass(dims, h, (0.0, 0.0, 0.0), rho), 3)
    s = 1.0 / np.sqrt(m)
    return np.linalg.eigvalsh(s[:, None] * K * s[None, :])[-1]


def test_stable_dt_of_one_element_is_its_dense_eigenvalue(oracle):
    """For a single element the element bound is the exact limit 2 / sqrt(lambda_max(M^-1 K))."""
    O = oracle
    rng = np.random.default_rng(7)
    for _ in range(6):
        mu = float(rng.uniform(0.2, 3.0))
        lam = float(rng.uniform(-0.6, 20.0)) * mu
        h, rho = float(rng.uniform(0.5, 2.0)), float(rng.uniform(1.0, 10.0))
        w2 = _global_omega2(O, (1, 1, 1), h, lam, mu, rho)
        assert O.stable_dt((1, 1, 1), h, (0, 0, 0), lam, mu, rho) == pytest.approx(2.0 / np.sqrt(w2), rel=1e-12)


def test_stable_dt_closed_form_for_cube_elements(oracle):
    """The element eigenvalue of a cube with 2x2x2 Gauss points is h * max(3/2 lambda + mu, mu), so the
    limit is h sqrt(rho / max(3 lambda + 2 mu, 2 mu)): the form the library evaluates per element."""
    O = oracle
    rng = np.random.default_rng(8)
    for lam_over_mu in list(rng.uniform(-0.66, 200.0, 20)) + [0.0, -0.5, 1.0]:
        mu, rho, h = 4e8, 1000.0, 0.01
        lam = lam_over_mu * mu
        ref = h * np.sqrt(rho / max(3 * lam + 2 * mu, 2 * mu))
        assert O.stable_dt((2, 1, 1), h, (0, 0, 0), lam, mu, rho) == pytest.approx(ref, rel=1e-12)
    # per-element materials: the limit is set by the stiffest element
    lam_e = np.full(6, 4e8)
    mu_e = np.full(6, 4e8)
    lam_e[4] = 1.6e9
    ref = 0.01 * np.sqrt(1000.0 / (3 * 1.6e9 + 2 * 4e8))
    assert O.stable_dt((1, 2, 3), 0.01, (0, 0, 0), 4e8, 4e8, 1000.0, lam_e=lam_e, mu_e=mu_e) == pytest.approx(ref, rel=1e-12)
    assert O.stable_dt((1, 1, 1), 0.01, (0, 0, 0), -3e8, 4e8, 1000.0) == 0.0  # 3 lambda + 2 mu < 0
    assert O.stable_dt((1, 1, 1), 0.01, (0, 0, 0), 4e8, 0.0, 1000.0) == 0.0


def test_element_bound_dominates_the_assembled_spectrum(oracle):
    """Irons-Treharne: the assembled lumped-mass spectrum never exceeds the element bound, and on a
    free 2x2x3 block the bound is within a factor 2 of it."""
    O = oracle
    dims, h, rho = (2, 2, 3), 0.01, 1000.0
    w2 = _global_omega2(O, dims, h, LAM, MU, rho)
    dt_elem = O.stable_dt(dims, h, (0, 0, 0), LAM, MU, rho)
    dt_glob = 2.0 / np.sqrt(w2)
    assert dt_elem <= dt_glob * (1 + 1e-12)
    assert dt_elem > 0.5 * dt_glob


def test_central_difference_blows_up_just_above_the_limit(oracle):
    """The explicit integrator is stable just below omega_max dt = 2 and unstable just above it."""
    O = oracle
    dims, h, rho = (2, 2, 3), 0.01, 1000.0
    dt_glob = 2.0 / np.sqrt(_global_omega2(O, dims, h, LAM, MU, rho))
    ne = 12
    le, me = np.full(ne, LAM), np.full(ne, MU)
    u0 = _rand_disp(dims, 1e-6, 5)
    dm = np.zeros(u0.shape[0], np.uint8)
    below = O.rollout(dims, h, (0, 0, 0), "le", le, me, rho, dm, u0, None, 0.99 * dt_glob, 400)
    above = O.rollout(dims, h, (0, 0, 0), "le", le, me, rho, dm, u0, None, 1.02 * dt_glob, 400)
    assert np.abs(below).max() < 10 * np.abs(u0).max()
    assert np.abs(above).max() > 1e6 * np.abs(u0).max()


def test_problem_rejects_a_step_above_the_limit(oracle):
    O = oracle
    spec = W.fom_fom_plain()
    lim = O.stable_dt(spec.subdomains[0].dims, spec.subdomains[0].h, spec.subdomains[0].origin,
                      spec.subdomains[0].lam, spec.subdomains[0].mu, spec.subdomains[0].rho)
    spec.dt = 1.01 * lim
    with pytest.raises(O.OracleError) as ei:
        O.Problem(spec)
    assert ei.value.code == O.ECFL
    spec.dt = 0.99 * lim
    O.Problem(spec)
    # the 1D bar at Courant number 1 sits exactly on the limit and is accepted
    O.Problem(W.wave1d(n_elem=40))


# ---------------------------------------------------------------------------------------------
# implicit Newmark (average acceleration) subdomains
# ---------------------------------------------------------------------------------------------
def _implicit(spec, which=None):
    for i, sd in enumerate(spec.subdomains):
        if which is None or i in which:
            sd.integrator = "implicit"
    return spec


def test_implicit_linear_elastic_conserves_energy(oracle):
    """The average-acceleration rule conserves 1/2 v.Mv + 1/2 u.Ku exactly on a linear system, also at
    a time step five times the explicit stability limit (unconditional stability)."""
    p = W.single_bar("energy_imp", 3, 8, "le", 1e9, 0.25, 1000.0, 1e-3, 2e-6, 5)
    sd = p.subdomains[0]
    lim = oracle.stable_dt(sd.dims, sd.h, sd.origin, sd.lam, sd.mu, sd.rho)
    for dt in (2e-6, 5.0 * lim):
        p.dt = dt
        prob = oracle.Problem(_implicit(p))
        m = oracle.lumped_mass(sd.dims, sd.h, sd.origin, sd.rho)
        free = np.repeat(sd.dirichlet == 0, 3).reshape(-1, 3)

        def energy():
            u, v, _ = prob.state(0)
            f = oracle.internal_force(sd.dims, sd.h, sd.origin, "le", sd.lam, sd.mu, u).reshape(-1, 3)
            return 0.5 * np.sum((m[:, None] * v * v)[free]) + 0.5 * np.sum((u * f)[free])

        e0 = energy()
        es = []
        for _ in range(30):
            prob.step()
            es.append(energy())
        assert np.abs(np.array(es) - e0).max() < 1e-9 * e0


def test_implicit_and_explicit_agree_to_second_order(oracle):
    """Both integrators are second order: their difference after a fixed time falls ~4x per halving
    of the step (Neo-Hookean bar)."""
    diffs = []
    for n_sub, dt in ((10, 2e-6), (20, 1e-6), (40, 5e-7)):
        pe = W.single_bar("cmp", 3, 8, "nh", 1e9, 0.25, 1000.0, 2e-3, dt, n_sub)
        pi = _implicit(W.single_bar("cmp", 3, 8, "nh", 1e9, 0.25, 1000.0, 2e-3, dt, n_sub))
        A, B = oracle.Problem(pe), oracle.Problem(pi)
        for _ in range(3):
            A.step()
            B.step()
        diffs.append(np.abs(A.state(0)[0] - B.state(0)[0]).max())
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0


def test_implicit_fom_fom_schwarz_converges_to_single_domain(oracle):
    """Two implicit subdomains coupled by O-SAM reach the single-domain implicit solution to the
    Schwarz tolerance (implicit information crosses the overlap in every iteration, so the iteration
    converges geometrically rather than terminating)."""
    p = _implicit(W.bar_chain("imp2", 3, [8, 8], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10))
    ps = _implicit(W.single_bar("imp1", 3, 14, "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10))
    A, S = oracle.Problem(p), oracle.Problem(ps)
    for _ in range(3):
        r = A.step()
        S.step()
        assert r["status"] == oracle.OK
    us = S.state(0)[0]
    nn = 4 * 4
    for i, k0 in ((0, 0), (1, 6)):
        u = A.state(i)[0]
        assert np.abs(u - us[k0 * nn:k0 * nn + u.shape[0]]).max() < 1e-7 * np.abs(us).max()


# ---------------------------------------------------------------------------------------------
# different time steps per subdomain (temporal interpolant Xi of Sec. 4.1)
# ---------------------------------------------------------------------------------------------
def _translating_pair(material, n_sub, integrators):
    """Two overlapping unclamped 3x3x6 FOMs moving as a rigid body at constant velocity V: the exact
    solution u = V t, v = V, a = 0 is reproduced by both integrators, so the coupled run stays exact
    to rounding whatever the time levels of each subdomain, provided every Schwarz datum is taken at
    the right time (a misplaced level or weight shears the overlap at O(|V| dt))."""
    p = W.bar_chain("trans", 3, [6, 6], ["fom", "fom"], material, 1e9, 0.25, 1000.0, 0.0, 1e-6, 6, max_iters=10)
    V = np.array([0.3, -0.2, 0.5])
    for sd, n, integ in zip(p.subdomains, n_sub, integrators):
        sd.dirichlet = np.zeros(sd.n_nodes, np.uint8)
        sd.u0 = np.zeros((sd.n_nodes, 3))
        sd.v0 = np.tile(V, (sd.n_nodes, 1))
        sd.n_substeps = n
        sd.integrator = integ
    return p, V


@pytest.mark.parametrize("n_sub", [(6, 6), (6, 4), (5, 3), (3, 7)])
@pytest.mark.parametrize("integrators", [("explicit", "explicit"), ("explicit", "implicit")])
@pytest.mark.parametrize("schwarz", ["multiplicative", "additive"])
def test_mixed_time_steps_keep_rigid_translation_exact(oracle, n_sub, integrators, schwarz):
    """Rigid motion at constant velocity is an exact solution of every integrator and of the
    temporal interpolant (linear in time), under either sweep order."""
    p, V = _translating_pair("nh", n_sub, integrators)
    p.schwarz = schwarz
    prob = oracle.Problem(p)
    t = 0.0
    for _ in range(3):
        r = prob.step()
        assert r["status"] == oracle.OK
        t += p.dt * p.n_substeps
    for i in range(2):
        u, v, a = prob.state(i)
        assert np.abs(u - V * t).max() < 1e-13 * np.abs(V).max() * t
        assert np.abs(v - V).max() < 1e-12 * np.abs(V).max()
        assert np.abs(a).max() < 1e-6 * np.abs(V).max() / p.dt


def test_mixed_time_steps_equal_counts_reduce_to_the_common_step(oracle):
    """Setting every subdomain's substep count to the problem's is the plain common-step run."""
    p = W.bar_chain("eq", 3, [6, 6], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5)
    A = oracle.Problem(p)
    for sd in p.subdomains:
        sd.n_substeps = 5
    B = oracle.Problem(p)
    for _ in range(2):
        A.step()
        B.step()
    for i in range(2):
        for f in range(3):
            assert np.array_equal(A.state(i)[f], B.state(i)[f])


def test_mixed_time_steps_converge_at_second_order(oracle):
    """Omega_1 explicit with n substeps, Omega_2 implicit with n/2 (the paper's explicit / implicit
    pairing with Delta t_2 = 2 Delta t_1): against a single-domain run with a step 8x finer than the
    finest coupled one, the error falls ~4x per halving of both steps (the linear interpolant and both
    integrators are second order; conforming overlap meshes add no spatial coupling error)."""
    T = 2e-5
    ref_p = W.single_bar("ref", 3, 14, "le", 1e9, 0.25, 1000.0, 1e-3, T / 256, 256)
    ref = oracle.Problem(ref_p)
    for _ in range(2):
        ref.step()
    uref = ref.state(0)[0]
    nn = 4 * 4
    errs = []
    for n in (8, 16, 32):
        p = W.bar_chain("mix", 3, [8, 8], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, T / n, n, tol_rel=1e-13,
                        max_iters=60)
        p.subdomains[1].integrator = "implicit"
        p.subdomains[1].n_substeps = n // 2
        prob = oracle.Problem(p)
        for _ in range(2):
            assert prob.step()["status"] == oracle.OK
        e = 0.0
        for i, k0 in ((0, 0), (1, 6)):
            u = prob.state(i)[0]
            e = max(e, np.abs(u - uref[k0 * nn:k0 * nn + u.shape[0]]).max())
        errs.append(e)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


# ---------------------------------------------------------------------------------------------
# additive Schwarz and ROM-ROM coupling
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("integrator", ["explicit", "implicit"])
def test_additive_schwarz_reaches_the_single_domain_solution(oracle, integrator):
    """Additive (Jacobi) sweeps converge to the same coupled solution as multiplicative ones: the
    single-domain solution for conforming overlapping FOMs (to the Schwarz tolerance), using more
    iterations (information crosses one overlap per iteration instead of a whole sweep)."""
    p = W.bar_chain("add", 3, [8, 8], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10, tol_rel=1e-13,
                    max_iters=80)
    ps = W.single_bar("one", 3, 14, "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10)
    for sd in p.subdomains + ps.subdomains:
        sd.integrator = integrator
    pm = W.bar_chain("mul", 3, [8, 8], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 10, tol_rel=1e-13,
                     max_iters=80)
    for sd in pm.subdomains:
        sd.integrator = integrator
    p.schwarz = "additive"
    A, S, M = oracle.Problem(p), oracle.Problem(ps), oracle.Problem(pm)
    its_a, its_m = [], []
    for _ in range(3):
        ra, rm = A.step(), M.step()
        S.step()
        assert ra["status"] == oracle.OK and rm["status"] == oracle.OK
        its_a.append(ra["iterations"])
        its_m.append(rm["iterations"])
    us = S.state(0)[0]
    nn = 4 * 4
    for i, k0 in ((0, 0), (1, 6)):
        u = A.state(i)[0]
        assert np.abs(u - us[k0 * nn:k0 * nn + u.shape[0]]).max() < 1e-7 * np.abs(us).max()
    assert sum(its_a) > sum(its_m)


def test_additive_first_iteration_uses_only_the_zero_order_hold(oracle):
    """One iteration: the first subdomain of the sweep runs on the held data in both variants (equal
    states); the second sees its neighbour's new trace only in the multiplicative variant."""
    p = W.bar_chain("add1", 3, [6, 6], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=1)
    p.schwarz = "additive"
    A = oracle.Problem(p)
    A.step()
    q = W.bar_chain("add1", 3, [6, 6], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=1)
    B = oracle.Problem(q)
    B.step()
    assert np.array_equal(A.state(0)[0], B.state(0)[0])
    assert not np.array_equal(A.state(1)[0], B.state(1)[0])


def test_rom_rom_full_basis_reproduces_fom_fom(oracle):
    """OpInf-OpInf coupling: two exact full-basis linear ROMs reproduce the FOM-FOM run to rounding
    (ROM -> ROM reconstruction into the other ROM's boundary snapshots), multiplicative and additive."""
    for variant in ("multiplicative", "additive"):
        pf = W.bar_chain("ff", 2, [4, 4], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=200)
        pr = W.bar_chain("rr", 2, [4, 4], ["rom", "rom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 5, max_iters=200)
        pf.schwarz = pr.schwarz = variant
        ops0, free0 = _exact_linear_rom(oracle, pf, 0)
        ops1, free1 = _exact_linear_rom(oracle, pf, 1)
        A = oracle.Problem(pf)
        B = oracle.Problem(pr, rom_ops={0: ops0, 1: ops1})
        for _ in range(4):
            ra, rb = A.step(), B.step()
            assert rb["status"] == oracle.OK and ra["iterations"] == rb["iterations"]
        for i, free in ((0, free0), (1, free1)):
            u = A.state(i)[0]
            q = B.rom_state(i)[0]
            assert np.abs(q - u.reshape(-1)[free]).max() < 1e-12 * np.abs(u).max()
            assert np.abs(B.state(i)[0] - u).max() < 1e-12 * np.abs(u).max()



# ---------------------------------------------------------------------------------------------
# Saint Venant-Kirchhoff (Appendix A.2) and the tangents of the implicit solver
# ---------------------------------------------------------------------------------------------
def test_svk_energy_uses_the_green_lagrange_strain(oracle):
    """A.2 with E = 1/2 (F^T F - I): a pure stretch F = diag(1 + a) has E = diag(a + a^2/2); the
    printed "1/2 F^T F - I" would give a nonzero energy at F = I."""
    a = np.array([0.02, -0.01, 0.03])
    E = a + 0.5 * a * a
    ref = 0.5 * LAM * E.sum() ** 2 + MU * (E * E).sum()
    assert abs(oracle.energy_density("svk", np.diag(a), LAM, MU) - ref) < 1e-12 * ref
    assert oracle.energy_density("svk", np.zeros((3, 3)), LAM, MU) == 0.0


def test_svk_force_is_cubic_in_the_displacement(oracle):
    """f(t u) is a polynomial of degree exactly three in t for Saint Venant-Kirchhoff (Appendix A.2:
    the PDE has cubic nonlinearities); the Neo-Hookean force is not a cubic."""
    dims, h, org = (2, 1, 2), 0.01, (0.0, 0.0, 0.0)
    u = _rand_disp(dims, 0.02 * h, 11)
    ts = np.array([-2.0, -1.0, 1.0, 2.0, 3.0, 0.5])
    for material, cubic in (("svk", True), ("nh", False)):
        f = np.array([oracle.internal_force(dims, h, org, material, LAM, MU, t * u) for t in ts])
        V = np.vander(ts[:4], 4)
        coef = np.linalg.solve(V, f[:4])
        pred = np.vander(ts[4:], 4) @ coef
        err = np.abs(pred - f[4:]).max() / np.abs(f).max()
        if cubic:
            assert err < 1e-10 and np.abs(coef[0]).max() > 1e-6 * np.abs(coef[2]).max()
        else:
            assert err > 1e-8


def test_svk_is_objective_and_linearises_to_linear_elastic(oracle):
    dims, h, org = (2, 3, 2), 0.01, (0.05, 0.0, -0.02)
    X, _ = _coords(dims, h, org)
    th = 0.4
    R = np.array([[1, 0, 0], [0, np.cos(th), -np.sin(th)], [0, np.sin(th), np.cos(th)]])
    u = X @ (R - np.eye(3)).T + np.array([0.1, -0.3, 0.2])
    f_ref = oracle.internal_force(dims, h, org, "svk", LAM, MU, X @ (0.01 * np.eye(3)).T)
    assert np.abs(oracle.internal_force(dims, h, org, "svk", LAM, MU, u)).max() < 1e-9 * np.abs(f_ref).max()
    base = _rand_disp(dims, 1.0, 3)
    gaps = []
    for eps in (1e-4, 1e-5):
        w = eps * h * base
        f_s = oracle.internal_force(dims, h, org, "svk", LAM, MU, w)
        f_l = oracle.internal_force(dims, h, org, "le", LAM, MU, w)
        gaps.append(np.abs(f_s - f_l).max() / np.abs(f_l).max())
    assert gaps[0] < 1e-2 and 5.0 < gaps[0] / gaps[1] < 20.0


@pytest.mark.parametrize("material", ["le", "nh", "svk"])
def test_tangent_action_is_the_derivative_of_the_force(oracle, material):
    """K(u) p of the assembled element tangents equals the central difference of f_int along p (the
    Newton matrix of the implicit integrator)."""
    dims, h, org = (2, 2, 3), 0.01, (0.0, 0.1, 0.0)
    u = _rand_disp(dims, 0.03 * h, 12)
    p = _rand_disp(dims, 1.0, 13)
    y = oracle.tangent_action(dims, h, org, material, LAM, MU, u, p)
    eps = 1e-7 * h
    fd = (oracle.internal_force(dims, h, org, material, LAM, MU, u + eps * p)
          - oracle.internal_force(dims, h, org, material, LAM, MU, u - eps * p)) / (2 * eps)
    assert np.abs(y - fd).max() < 1e-6 * np.abs(fd).max()


def _free_mask(spec, i):
    """Free dofs of subdomain i from the spec alone: not clamped, not on a Schwarz node."""
    sd = spec.subdomains[i]
    snodes = np.zeros(sd.n_nodes, bool)
    for c in spec.couplings:
        if c.dst == i:
            snodes |= np.asarray(c.nodes, bool)
    dm = np.zeros(sd.n_nodes, np.uint8) if sd.dirichlet is None else np.asarray(sd.dirichlet)
    free = np.zeros((sd.n_nodes, 3), bool)
    for comp in range(3):
        free[:, comp] = ((dm >> comp) & 1) == 0
    free[snodes] = False
    return free.reshape(-1)


def test_convergence_criterion_is_eq_conv_criterion(oracle):
    """The c_num, c_den reported after the second sweep equal Eq. conv_criterion written out from the
    first and second iterates at t_k: each subdomain with its own step Delta t_i (here 1.5 us and 2 us
    in a 6 us interval),
    FOM terms over free dofs (neither clamped nor Schwarz), ROM terms over q and qdot.  The same sums
    with the common step, or without the velocity term, miss by far more than rounding."""
    def spec_with(max_iters):
        s = W.bar_chain("crit", 3, [7, 6], ["fom", "rom"], "nh", 1e9, 0.25, 1000.0, 2e-3, 1e-6, 6,
                        max_iters=max_iters)
        s.subdomains[0].n_substeps, s.subdomains[1].n_substeps = 4, 3
        return s
    s1 = spec_with(1)
    free0, free1 = _free_mask(s1, 0), _free_mask(s1, 1)
    n_sdof = 3 * int(np.asarray(s1.couplings[[c.dst for c in s1.couplings].index(1)].nodes, bool).sum())
    ops = {1: W.synthetic_rom_operators(int(free1.sum()), n_sdof, 5, 4, 31)}
    first = oracle.Problem(s1, rom_ops=ops)
    assert first.step()["iterations"] == 1
    second = oracle.Problem(spec_with(2), rom_ops=ops)
    rep = second.step()
    assert rep["iterations"] == 2
    T = s1.dt * s1.n_substeps
    dts = (T / 4, T / 3)
    (u1, v1, _), (u2, v2, _) = first.state(0), second.state(0)
    (q1, qd1, _), (q2, qd2, _) = first.rom_state(1), second.rom_state(1)
    du = (u2 - u1).reshape(-1)[free0]
    dv = (v2 - v1).reshape(-1)[free0]
    uu, vv = u2.reshape(-1)[free0], v2.reshape(-1)[free0]

    def sums(dt0, dt1, vel=1.0):
        num = np.sum((du + vel * dt0 * dv) ** 2) + np.sum(((q2 - q1) + vel * dt1 * (qd2 - qd1)) ** 2)
        den = np.sum((uu + vel * dt0 * vv) ** 2) + np.sum((q2 + vel * dt1 * qd2) ** 2)
        return num, den

    num, den = sums(*dts)
    assert rep["cnum"] > 0.0
    assert abs(rep["cnum"] - num) <= 1e-12 * num
    assert abs(rep["cden"] - den) <= 1e-12 * den
    for alt in (sums(s1.dt, s1.dt), sums(*dts, vel=0.0)):
        assert abs(alt[0] - num) > 1e-6 * num
