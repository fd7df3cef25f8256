"""Pins of the oracle's offline OpInf fit and of its reverse-mode adjoint (CPU only)."""
import numpy as np
import pytest

from oracle import fit as OF
from paper_2511_20687_gb300 import workloads as W


def _orthonormal(n, r, rng):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def test_pod_eckart_young_and_orthonormality():
    """Eq. pod_cutoff: ||U - Phi_r Phi_r^T U||_F^2 = sum_{i>r} sigma_i^2, Phi_r orthonormal, and the
    energy rank is the smallest r with E_r >= delta (Eq. pod_energy, reading of its inequality)."""
    rng = np.random.default_rng(0)
    U = rng.standard_normal((300, 40)) @ np.diag(0.7 ** np.arange(40)) @ rng.standard_normal((40, 60))
    for r in (3, 10, 25):
        Phi, s = OF.pod(U, r)
        resid = np.linalg.norm(U - Phi @ (Phi.T @ U)) ** 2
        assert abs(resid - np.sum(s[r:] ** 2)) < 1e-10 * np.sum(s ** 2)
        assert np.abs(Phi.T @ Phi - np.eye(r)).max() < 1e-13
    E = OF.energy(s)
    r = OF.energy_rank(s, 0.999, 100)
    assert E[r - 1] >= 0.999 and E[r - 2] < 0.999


def test_kron_c_order():
    q = np.array([2.0, 3.0, 5.0])
    assert np.allclose(OF.kron_c(q[:, None])[:, 0], [4, 6, 10, 9, 15, 25])


def test_tikhonov_equals_augmented_least_squares():
    """The regularised problem equals plain least squares on [D; sqrt(lam) I] O = [Y; 0]."""
    rng = np.random.default_rng(1)
    D = rng.standard_normal((50, 80))
    Y = rng.standard_normal((50, 6))
    lam = 1e-3
    O = OF.tikhonov(D, Y, lam)
    Da = np.vstack([D, np.sqrt(lam) * np.eye(80)])
    Ya = np.vstack([Y, np.zeros((80, 6))])
    O2 = np.linalg.lstsq(Da, Ya, rcond=None)[0]
    assert np.abs(O - O2).max() < 1e-10 * np.abs(O2).max()
    # dual form D^T (D D^T + lam I)^-1 Y gives the same minimiser
    O3 = D.T @ np.linalg.solve(D @ D.T + lam * np.eye(50), Y)
    assert np.abs(O - O3).max() < 1e-9 * np.abs(O3).max()


def test_opinf_recovers_known_quadratic_operators():
    """Consistency of OpInf (Sec. 3.2): data drawn from a known quadratic model
    qdd = K q + H kron_c(q) + B ghat + c in known orthonormal bases is recovered with lambda -> 0.
    Bases are unique only up to rotation, so the check is basis-invariant: full-space accelerations
    Phi rhs(Phi^T u, Phi_S^T s) at fresh states."""
    rng = np.random.default_rng(2)
    n, ns, r, rs = 120, 30, 5, 3
    nq = r * (r + 1) // 2
    Phi_t, PhiS_t = _orthonormal(n, r, rng), _orthonormal(ns, rs, rng)
    K = rng.standard_normal((r, r))
    H = rng.standard_normal((r, nq))
    B = rng.standard_normal((r, rs))
    c = rng.standard_normal(r)
    nsnap = 3 * (r + nq + rs + 1)
    # well-spread singular values so the POD ordering is unambiguous
    Q = np.diag([5.0, 4.0, 3.0, 2.0, 1.0]) @ rng.standard_normal((r, nsnap))
    G = np.diag([3.0, 2.0, 1.0]) @ rng.standard_normal((rs, nsnap))
    Qdd = K @ Q + H @ OF.kron_c(Q) + B @ G + c[:, None]
    U, A, S = Phi_t @ Q, Phi_t @ Qdd, PhiS_t @ G
    ops = OF.opinf_fit(U, A, S, r=r, lam=1e-14, r_s=rs)
    q_new = rng.standard_normal((r, 10))
    g_new = rng.standard_normal((rs, 10))
    u_new, s_new = Phi_t @ q_new, PhiS_t @ g_new
    for k in range(10):
        want = Phi_t @ OF.rom_rhs(K, H, B, c, q_new[:, k], g_new[:, k])
        q = ops["Phi"].T @ u_new[:, k]
        g = ops["Phi_S"].T @ s_new[:, k]
        got = ops["Phi"] @ OF.rom_rhs(ops["K"], ops["H"], ops["B"], ops["c"], q, g)
        assert np.linalg.norm(got - want) < 1e-8 * np.linalg.norm(want)


# ---------------------------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_adjoint_case():
    p, w = W.adjoint_bar(n=2, nz=4, n_steps=30)
    sd = p.subdomains[0]
    # larger pulse so the nonlinearity matters
    return sd, w, p.dt, 30


@pytest.mark.parametrize("material", ["nh", "le"])
def test_force_vjp_dot_product(oracle, small_adjoint_case, material):
    """<ybar, (df/du) du> = <(df/du)^T ybar, du> with df/du du by central differences, and the
    parameter gradients match central differences of ybar . f in lambda_e, mu_e."""
    sd, _, _, _ = small_adjoint_case
    rng = np.random.default_rng(3)
    u = 2e-4 * rng.standard_normal((sd.n_nodes, 3))
    y = rng.standard_normal(3 * sd.n_nodes)
    du = rng.standard_normal(3 * sd.n_nodes)
    ub, lb, mb = oracle.force_vjp(sd.dims, sd.h, sd.origin, material, sd.lam_e, sd.mu_e, u, y)
    eps = 1e-7 * np.abs(u).max()
    f = lambda uu, le=sd.lam_e, me=sd.mu_e: oracle.internal_force(sd.dims, sd.h, sd.origin, material, 0, 0, uu,  # noqa
                                                                  lam_e=le, mu_e=me)
    jvp = (f(u.reshape(-1) + eps * du) - f(u.reshape(-1) - eps * du)) / (2 * eps)
    assert abs(y @ jvp - ub @ du) < 1e-7 * abs(ub @ du)
    dl = rng.standard_normal(sd.n_elements)
    el = 1e-6 * sd.lam
    fl = (f(u, le=sd.lam_e + el * dl) - f(u, le=sd.lam_e - el * dl)) / (2 * el)
    assert abs(y @ fl - lb @ dl) < 1e-7 * abs(lb @ dl)
    em = 1e-6 * sd.mu
    fm = (f(u, me=sd.mu_e + em * dl) - f(u, me=sd.mu_e - em * dl)) / (2 * em)
    assert abs(y @ fm - mb @ dl) < 1e-7 * abs(mb @ dl)


def test_rollout_adjoint_matches_central_differences(oracle, small_adjoint_case):
    """Gradients of J = w . u_T through the explicit rollout vs central differences (relative 1e-6)."""
    sd, w, dt, nsteps = small_adjoint_case
    args = (sd.dims, sd.h, sd.origin, "nh")
    u0 = sd.u0 * 3.0
    J, gu, gv, gl, gm = oracle.adjoint(*args, sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, u0, None, dt, nsteps, w)
    rng = np.random.default_rng(4)

    def Jof(uu=u0, vv=None, le=sd.lam_e, me=sd.mu_e):
        return w.reshape(-1) @ oracle.rollout(*args, le, me, sd.rho, sd.dirichlet, uu, vv, dt, nsteps)

    assert abs(Jof() - J) < 1e-14 * abs(J)
    d = rng.standard_normal(u0.shape)
    d[np.repeat(sd.dirichlet, 3).reshape(-1, 3) > 0] = 0
    h = 1e-6 * np.abs(u0).max()
    fd = (Jof(uu=u0 + h * d) - Jof(uu=u0 - h * d)) / (2 * h)
    assert abs(fd - gu @ d.reshape(-1)) < 1e-6 * abs(fd)
    hv = 1e-6 * np.abs(u0).max() / dt
    fdv = (Jof(vv=hv * d) - Jof(vv=-hv * d)) / (2 * hv)
    assert abs(fdv - gv @ d.reshape(-1)) < 1e-6 * abs(fdv)
    dl = rng.standard_normal(sd.n_elements)
    hl = 1e-6 * sd.lam
    fdl = (Jof(le=sd.lam_e + hl * dl) - Jof(le=sd.lam_e - hl * dl)) / (2 * hl)
    assert abs(fdl - gl @ dl) < 1e-6 * abs(fdl)
    hm = 1e-6 * sd.mu
    fdm = (Jof(me=sd.mu_e + hm * dl) - Jof(me=sd.mu_e - hm * dl)) / (2 * hm)
    assert abs(fdm - gm @ dl) < 1e-6 * abs(fdm)


# ---------------------------------------------------------------------------------------------
# regularisation selection (Algorithm 3)
# ---------------------------------------------------------------------------------------------
def _known_quadratic_trajectory(n=5, n_g=2, steps=400, dt=0.02, seed=3, k=1, cubic=0.0):
    """Trajectory of q'' = K q + H kron_c(q) (+ C kron3_c(q)) + B g(t) + c by explicit central
    differences with step dt, recorded every k steps; g(t) smooth; C of scale `cubic` (0: none).
    Returns snapshots (U, A, S, v0) and the step."""
    rng = np.random.default_rng(seed)
    K = -np.diag(rng.uniform(1.0, 4.0, n) ** 2)
    H = 0.05 * rng.standard_normal((n, n * (n + 1) // 2))
    B = rng.standard_normal((n, n_g))
    c = 0.1 * rng.standard_normal(n)
    Cc = None
    if cubic:   # restoring (Duffing) terms -cubic q_i^3 plus a small random part of the cube
        trip = [(i, j, l) for i in range(n) for j in range(i, n) for l in range(j, n)]
        Cc = 0.02 * cubic * rng.standard_normal((n, len(trip)))
        for i in range(n):
            Cc[i, trip.index((i, i, i))] -= cubic
    g = lambda t: np.array([np.sin(1.3 * t), np.cos(0.7 * t)])[:n_g]
    q = 0.1 * rng.standard_normal(n)
    qd = 0.1 * rng.standard_normal(n)
    qdd = OF.rom_rhs(K, H, B, c, q, g(0.0), Cc)
    U, A, S, V = [q.copy()], [qdd.copy()], [g(0.0)], [qd.copy()]
    t = 0.0
    for j in range(steps):
        for _ in range(k):
            t += dt
            q = q + dt * qd + 0.5 * dt * dt * qdd
            qn = OF.rom_rhs(K, H, B, c, q, g(t), Cc)
            qd = qd + 0.5 * dt * (qdd + qn)
            qdd = qn
        U.append(q.copy()); A.append(qdd.copy()); S.append(g(t)); V.append(qd.copy())
    return np.array(U).T, np.array(A).T, np.array(S).T, np.array(V)[0]


def test_selection_recovers_the_generating_model():
    """Noise-free data of a known quadratic model: small lambdas reproduce the trajectory, the largest
    ones do not, and the selected lambda is one of the small ones."""
    U, A, S, v0 = _known_quadratic_trajectory()
    lams = OF.lambda_grid()
    assert lams[0] == pytest.approx(1e-10) and lams[-1] == pytest.approx(1.0) and len(lams) == 11
    errs, best, ops = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.02, k=1, r_s=2)
    assert errs[0] < 1e-6 and errs[best] < 1e-6
    assert errs[-1] > 1e-3
    assert lams[best] <= 1e-4


CUBIC_SCALE = 20.0


def test_cubic_selection_recovers_a_cubic_model_that_the_quadratic_one_misses():
    """Noise-free data of a model with a cubic term: cubic candidates at small lambda reproduce the
    trajectory; the best quadratic candidate, which has no C block, stays orders of magnitude worse."""
    U, A, S, v0 = _known_quadratic_trajectory(cubic=CUBIC_SCALE, seed=4)
    lams = OF.lambda_grid()
    errs_c, best_c, ops = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.02, k=1, r_s=2, cubic=True)
    errs_q, best_q, _ = OF.select_lambda(U, A, S, v0, r=5, lambdas=lams, dt=0.02, k=1, r_s=2)
    assert errs_c[0] < 1e-6 and errs_c[best_c] < 1e-6 and lams[best_c] <= 1e-4
    assert ops["C"].shape == (5, 35)
    assert errs_q[best_q] > 1e3 * errs_c[best_c]


def test_selection_rollout_interpolates_the_boundary_between_snapshots():
    """Snapshots every 3 steps with a boundary input that is linear in time: the interpolated frozen
    boundary is exact, so the rollout of the generating operators reproduces the recorded states."""
    n, dt, k = 4, 0.01, 3
    rng = np.random.default_rng(5)
    K = -np.diag(rng.uniform(1.0, 3.0, n) ** 2)
    H = 0.02 * rng.standard_normal((n, n * (n + 1) // 2))
    B = rng.standard_normal((n, 1))
    c = np.zeros(n)
    q0, qd0 = 0.1 * rng.standard_normal(n), 0.1 * rng.standard_normal(n)
    g = lambda t: np.array([0.5 - 2.0 * t])
    # reference: every step with the exact boundary, recorded every k steps
    q, qd = q0.copy(), qd0.copy()
    qdd = OF.rom_rhs(K, H, B, c, q, g(0.0))
    Qref, G = [q.copy()], [g(0.0)]
    t = 0.0
    for j in range(60):
        for _ in range(k):
            t += dt
            q = q + dt * qd + 0.5 * dt * dt * qdd
            qn = OF.rom_rhs(K, H, B, c, q, g(t))
            qd = qd + 0.5 * dt * (qdd + qn)
            qdd = qn
        Qref.append(q.copy()); G.append(g(t))
    Qref, G = np.array(Qref).T, np.array(G).T
    Q = OF.rollout_frozen(K, H, B, c, q0, qd0, OF.rom_rhs(K, H, B, c, q0, g(0.0)), G, dt, k)
    assert np.abs(Q - Qref).max() < 1e-12 * np.abs(Qref).max()


def test_selection_penalises_a_non_finite_rollout():
    """A candidate whose rollout overflows scores +inf and is never selected."""
    n = 3
    K = np.diag([50.0, 1.0, -1.0]) ** 2  # one exponentially growing mode
    H = np.zeros((n, n * (n + 1) // 2)); B = np.zeros((n, 1)); c = np.zeros(n)
    G = np.zeros((1, 2000))
    Q = OF.rollout_frozen(K, H, B, c, np.ones(n), np.zeros(n), np.zeros(n), G, 1.0, 1)
    assert not np.all(np.isfinite(Q))


# ---------------------------------------------------------------------------------------------
# cubic OpInf (COpInf)
# ---------------------------------------------------------------------------------------------
def test_kron3_c_order():
    """Compressed Kronecker cube = products over index triples i <= j <= k in lexicographic order
    (itertools' combinations with replacement)."""
    import itertools
    q = np.array([2.0, 3.0, 5.0, 7.0])
    want = [np.prod(c) for c in itertools.combinations_with_replacement(q, 3)]
    assert np.array_equal(OF.kron3_c(q[:, None])[:, 0], want)
    assert OF.kron3_c(np.ones((6, 1))).shape[0] == 6 * 7 * 8 // 6


def test_opinf_recovers_known_cubic_operators():
    """Data of a known cubic model qdd = K q + H kron_c(q) + C kron3_c(q) + B ghat + c is recovered
    (basis-invariant check on fresh states), and dropping the cubic block leaves a visible residual."""
    rng = np.random.default_rng(5)
    n, ns, r, rs = 90, 20, 4, 2
    nq, nc = r * (r + 1) // 2, r * (r + 1) * (r + 2) // 6
    Phi_t, PhiS_t = _orthonormal(n, r, rng), _orthonormal(ns, rs, rng)
    K = rng.standard_normal((r, r))
    H = rng.standard_normal((r, nq))
    Cc = rng.standard_normal((r, nc))
    B = rng.standard_normal((r, rs))
    c = rng.standard_normal(r)
    nsnap = 3 * (r + nq + nc + rs + 1)
    Q = np.diag([4.0, 3.0, 2.0, 1.0]) @ rng.standard_normal((r, nsnap))
    G = np.diag([2.0, 1.0]) @ rng.standard_normal((rs, nsnap))
    Qdd = K @ Q + H @ OF.kron_c(Q) + Cc @ OF.kron3_c(Q) + B @ G + c[:, None]
    U, A, S = Phi_t @ Q, Phi_t @ Qdd, PhiS_t @ G
    ops = OF.opinf_fit(U, A, S, r=r, lam=1e-14, r_s=rs, cubic=True)
    quad = OF.opinf_fit(U, A, S, r=r, lam=1e-14, r_s=rs)
    q_new = rng.standard_normal((r, 10))
    g_new = rng.standard_normal((rs, 10))
    for k in range(10):
        want = Phi_t @ OF.rom_rhs(K, H, B, c, q_new[:, k], g_new[:, k], Cc)
        q = ops["Phi"].T @ (Phi_t @ q_new[:, k])
        g = ops["Phi_S"].T @ (PhiS_t @ g_new[:, k])
        got = ops["Phi"] @ OF.rom_rhs(ops["K"], ops["H"], ops["B"], ops["c"], q, g, ops["C"])
        assert np.linalg.norm(got - want) < 1e-8 * np.linalg.norm(want)
        got_q = quad["Phi"] @ OF.rom_rhs(quad["K"], quad["H"], quad["B"], quad["c"], q, g)
        assert np.linalg.norm(got_q - want) > 1e-2 * np.linalg.norm(want)


def test_cubic_rom_subdomain_integrates_a_duffing_oscillator(oracle):
    """A one-mode cubic ROM subdomain q'' = -w^2 q - g q^3 (K = -w^2, C = -g) advanced by the
    controller: its trajectory converges at second order to the ODE's solution (scipy, tight
    tolerances), and the cubic term changes it at leading order (sign and placement of C)."""
    from scipy.integrate import solve_ivp
    w, g, a0, T = 2.0e4, 4.0e14, 1e-3, 4e-4
    ref = solve_ivp(lambda t, y: [y[1], -w * w * y[0] - g * y[0] ** 3], (0.0, T), [a0, 0.0], rtol=1e-12,
                    atol=1e-16, method="DOP853").y[0, -1]
    lin = a0 * np.cos(w * T)
    assert abs(ref - lin) > 0.1 * a0  # the cubic term matters

    def run(n_steps):
        sd = W.Subdomain(kind="rom", dims=(1, 1, 1), h=0.01, origin=(0.0, 0.0, 0.0))
        sd.dirichlet = np.zeros(sd.n_nodes, np.uint8)
        sd.u0 = np.zeros((sd.n_nodes, 3))
        sd.u0[0, 0] = a0
        sd.v0 = np.zeros((sd.n_nodes, 3))
        p = W.Problem(name="duffing", subdomains=[sd], couplings=[], dt=T / n_steps, n_substeps=n_steps)
        Phi = np.zeros((3 * sd.n_nodes, 1))
        Phi[0, 0] = 1.0
        ops = {"Phi": Phi, "Phi_S": np.zeros((0, 0)), "K": np.array([[-w * w]]), "H": np.zeros((1, 1)),
               "C": np.array([[-g]]), "B": np.zeros((1, 0)), "c": np.zeros(1)}
        prob = oracle.Problem(p, rom_ops={0: ops})
        prob.step()
        return prob.rom_state(0)[0][0]

    errs = [abs(run(n) - ref) for n in (400, 800, 1600)]
    assert errs[2] < 1e-3 * a0
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_quadratic_rom_subdomain_integrates_its_ode(oracle):
    """A two-mode quadratic ROM subdomain q'' = K q + H kron_c(q) + c (Eq. schwarz_opinf_discrete with
    the constant of reading c10), kron_c(q) = (q0^2, q0 q1, q1^2), every H column and both c entries
    distinct: the controller's trajectory converges at second order to the ODE's solution (scipy,
    tight tolerances), and dropping H changes it at leading order -- so the compressed column order,
    the row order of H and the sign and placement of c are all pinned."""
    from scipy.integrate import solve_ivp
    w0, w1, a0, a1, T = 2.0e4, 3.0e4, 1e-3, 5e-4, 4e-4
    K = np.diag([-w0 * w0, -w1 * w1])
    H = np.array([[1e11, 3e11, -2e11], [-4e11, 2e11, 5e11]])
    c = np.array([1e4, -2e4])

    def rhs(t, y, Hm):
        q = y[:2]
        kq = np.array([q[0] * q[0], q[0] * q[1], q[1] * q[1]])
        return np.concatenate([y[2:], K @ q + Hm @ kq + c])

    ode = lambda Hm: solve_ivp(rhs, (0.0, T), [a0, a1, 0.0, 0.0], args=(Hm,), rtol=1e-12, atol=1e-18,
                               method="DOP853").y[:2, -1]
    ref = ode(H)
    assert np.abs(ref - ode(np.zeros_like(H))).max() > 0.05 * a0   # the quadratic term matters

    def run(n_steps):
        sd = W.Subdomain(kind="rom", dims=(1, 1, 1), h=0.01, origin=(0.0, 0.0, 0.0))
        sd.dirichlet = np.zeros(sd.n_nodes, np.uint8)
        sd.u0 = np.zeros((sd.n_nodes, 3))
        sd.u0[0, 0], sd.u0[0, 1] = a0, a1
        sd.v0 = np.zeros((sd.n_nodes, 3))
        p = W.Problem(name="quadratic", subdomains=[sd], couplings=[], dt=T / n_steps, n_substeps=n_steps)
        Phi = np.zeros((3 * sd.n_nodes, 2))
        Phi[0, 0] = Phi[1, 1] = 1.0
        ops = {"Phi": Phi, "Phi_S": np.zeros((0, 0)), "K": K, "H": H, "B": np.zeros((2, 0)), "c": c}
        prob = oracle.Problem(p, rom_ops={0: ops})
        prob.step()
        return prob.rom_state(0)[0]

    errs = [np.abs(run(n) - ref).max() for n in (400, 800, 1600)]
    assert errs[2] < 1e-3 * a0
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
