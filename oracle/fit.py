"""Plain FP64 oracle of the offline OpInf stage (POD bases + Tikhonov least squares).

TEST INFRASTRUCTURE ONLY (tests/, smoke() and bench.py's CPU legs).  Library primitives serve as
steps: numpy's thin SVD for POD and a dense solve of the normal equations for the regression.

  * POD (Sec. 3.1, Eq. pod_cutoff): thin SVD U = Phi Sigma Psi^T of the uncentered snapshot matrix,
    basis = first r left singular vectors (Euclidean inner product).
  * energy criterion (Eq. pod_energy): E_r = sum_{i<=r} sigma_i^2 / sum_i sigma_i^2; the reduced
    dimension is the smallest r with E_r >= delta_E.
  * boundary POD (Sec. 4.2.1): a separate basis Phi_S of the Schwarz boundary snapshots, reduced
    boundary data ghat = Phi_S^T s.
  * regression (Eq. opinf_schwarz_inference), solved form qdd = K q + H kron_c(q) + B ghat + c:
    minimise ||D O - Y||_F^2 + lambda ||O||_F^2 with D = [Ubar^T, kron_c(Ubar)^T, Ghat^T, 1],
    Y = Abar^T (projected acceleration snapshots), one scalar lambda for every block.  The cubic
    model (COpInf, Eq. quadratic_opinf with all terms) adds C kron3_c(q) and the block
    kron3_c(Ubar)^T after the quadratic one.
  * kron_c(q) = (q_i q_j)_{i <= j} in row-major upper-triangle order (compressed symmetric
    Kronecker square, the footnote of Sec. 2); kron3_c(q) = (q_i q_j q_k)_{i <= j <= k} in the same
    lexicographic order (compressed Kronecker cube, r(r+1)(r+2)/6 entries).
"""
from __future__ import annotations

import numpy as np


def pod(U: np.ndarray, r: int):
    """Thin SVD of the snapshot matrix U (n_dof x n_snap); returns (Phi_r, sigma)."""
    Phi, sigma, _ = np.linalg.svd(U, full_matrices=False)
    return Phi[:, :r].copy(), sigma


def energy(sigma: np.ndarray) -> np.ndarray:
    """E_r for r = 1..len(sigma)."""
    s2 = sigma.astype(np.float64) ** 2
    return np.cumsum(s2) / s2.sum()


def energy_rank(sigma: np.ndarray, delta: float, r_max: int) -> int:
    E = energy(sigma)
    r = int(np.searchsorted(E, delta, side="left")) + 1
    return max(1, min(r, r_max, len(sigma)))


def kron_c(Q: np.ndarray) -> np.ndarray:
    """Compressed Khatri-Rao square of the columns of Q (r x n) -> (r(r+1)/2 x n)."""
    r = Q.shape[0]
    rows = []
    for i in range(r):
        for j in range(i, r):
            rows.append(Q[i] * Q[j])
    return np.array(rows)


def kron3_c(Q: np.ndarray) -> np.ndarray:
    """Compressed Khatri-Rao cube of the columns of Q (r x n) -> (r(r+1)(r+2)/6 x n)."""
    r = Q.shape[0]
    rows = []
    for i in range(r):
        for j in range(i, r):
            for k in range(j, r):
                rows.append(Q[i] * Q[j] * Q[k])
    return np.array(rows).reshape(-1, Q.shape[1])


def data_matrix(Ubar: np.ndarray, Ghat: np.ndarray, quadratic: bool = True, cubic: bool = False) -> np.ndarray:
    blocks = [Ubar.T]
    if quadratic or cubic:
        blocks.append(kron_c(Ubar).T)
    if cubic:
        blocks.append(kron3_c(Ubar).T)
    blocks.append(Ghat.T)
    blocks.append(np.ones((Ubar.shape[1], 1)))
    return np.hstack(blocks)


def tikhonov(D: np.ndarray, Y: np.ndarray, lam: float) -> np.ndarray:
    """argmin_O ||D O - Y||_F^2 + lam ||O||_F^2 via the normal equations (D^T D + lam I) O = D^T Y."""
    d = D.shape[1]
    return np.linalg.solve(D.T @ D + lam * np.eye(d), D.T @ Y)


def unpack(O: np.ndarray, r: int, r_s: int, quadratic: bool = True, cubic: bool = False):
    """Operator blocks of the stacked solution O; with cubic=True returns (K, H, C, B, c)."""
    quadratic = quadratic or cubic
    nq = r * (r + 1) // 2 if quadratic else 0
    nc = r * (r + 1) * (r + 2) // 6 if cubic else 0
    K = O[:r].T.copy()
    H = O[r:r + nq].T.copy() if quadratic else np.zeros((r, r * (r + 1) // 2))
    C = O[r + nq:r + nq + nc].T.copy()
    B = O[r + nq + nc:r + nq + nc + r_s].T.copy()
    c = O[r + nq + nc + r_s].copy()
    if cubic:
        return K, H, C, B, c
    return K, H, B, c


def opinf_fit(U: np.ndarray, A: np.ndarray, S: np.ndarray, r: int, lam: float, r_s: int = None,
              energy_s: float = 1.0 - 1e-6, r_s_max: int = 64, quadratic: bool = True, cubic: bool = False):
    """U, A: free-dof displacement / acceleration snapshots (n_dof x n_snap); S: Schwarz boundary
    snapshots (n_sdof x n_snap).  Returns the ROM operators and bases."""
    Phi, sigma = pod(U, r)
    _, sigma_s, _ = np.linalg.svd(S, full_matrices=False)
    if r_s is None:
        r_s = energy_rank(sigma_s, energy_s, r_s_max)
    Phi_S, _ = pod(S, r_s)
    Ubar = Phi.T @ U
    Abar = Phi.T @ A
    Ghat = Phi_S.T @ S
    D = data_matrix(Ubar, Ghat, quadratic, cubic)
    O = tikhonov(D, Abar.T, lam)
    ops = {"Phi": Phi, "Phi_S": Phi_S, "sigma": sigma, "sigma_s": sigma_s, "r": r, "r_s": r_s}
    if cubic:
        ops["K"], ops["H"], ops["C"], ops["B"], ops["c"] = unpack(O, r, r_s, quadratic, cubic)
    else:
        ops["K"], ops["H"], ops["B"], ops["c"] = unpack(O, r, r_s, quadratic)
    return ops


def rom_rhs(K, H, B, c, q, ghat, C=None):
    out = K @ q + H @ kron_c(q[:, None])[:, 0] + B @ ghat + c
    if C is not None:
        out = out + C @ kron3_c(q[:, None])[:, 0]
    return out


# ---------------------------------------------------------------------------------------------
# Schwarz-aware regularisation selection (Sec. 4.2.4, Algorithm 3, Eq. schwarz_regularization_error)
# ---------------------------------------------------------------------------------------------
def lambda_grid(n: int = 11, lo: float = 1e-10, hi: float = 1.0) -> np.ndarray:
    """Logarithmically spaced candidates lo .. hi (the paper's grid: 11 values from 1e-10 to 1)."""
    return np.logspace(np.log10(lo), np.log10(hi), n)


def rollout_frozen(K, H, B, c, q0, qd0, qdd0, Ghat, dt, k, C=None):
    """Advance the ROM alone with its Schwarz boundary data frozen to the training columns.

    Explicit central differences (Newmark beta = 0, gamma = 1/2) with step dt; the snapshot columns
    are k steps apart, and within an interval the boundary vector is the linear interpolant in time of
    the two columns (k = 1: the stored column of the new time level, as the paper prescribes).
    Returns the reduced displacements at the snapshot times (r x n_snap)."""
    q, qd, qdd = q0.astype(np.float64).copy(), qd0.astype(np.float64).copy(), qdd0.astype(np.float64).copy()
    n = Ghat.shape[1]
    Q = np.empty((q.shape[0], n))
    Q[:, 0] = q
    with np.errstate(all="ignore"):
        for j in range(n - 1):
            for s in range(1, k + 1):
                g = Ghat[:, j] + (s / k) * (Ghat[:, j + 1] - Ghat[:, j])
                q = q + dt * qd + 0.5 * dt * dt * qdd
                qdd_new = rom_rhs(K, H, B, c, q, g, C)
                qd = qd + 0.5 * dt * (qdd + qdd_new)
                qdd = qdd_new
            Q[:, j + 1] = q
    return Q


def select_lambda(U, A, S, v0, r, lambdas, dt, k, r_s=None, energy_s=1.0 - 1e-6, r_s_max=64, quadratic=True,
                  cubic=False):
    """Algorithm 3: for every candidate lambda fit the operators (Eq. opinf_schwarz_inference), roll
    the ROM out from the training initial state (q0 = Phi^T u_0, qd0 = Phi^T v_0, qdd0 = Phi^T a_0)
    under the frozen training boundary data, score E(lambda) = ||Q - Ubar||_F / ||Ubar||_F (a
    non-finite rollout scores +inf), and return (errors, index of the minimum, operators refitted at
    the selected lambda)."""
    errors = []
    for lam in lambdas:
        ops = opinf_fit(U, A, S, r, lam, r_s, energy_s, r_s_max, quadratic, cubic)
        Phi, PhiS = ops["Phi"], ops["Phi_S"]
        Ubar = Phi.T @ U
        Q = rollout_frozen(ops["K"], ops["H"], ops["B"], ops["c"], Ubar[:, 0], Phi.T @ v0, Phi.T @ A[:, 0],
                           PhiS.T @ S, dt, k, ops.get("C"))
        if np.all(np.isfinite(Q)):
            errors.append(float(np.linalg.norm(Q - Ubar) / np.linalg.norm(Ubar)))
        else:
            errors.append(np.inf)
        if r_s is None:
            r_s = ops["r_s"]   # the boundary basis does not depend on lambda
    errors = np.array(errors)
    best = int(np.argmin(errors))
    return errors, best, opinf_fit(U, A, S, r, float(lambdas[best]), r_s, energy_s, r_s_max, quadratic, cubic)
