"""Shared test helpers: error metrics and oracle-trained ROM operators (CPU oracle only)."""
import numpy as np

from oracle import fit as OF
from oracle import oracle as O


def rel_l2(hist, ref):
    """Eq. mse of the paper: sqrt(sum_k ||u_k - u_ref,k||^2) / sqrt(sum_k ||u_ref,k||^2)."""
    num = sum(np.sum((np.asarray(a) - np.asarray(b)) ** 2) for a, b in zip(hist, ref))
    den = sum(np.sum(np.asarray(b) ** 2) for b in ref)
    return np.sqrt(num / den)


def oracle_training(spec_ff, rom_index, n_ctrl):
    """Snapshots of subdomain rom_index from an oracle FOM-FOM run: displacement / acceleration on
    its free dofs and displacement on its Schwarz dofs, one per controller step."""
    prob = O.Problem(spec_ff)
    free = prob.free_dofs(rom_index)
    sdof = prob.schwarz_dofs(rom_index)
    U, A, S = [], [], []
    for _ in range(n_ctrl):
        prob.step()
        u, _, a = prob.state(rom_index)
        U.append(u.reshape(-1)[free])
        A.append(a.reshape(-1)[free])
        S.append(u.reshape(-1)[sdof])
    return np.array(U), np.array(A), np.array(S), free, sdof


def oracle_rom_ops(spec_ff, rom_index, n_ctrl, r, lam, r_s=None):
    U, A, S, free, sdof = oracle_training(spec_ff, rom_index, n_ctrl)
    ops = OF.opinf_fit(U.T, A.T, S.T, r=r, lam=lam, r_s=r_s)
    return ops, (U, A, S)
