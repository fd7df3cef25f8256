"""Seeded synthetic workloads for the O-SAM FOM / OpInf hot path.

This module only builds inputs: mesh sizes, material parameters, node masks for the clamped and
Schwarz boundaries, and initial fields.  It holds none of the method's arithmetic, so both the
CUDA library and the CPU oracle can be fed from it.

Geometry conventions (shared interface of every consumer):
  * a subdomain is a structured box of nx*ny*nz cubic hex8 elements of edge h, origin at its
    (x, y, z)-minimum corner;
  * node (i, j, k) has index i + (nx+1)*(j + (ny+1)*k) and sits at origin + (i, j, k)*h;
  * per-node Dirichlet masks hold bit c set when component c is clamped to zero;
  * fields are [node][3] float64 arrays.

Workloads follow the paper's problems where it fixes them (the 1D wave bar of Sec. 5.1 with the
Symmetric Gaussian initial condition of its table of initial conditions) and the stated synthetic
configurations otherwise: a bar along z split into subdomains stacked with a 2-element-layer
overlap, clamped at z = 0, Gaussian initial z-displacement a*exp(-(z - z_c)^2 / (2 s^2)) with
z_c = mid-length and s = length / 10, zero initial velocity.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

H_DEFAULT = 0.01          # element edge [m]
OVERLAP_LAYERS = 2        # element layers shared by neighbouring subdomains
SEED_BASE = 20687


@dataclass
class Subdomain:
    kind: str                       # "fom" or "rom"
    dims: tuple                     # (nx, ny, nz) elements
    h: float
    origin: tuple
    material: str = "le"            # "le" (linear elastic) or "nh" (Neo-Hookean)
    lam: float = 0.0
    mu: float = 0.0
    rho: float = 1000.0
    lam_e: Optional[np.ndarray] = None
    mu_e: Optional[np.ndarray] = None
    dirichlet: Optional[np.ndarray] = None   # uint8 [N]
    u0: Optional[np.ndarray] = None          # [N, 3]
    v0: Optional[np.ndarray] = None          # [N, 3]
    integrator: str = "explicit"             # FOM time integrator: "explicit" (central differences) or "implicit"
    n_substeps: int = 0                      # substeps per controller step (0: the problem's n_substeps)

    @property
    def n_nodes(self) -> int:
        nx, ny, nz = self.dims
        return (nx + 1) * (ny + 1) * (nz + 1)

    @property
    def n_elements(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz

    def node_grid(self):
        nx, ny, nz = self.dims
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        return i.reshape(-1), j.reshape(-1), k.reshape(-1)

    def node_coords(self) -> np.ndarray:
        i, j, k = self.node_grid()
        o = self.origin
        return np.stack([o[0] + i * self.h, o[1] + j * self.h, o[2] + k * self.h], axis=1)


@dataclass
class Coupling:
    dst: int
    src: int
    nodes: np.ndarray                 # uint8 [N_dst]: nonzero = Schwarz node of dst fed by src


@dataclass
class Problem:
    name: str
    subdomains: List[Subdomain]
    couplings: List[Coupling]
    dt: float
    n_substeps: int
    tol_abs: float = 0.0
    tol_rel: float = 1e-12
    max_iters: int = 64
    n_controller_steps: int = 1
    info: dict = field(default_factory=dict)
    schwarz: str = "multiplicative"          # "multiplicative" (sequential sweep) or "additive"

    @property
    def fom_elements(self) -> int:
        return sum(s.n_elements for s in self.subdomains if s.kind == "fom")


def lame(E: float, nu: float):
    """Lame pair (lambda, mu) from Young's modulus and Poisson's ratio (standard relations)."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return lam, mu


def gaussian_z(coords: np.ndarray, amplitude: float, z_c: float, s: float) -> np.ndarray:
    u = np.zeros_like(coords)
    u[:, 2] = amplitude * np.exp(-((coords[:, 2] - z_c) ** 2) / (2.0 * s * s))
    return u


def bar_chain(name: str, nxy: int, nz_list: Sequence[int], kinds: Sequence[str], material: str, E: float,
              nu: float, rho: float, amplitude: float, dt: float, n_substeps: int, h: float = H_DEFAULT,
              overlap: int = OVERLAP_LAYERS, tol_rel: float = 1e-12, tol_abs: float = 0.0, max_iters: int = 64,
              n_controller_steps: int = 1, clamp_top: bool = False) -> Problem:
    """Bar along z made of len(nz_list) subdomains stacked with `overlap` shared element layers.

    Subdomain i's bottom face takes Schwarz data from i-1 and its top face from i+1; the bottom face of
    subdomain 0 is clamped (all components).  Each subdomain has nxy*nxy*nz_list[i] elements.
    """
    lam, mu = lame(E, nu)
    starts = [0]
    for nz in nz_list[:-1]:
        starts.append(starts[-1] + nz - overlap)
    length_layers = starts[-1] + nz_list[-1]
    L = length_layers * h
    z_c, s = 0.5 * L, L / 10.0
    subs, cpls = [], []
    for i, (nz, kind) in enumerate(zip(nz_list, kinds)):
        sd = Subdomain(kind=kind, dims=(nxy, nxy, nz), h=h, origin=(0.0, 0.0, starts[i] * h), material=material,
                       lam=lam, mu=mu, rho=rho)
        _, _, kk = sd.node_grid()
        dm = np.zeros(sd.n_nodes, np.uint8)
        if i == 0:
            dm[kk == 0] = 7
        if clamp_top and i == len(nz_list) - 1:
            dm[kk == nz] = 7
        sd.dirichlet = dm
        sd.u0 = gaussian_z(sd.node_coords(), amplitude, z_c, s)
        sd.v0 = np.zeros_like(sd.u0)
        subs.append(sd)
        if i > 0:
            cpls.append(Coupling(dst=i, src=i - 1, nodes=(kk == 0).astype(np.uint8)))
        if i < len(nz_list) - 1:
            cpls.append(Coupling(dst=i, src=i + 1, nodes=(kk == nz).astype(np.uint8)))
    return Problem(name=name, subdomains=subs, couplings=cpls, dt=dt, n_substeps=n_substeps, tol_abs=tol_abs,
                   tol_rel=tol_rel, max_iters=max_iters, n_controller_steps=n_controller_steps,
                   info={"length": L, "z_c": z_c, "s": s, "E": E, "nu": nu, "amplitude": amplitude})


def single_bar(name: str, nxy: int, nz: int, material: str, E: float, nu: float, rho: float, amplitude: float,
               dt: float, n_substeps: int, h: float = H_DEFAULT) -> Problem:
    """One subdomain covering the whole bar (the reference for FOM-FOM = single-domain checks)."""
    return bar_chain(name, nxy, [nz], ["fom"], material, E, nu, rho, amplitude, dt, n_substeps, h=h)


# ---------------------------------------------------------------------------------------------
# named configurations
# ---------------------------------------------------------------------------------------------
def fom_fom_plain() -> Problem:
    """Two 6x6x12 linear-elastic FOMs, 2-layer overlap (global 6x6x22), E=1e9, nu=0.25, rho=1000,
    pulse amplitude 1e-3 m, dt=1e-6 s, 200 steps in controller steps of 20, tol 1e-12, max 64 its."""
    return bar_chain("fom_fom_plain_6x6x12", 6, [12, 12], ["fom", "fom"], "le", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20,
                     max_iters=64, n_controller_steps=10)


def fom_opinf_hybrid(n: int = 40, nz: int = 80, rom: bool = True, n_controller_steps: int = 100) -> Problem:
    """Neo-Hookean FOM subdomain A (n x n x nz) coupled to subdomain B (mirror mesh) that is a
    quadratic OpInf ROM (rom=True) or a FOM (rom=False, the training run); dt=1e-6 s, controller 20."""
    kinds = ["fom", "rom" if rom else "fom"]
    return bar_chain(f"fom_opinf_hybrid_{n}x{n}x{nz}", n, [nz, nz], kinds, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20,
                     max_iters=64, n_controller_steps=n_controller_steps)


def adjoint_bar(n: int = 20, nz: int = 40, seed: int = SEED_BASE + 2, n_steps: int = 1000):
    """Single Neo-Hookean bar n x n x nz, per-element Lame parameters = nominal (E=1e9, nu=0.25) times
    (1 + 0.1 U[-1,1]), Gaussian initial displacement; returns (problem, tip weights w with J = w . u_T)."""
    p = single_bar(f"adjoint_{n}x{n}x{nz}", n, nz, "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, n_steps)
    sd = p.subdomains[0]
    rng = np.random.default_rng(seed)
    ne = sd.n_elements
    sd.lam_e = sd.lam * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, ne))
    sd.mu_e = sd.mu * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, ne))
    _, _, kk = sd.node_grid()
    tip = kk == nz
    w = np.zeros((sd.n_nodes, 3))
    w[tip, 2] = 1.0 / tip.sum()
    p.info["n_steps"] = n_steps
    p.info["checkpoint_every"] = 50
    return p, w


def batched_samples(n_samples: int = 256, seed: int = SEED_BASE + 3, n_min: int = 8, n_max: int = 32,
                    rom: bool = True) -> List[Problem]:
    """Parameter samples: E ~ U[0.5, 2]e9, nu ~ U[0.2, 0.35], amplitude ~ U[1e-4, 1e-3], mesh n x n x 2n
    per subdomain with n ~ U{n_min..n_max}; each a FOM / OpInf (or FOM / FOM) pair, dt=1e-6, controller 20."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_samples):
        E = rng.uniform(0.5e9, 2.0e9)
        nu = rng.uniform(0.2, 0.35)
        amp = rng.uniform(1e-4, 1e-3)
        n = int(rng.integers(n_min, n_max + 1))
        kinds = ["fom", "rom" if rom else "fom"]
        out.append(bar_chain(f"sample{s}_{n}", n, [2 * n, 2 * n], kinds, "nh", E, nu, 1000.0, amp, 1e-6, 20,
                             n_controller_steps=100))
    return out


def large_chain(n: int = 96, nz: int = 192, rom_middle: bool = True, amplitude: float = 1e-3,
                n_substeps: int = 20) -> Problem:
    """FOM / OpInf / FOM chain, FOM meshes n x n x nz Neo-Hookean, dt=5e-7 s, 10000 steps (controller 20).
    rom_middle=False gives the FOM-FOM-FOM run of the same geometry (the ROM's training run)."""
    kinds = ["fom", "rom" if rom_middle else "fom", "fom"]
    return bar_chain(f"large_chain_{n}x{n}x{nz}", n, [nz, nz, nz], kinds, "nh", 1e9, 0.25, 1000.0, amplitude, 5e-7,
                     n_substeps, n_controller_steps=10000 // n_substeps)


def subdomain_dof_masks(spec: Problem, i: int):
    """(free, schwarz) boolean masks over the dofs (node-major, 3 components) of subdomain i: Schwarz
    dofs are all components of the nodes a coupling into i feeds, free dofs are the rest minus the
    clamped components (the ROM's dof sets, in increasing dof order)."""
    sd = spec.subdomains[i]
    schwarz = np.zeros(sd.n_nodes, bool)
    for c in spec.couplings:
        if c.dst == i:
            schwarz |= np.asarray(c.nodes).astype(bool)
    dm = np.zeros(sd.n_nodes, np.uint8) if sd.dirichlet is None else np.asarray(sd.dirichlet, np.uint8)
    clamped = ((dm[:, None] >> np.arange(3, dtype=np.uint8)) & 1).astype(bool)
    free = (~clamped & ~schwarz[:, None]).reshape(-1)
    return free, np.repeat(schwarz, 3)


def wave1d(n_elem: int = 1000, dt: Optional[float] = None, subdomains: bool = False, n_substeps: int = 10) -> Problem:
    """The paper's 1D linear elastic wave bar (Sec. 5.1): (+-5e-4)^2 x (-0.5, 0.5) m, dx = 1e-3 m,
    E = 1 GPa, nu = 0, rho = 1000, x/y displacement fixed on the lateral faces, z clamped at both ends,
    Symmetric Gaussian u_z = a exp(-(z - b)^2 / (2 s^2)), a = 1e-3, b = 0, s = 2e-2.
    subdomains=True splits it into Omega_1 = (-0.5, 0.25) and Omega_2 = (-0.25, 0.5)."""
    L = 1.0
    h = L / n_elem
    E, rho, a, b, s = 1e9, 1000.0, 1e-3, 0.0, 2e-2
    c = (E / rho) ** 0.5
    dt = h / c if dt is None else dt
    lam, mu = lame(E, 0.0)
    if subdomains:
        n1 = int(round(0.75 / h))
        ranges = [(0, n1), (int(round(0.25 / h)), n_elem)]
    else:
        ranges = [(0, n_elem)]
    subs, cpls = [], []
    for i, (k0, k1) in enumerate(ranges):
        sd = Subdomain(kind="fom", dims=(1, 1, k1 - k0), h=h, origin=(-5e-4, -5e-4, -0.5 + k0 * h), material="le",
                       lam=lam, mu=mu, rho=rho)
        # the 1x1 cross-section has all nodes on the lateral faces: x and y fixed everywhere
        sd.h = h
        coords = sd.node_coords()
        _, _, kk = sd.node_grid()
        dm = np.full(sd.n_nodes, 3, np.uint8)
        if k0 == 0:
            dm[kk == 0] |= 4
        if k1 == n_elem:
            dm[kk == k1 - k0] |= 4
        sd.dirichlet = dm
        sd.u0 = gaussian_z(coords, a, b, s)
        sd.v0 = np.zeros_like(sd.u0)
        subs.append(sd)
    if subdomains:
        _, _, k0 = subs[0].node_grid()
        _, _, k1 = subs[1].node_grid()
        cpls.append(Coupling(dst=0, src=1, nodes=(k0 == subs[0].dims[2]).astype(np.uint8)))
        cpls.append(Coupling(dst=1, src=0, nodes=(k1 == 0).astype(np.uint8)))
    return Problem(name="wave1d", subdomains=subs, couplings=cpls, dt=dt, n_substeps=n_substeps, tol_abs=0.0,
                   tol_rel=1e-12, max_iters=64, info={"E": E, "rho": rho, "a": a, "b": b, "s": s, "c": c, "L": L})


def random_field(n_nodes: int, scale: float, seed: int) -> np.ndarray:
    return scale * np.random.default_rng(seed).standard_normal((n_nodes, 3))


def synthetic_rom_operators(n_free: int, n_sdof: int, r: int, r_s: int, seed: int,
                            omega_range=(1e4, 1e5)) -> dict:
    """Seeded stand-in operators of a quadratic ROM of the given sizes (random orthonormal bases,
    K = -diag(omega^2) with omega in omega_range rad/s, small random H and B, c = 0).  Used where a run
    needs ROM-sized work but no trained model (CPU baselines, full-size parity at a fixed iteration
    count)."""
    rng = np.random.default_rng(seed)
    Phi, _ = np.linalg.qr(rng.standard_normal((n_free, r)))
    Phi_S, _ = np.linalg.qr(rng.standard_normal((n_sdof, r_s)))
    omega = rng.uniform(omega_range[0], omega_range[1], r)
    K = -np.diag(omega ** 2)
    H = 1e6 * rng.standard_normal((r, r * (r + 1) // 2)) / r
    B = 1e8 * rng.standard_normal((r, r_s)) / r_s
    return {"Phi": Phi, "Phi_S": Phi_S, "K": K, "H": H, "B": B, "c": np.zeros(r)}
