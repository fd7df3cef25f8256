"""Python handle on the plain FP64 CPU oracle (``osam_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference legs may import this module; the product path never does.  It shares no code with the
CUDA library: it compiles and loads its own C file with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osam_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, MAXITER, EINVAL, ECFL, ENONFINITE, EDONOR, ENOMEM = 0, 1, -1, -2, -3, -4, -7


class OracleError(ValueError):
    def __init__(self, code, msg):
        super().__init__(f"{msg}: {code}")
        self.code = code
LE, NH, SVK = 0, 1, 2

_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int)
_u8 = C.POINTER(C.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, single thread, no OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_internal_force.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, C.c_double,
                                             C.c_double, _d, _d, _d, _d]
            L.orc_strain_energy.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, C.c_double,
                                            C.c_double, _d, _d, _d]
            L.orc_strain_energy.restype = C.c_double
            L.orc_stress.argtypes = [C.c_int, _d, C.c_double, C.c_double, _d]
            L.orc_energy_density.argtypes = [C.c_int, _d, C.c_double, C.c_double]
            L.orc_energy_density.restype = C.c_double
            L.orc_lumped_mass.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_double, _d]
            L.orc_lumped_mass.restype = None
            L.orc_force_vjp.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, _d, _d, _d, _d, _d,
                                        _d, _d]
            L.orc_donor.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, _d, _i, _d]
            L.orc_stable_dt.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_double, C.c_double, _d, _d,
                                        C.c_double]
            L.orc_stable_dt.restype = C.c_double
            L.orc_problem_new.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
            L.orc_problem_new.restype = C.c_void_p
            L.orc_problem_free.argtypes = [C.c_void_p]
            L.orc_problem_free.restype = None
            L.orc_add_fom.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, C.c_double,
                                      C.c_double, C.c_double, _d, _d, _u8, _d, _d]
            L.orc_add_rom.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, _d, _u8, C.c_int, C.c_int,
                                      C.c_int, C.c_int, _d, _d, _d, _d, _d, _d, _d, _d]
            L.orc_couple.argtypes = [C.c_void_p, C.c_int, C.c_int, _u8]
            L.orc_init.argtypes = [C.c_void_p]
            L.orc_set_implicit.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_set_substeps.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_tangent_action.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, C.c_double,
                                             C.c_double, _d, _d, _d]
            L.orc_set_additive.argtypes = [C.c_void_p, C.c_int]
            L.orc_set_rom_cubic.argtypes = [C.c_void_p, C.c_int, _d]
            L.orc_step.argtypes = [C.c_void_p, _i, _d, _d]
            L.orc_num_nodes.argtypes = [C.c_void_p, C.c_int]
            L.orc_num_free.argtypes = [C.c_void_p, C.c_int]
            L.orc_num_schwarz.argtypes = [C.c_void_p, C.c_int]
            L.orc_get_state.argtypes = [C.c_void_p, C.c_int, _d, _d, _d]
            L.orc_get_rom.argtypes = [C.c_void_p, C.c_int, _d, _d, _d]
            L.orc_schwarz_dofs.argtypes = [C.c_void_p, C.c_int, _i]
            L.orc_free_dofs.argtypes = [C.c_void_p, C.c_int, _i]
            L.orc_rollout.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, _d, _d, C.c_double, _u8,
                                      _d, _d, C.c_double, C.c_int, _d]
            L.orc_adjoint.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _d, C.c_int, _d, _d, C.c_double, _u8,
                                      _d, _d, C.c_double, C.c_int, _d, _d, _d, _d, _d, _d]
            _lib = L
    return _lib


def _p(a):
    """ctypes pointer to a C-contiguous float64 / int32 / uint8 array, or NULL for None."""
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_d)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_i)
    if a.dtype == np.uint8:
        return a.ctypes.data_as(_u8)
    raise TypeError(a.dtype)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _mat(name):
    if name in ("svk", "saint_venant_kirchhoff", SVK):
        return SVK
    return NH if name in ("nh", "neo_hookean", NH) else LE


# ---------------------------------------------------------------------------------------------
# element-level functions
# ---------------------------------------------------------------------------------------------
def internal_force(dims, h, origin, material, lam, mu, u, lam_e=None, mu_e=None):
    nx, ny, nz = dims
    u = _f64(u).reshape(-1)
    f = np.zeros_like(u)
    org = _f64(origin)
    lam_e, mu_e = _f64(lam_e), _f64(mu_e)
    lib().orc_internal_force(nx, ny, nz, h, _p(org), _mat(material), lam, mu, _p(lam_e), _p(mu_e), _p(u), _p(f))
    return f


def strain_energy(dims, h, origin, material, lam, mu, u, lam_e=None, mu_e=None):
    nx, ny, nz = dims
    u = _f64(u).reshape(-1)
    org = _f64(origin)
    lam_e, mu_e = _f64(lam_e), _f64(mu_e)
    return lib().orc_strain_energy(nx, ny, nz, h, _p(org), _mat(material), lam, mu, _p(lam_e), _p(mu_e), _p(u))


def stress(material, H, lam, mu):
    H = _f64(H).reshape(9)
    P = np.zeros(9)
    lib().orc_stress(_mat(material), _p(H), lam, mu, _p(P))
    return P.reshape(3, 3)


def energy_density(material, H, lam, mu):
    H = _f64(H).reshape(9)
    return lib().orc_energy_density(_mat(material), _p(H), lam, mu)


def tangent_action(dims, h, origin, material, lam, mu, u, p):
    """K(u) p with the oracle's assembled element tangents (Appendix A tangents)."""
    nx, ny, nz = dims
    u, p = _f64(u), _f64(p)
    y = np.zeros(u.size)
    lib().orc_tangent_action(nx, ny, nz, h, _p(_f64(origin)), _mat(material), lam, mu, _p(u), _p(p), _p(y))
    return y


def lumped_mass(dims, h, origin, rho):
    nx, ny, nz = dims
    m = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    lib().orc_lumped_mass(nx, ny, nz, h, _p(_f64(origin)), rho, _p(m))
    return m


def stable_dt(dims, h, origin, lam, mu, rho, lam_e=None, mu_e=None):
    """Largest stable explicit time step by the element eigenvalue bound (0: material not positive definite)."""
    nx, ny, nz = dims
    le, me = _f64(lam_e), _f64(mu_e)
    return lib().orc_stable_dt(nx, ny, nz, h, _p(_f64(origin)), lam, mu, _p(le), _p(me), rho)


def force_vjp(dims, h, origin, material, lam_e, mu_e, u, ybar):
    nx, ny, nz = dims
    u, ybar = _f64(u).reshape(-1), _f64(ybar).reshape(-1)
    lam_e, mu_e = _f64(lam_e), _f64(mu_e)
    ub = np.zeros_like(u)
    lb = np.zeros(nx * ny * nz)
    mb = np.zeros(nx * ny * nz)
    lib().orc_force_vjp(nx, ny, nz, h, _p(_f64(origin)), _mat(material), _p(lam_e), _p(mu_e), _p(u), _p(ybar),
                        _p(ub), _p(lb), _p(mb))
    return ub, lb, mb


def donor(dims, h, origin, x):
    nx, ny, nz = dims
    nodes = np.zeros(8, np.int32)
    w = np.zeros(8)
    rc = lib().orc_donor(nx, ny, nz, h, _p(_f64(origin)), _p(_f64(x)), _p(nodes), _p(w))
    if rc != OK:
        raise ValueError("no donor element")
    return nodes, w


def rollout(dims, h, origin, material, lam_e, mu_e, rho, dmask, u0, v0, dt, nsteps):
    nx, ny, nz = dims
    u0 = _f64(u0).reshape(-1)
    v0 = _f64(v0).reshape(-1) if v0 is not None else np.zeros_like(u0)
    uT = np.zeros_like(u0)
    lib().orc_rollout(nx, ny, nz, h, _p(_f64(origin)), _mat(material), _p(_f64(lam_e)), _p(_f64(mu_e)), rho,
                      _p(np.ascontiguousarray(dmask, np.uint8)), _p(u0), _p(v0), dt, nsteps, _p(uT))
    return uT


def adjoint(dims, h, origin, material, lam_e, mu_e, rho, dmask, u0, v0, dt, nsteps, w):
    """J = w . u_T and its gradients w.r.t. u0, v0, lambda_e, mu_e (reverse-mode of the explicit rollout)."""
    nx, ny, nz = dims
    u0 = _f64(u0).reshape(-1)
    v0 = _f64(v0).reshape(-1) if v0 is not None else np.zeros_like(u0)
    w = _f64(w).reshape(-1)
    J = np.zeros(1)
    gu, gv = np.zeros_like(u0), np.zeros_like(u0)
    gl, gm = np.zeros(nx * ny * nz), np.zeros(nx * ny * nz)
    rc = lib().orc_adjoint(nx, ny, nz, h, _p(_f64(origin)), _mat(material), _p(_f64(lam_e)), _p(_f64(mu_e)), rho,
                           _p(np.ascontiguousarray(dmask, np.uint8)), _p(u0), _p(v0), dt, nsteps, _p(w), _p(J),
                           _p(gu), _p(gv), _p(gl), _p(gm))
    if rc != OK:
        raise MemoryError("oracle adjoint failed")
    return float(J[0]), gu, gv, gl, gm


# ---------------------------------------------------------------------------------------------
# coupled Schwarz problem
# ---------------------------------------------------------------------------------------------
class Problem:
    """The oracle's O-SAM problem built from a workload spec (see paper_2511_20687_gb300.workloads)."""

    def __init__(self, spec, rom_ops=None):
        L = lib()
        self._keep = []
        self.spec = spec
        self.h = L.orc_problem_new(spec.dt, spec.n_substeps, spec.tol_abs, spec.tol_rel, spec.max_iters)
        rom_ops = rom_ops or {}
        self.rank = {}
        for i, sd in enumerate(spec.subdomains):
            nx, ny, nz = sd.dims
            org = _f64(sd.origin)
            dm = np.ascontiguousarray(sd.dirichlet, np.uint8)
            u0 = _f64(sd.u0).reshape(-1)
            v0 = _f64(sd.v0).reshape(-1) if sd.v0 is not None else None
            self._keep += [org, dm, u0, v0]
            if sd.kind == "fom":
                le, me = _f64(sd.lam_e), _f64(sd.mu_e)
                self._keep += [le, me]
                rc = L.orc_add_fom(self.h, nx, ny, nz, sd.h, _p(org), _mat(sd.material), sd.lam, sd.mu, sd.rho,
                                   _p(le), _p(me), _p(dm), _p(u0), _p(v0))
                if rc >= 0 and getattr(sd, "integrator", "explicit") == "implicit":
                    rc = L.orc_set_implicit(self.h, i, 1)
            else:
                ops = rom_ops[i]
                arrs = [_f64(ops[k]) for k in ("Phi", "Phi_S", "K", "H", "B", "c")]
                self._keep += arrs
                r = arrs[0].shape[1]
                rs = arrs[1].shape[1]
                self.rank[i] = r
                rc = L.orc_add_rom(self.h, nx, ny, nz, sd.h, _p(org), _p(dm), r, rs, arrs[0].shape[0],
                                   arrs[1].shape[0], *[_p(a) for a in arrs], _p(u0), _p(v0))
                if rc >= 0 and ops.get("C") is not None:
                    Cc = _f64(ops["C"])
                    self._keep.append(Cc)
                    rc = L.orc_set_rom_cubic(self.h, i, _p(Cc))
            if rc >= 0 and getattr(sd, "n_substeps", 0):
                rc = L.orc_set_substeps(self.h, i, int(sd.n_substeps))
            if rc < 0:
                raise OracleError(rc, f"oracle add subdomain {i}")
        for cp in spec.couplings:
            m = np.ascontiguousarray(cp.nodes, np.uint8)
            self._keep.append(m)
            if L.orc_couple(self.h, cp.dst, cp.src, _p(m)) < 0:
                raise ValueError("oracle couple")
        if getattr(spec, "schwarz", "multiplicative") == "additive":
            L.orc_set_additive(self.h, 1)
        rc = L.orc_init(self.h)
        if rc != OK:
            raise OracleError(rc, "oracle init failed")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_problem_free(self.h)
            self.h = None

    def step(self):
        it = np.zeros(1, np.int32)
        cn, cd = np.zeros(1), np.zeros(1)
        rc = lib().orc_step(self.h, _p(it), _p(cn), _p(cd))
        if rc < 0:
            raise OracleError(rc, "oracle step failed")
        return {"status": rc, "iterations": int(it[0]), "cnum": float(cn[0]), "cden": float(cd[0])}

    def state(self, i):
        n = lib().orc_num_nodes(self.h, i)
        u, v, a = (np.zeros(3 * n) for _ in range(3))
        lib().orc_get_state(self.h, i, _p(u), _p(v), _p(a))
        return u.reshape(n, 3), v.reshape(n, 3), a.reshape(n, 3)

    def rom_state(self, i):
        r = self.rank[i]
        q, qd, qdd = np.zeros(r), np.zeros(r), np.zeros(r)
        lib().orc_get_rom(self.h, i, _p(q), _p(qd), _p(qdd))
        return q, qd, qdd

    def free_dofs(self, i):
        n = lib().orc_num_nodes(self.h, i)
        out = np.zeros(3 * n, np.int32)
        k = lib().orc_free_dofs(self.h, i, _p(out))
        return out[:k].copy()

    def schwarz_dofs(self, i):
        n = lib().orc_num_nodes(self.h, i)
        out = np.zeros(3 * n, np.int32)
        k = lib().orc_schwarz_dofs(self.h, i, _p(out))
        return out[:k].copy()
