"""Thin Python binding of libosam (include/osam.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  If libosam.so is missing or no usable
GPU is present the calls raise; there is no CPU fallback.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); they must be C-contiguous float64 / uint8 as documented in osam.h.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libosam.so")

OK, MAXITER, EINVAL, ECFL, ENONFINITE, EDONOR, ECUDA, ETIMEOUT, ENOMEM = 0, 1, -1, -2, -3, -4, -5, -6, -7
FOM, ROM = 0, 1
LINEAR_ELASTIC, NEO_HOOKEAN, SAINT_VENANT_KIRCHHOFF = 0, 1, 2
EXPLICIT, IMPLICIT = 0, 1
MULTIPLICATIVE, ADDITIVE = 0, 1
FP64, FP32_FORCE, F32X2_FORCE, FP64_TANGENT32 = 0, 1, 2, 3
SCATTER_AUTO, SCATTER_ATOMIC, SCATTER_GATHER, SCATTER_GATHER_LOWREG, SCATTER_GATHER_TILED = 0, 1, 2, 3, 4
SCATTER_GATHER_TILED_LOWREG = 5

EXPORTED = ["schwarz_init", "subdomain_advance", "transfer_overlap", "osam_begin_interval", "osam_restore_interval",
            "osam_criterion", "schwarz_step", "osam_get_state", "osam_set_state", "osam_get_reduced_state",
            "osam_set_reduced_state", "osam_sizes", "osam_scatter_mode", "osam_destroy", "osam_last_error",
            "osam_hex8_force", "osam_hex8_force_vjp", "opinf_fit", "osam_fit_last_error", "osam_adjoint",
            "osam_profile", "osam_profile_read", "osam_implicit_profile", "osam_fp64_peak", "osam_fp64_probe", "osam_fp64_issue_probe", "osam_hex8_force_noalloc", "osam_batch_init",
            "osam_batch_step", "osam_num_instances", "osam_instance_get_state", "osam_instance_set_state",
            "osam_instance_get_reduced_state", "osam_instance_set_reduced_state", "osam_instance_sizes",
            "osam_set_graph", "osam_tuning", "opinf_select", "osam_fit_profile"]

_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


class OsamError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"osam error {code}: {msg}")
        self.code = code


class SubdomainDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("origin", C.c_double * 3), ("material", C.c_int), ("lambda_", C.c_double), ("mu", C.c_double),
                ("rho", C.c_double), ("lambda_e", _vp), ("mu_e", _vp), ("dirichlet", _vp), ("u0", _vp), ("v0", _vp),
                ("r", C.c_int), ("r_s", C.c_int), ("Phi", _vp), ("Phi_S", _vp), ("K", _vp), ("H", _vp), ("B", _vp),
                ("c", _vp), ("integrator", C.c_int), ("n_substeps", C.c_int), ("C", _vp)]


class CouplingDesc(C.Structure):
    _fields_ = [("dst", C.c_int), ("src", C.c_int), ("nodes", _vp)]


class ProblemDesc(C.Structure):
    _fields_ = [("n_subdomains", C.c_int), ("subdomains", C.POINTER(SubdomainDesc)), ("n_couplings", C.c_int),
                ("couplings", C.POINTER(CouplingDesc)), ("dt", C.c_double), ("n_substeps", C.c_int),
                ("tol_abs", C.c_double), ("tol_rel", C.c_double), ("max_iters", C.c_int), ("precision", C.c_int),
                ("scatter", C.c_int), ("stream", _vp), ("device", C.c_int), ("schwarz", C.c_int)]


class StepReport(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("cnum", C.c_double), ("cden", C.c_double),
                ("element_updates", C.c_longlong), ("elapsed_ms", C.c_double)]


class FitInput(C.Structure):
    _fields_ = [("n_dof", C.c_int), ("n_snap", C.c_int), ("n_sdof", C.c_int), ("U", _vp), ("A", _vp), ("S", _vp),
                ("r", C.c_int), ("r_s", C.c_int), ("energy_s", C.c_double), ("r_s_max", C.c_int),
                ("lambda_", C.c_double), ("quadratic", C.c_int), ("stream", _vp), ("device", C.c_int),
                ("cubic", C.c_int)]


class FitOutput(C.Structure):
    _fields_ = [("Phi", _vp), ("Phi_S", _vp), ("K", _vp), ("H", _vp), ("B", _vp), ("c", _vp), ("sigma", _vp),
                ("sigma_s", _vp), ("r_s", C.c_int), ("C", _vp)]


class SelectInput(C.Structure):
    _fields_ = [("lambdas", _vp), ("n_lambda", C.c_int), ("v0", _vp), ("dt", C.c_double), ("substeps", C.c_int)]


class AdjointDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double), ("material", C.c_int),
                ("lambda_e", _vp), ("mu_e", _vp), ("rho", C.c_double), ("dirichlet", _vp), ("u0", _vp), ("v0", _vp),
                ("dt", C.c_double), ("n_steps", C.c_int), ("checkpoint_every", C.c_int), ("w", _vp), ("stream", _vp),
                ("device", C.c_int)]


class AdjointOut(C.Structure):
    _fields_ = [("J", C.c_double), ("grad_u0", _vp), ("grad_v0", _vp), ("grad_lambda", _vp), ("grad_mu", _vp),
                ("elapsed_ms", C.c_double)]


_lib = None


def load():
    """Load libosam.so (built in-tree by build_lib.build()); raise loudly when it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libosam.so not built ({LIB_PATH}); run paper_2511_20687_gb300.build_lib.build()")
    L = C.CDLL(LIB_PATH)
    L.schwarz_init.argtypes = [C.POINTER(ProblemDesc), C.POINTER(_vp)]
    L.subdomain_advance.argtypes = [_vp, C.c_int]
    L.transfer_overlap.argtypes = [_vp, C.c_int, C.c_int]
    L.osam_begin_interval.argtypes = [_vp]
    L.osam_restore_interval.argtypes = [_vp]
    L.osam_criterion.argtypes = [_vp, _dp, _dp]
    L.schwarz_step.argtypes = [_vp, C.POINTER(StepReport)]
    for f in ("osam_get_state", "osam_set_state", "osam_get_reduced_state", "osam_set_reduced_state"):
        getattr(L, f).argtypes = [_vp, C.c_int, _vp, _vp, _vp]
    L.osam_sizes.argtypes = [_vp, C.c_int] + [C.POINTER(C.c_int)] * 4
    L.osam_scatter_mode.argtypes = [_vp]
    L.osam_destroy.argtypes = [_vp]
    L.osam_destroy.restype = None
    L.osam_last_error.argtypes = [_vp]
    L.osam_last_error.restype = C.c_char_p
    L.osam_fit_last_error.restype = C.c_char_p
    L.osam_hex8_force.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, _vp, _vp,
                                  _vp, _vp, _vp]
    L.osam_hex8_force_vjp.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, _vp,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.opinf_fit.argtypes = [C.POINTER(FitInput), C.POINTER(FitOutput)]
    L.opinf_select.argtypes = [C.POINTER(FitInput), C.POINTER(SelectInput), _dp, C.POINTER(C.c_int),
                               C.POINTER(FitOutput)]
    L.osam_adjoint.argtypes = [C.POINTER(AdjointDesc), C.POINTER(AdjointOut)]
    L.osam_profile.argtypes = [_vp, C.c_int]
    L.osam_profile_read.argtypes = [_vp, _dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong)]
    L.osam_implicit_profile.argtypes = [_vp, _dp] + [C.POINTER(C.c_longlong)] * 4
    L.osam_fp64_peak.argtypes = [C.c_int, _dp]
    L.osam_fp64_probe.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
    L.osam_fp64_issue_probe.argtypes = [C.c_int, C.c_int, C.c_int, _dp]
    L.osam_fit_profile.argtypes = [C.c_int, _dp, _dp, C.POINTER(C.c_longlong)]
    L.osam_batch_init.argtypes = [C.c_int, C.POINTER(ProblemDesc), C.POINTER(_vp)]
    L.osam_batch_step.argtypes = [_vp, C.POINTER(StepReport), C.POINTER(StepReport)]
    L.osam_num_instances.argtypes = [_vp]
    for f in ("osam_instance_get_state", "osam_instance_set_state", "osam_instance_get_reduced_state",
              "osam_instance_set_reduced_state"):
        getattr(L, f).argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, _vp]
    L.osam_instance_sizes.argtypes = [_vp, C.c_int, C.c_int] + [C.POINTER(C.c_int)] * 4
    L.osam_set_graph.argtypes = [_vp, C.c_int]
    L.osam_tuning.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.osam_hex8_force_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                          _vp, _vp, _vp, _vp, _vp]
    _lib = L
    return L


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _f64(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.uint8).contiguous()
    return np.ascontiguousarray(a, dtype=np.uint8)


def _check(code, ctx=None):
    if code < 0:
        msg = load().osam_last_error(ctx)
        raise OsamError(code, msg.decode() if msg else "")
    return code


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


_MAT = {"le": LINEAR_ELASTIC, "nh": NEO_HOOKEAN, "svk": SAINT_VENANT_KIRCHHOFF, LINEAR_ELASTIC: LINEAR_ELASTIC,
        NEO_HOOKEAN: NEO_HOOKEAN, SAINT_VENANT_KIRCHHOFF: SAINT_VENANT_KIRCHHOFF}


class Batch:
    """n instances of one coupled O-SAM problem advanced together on the GPU (osam_batch_init).

    specs: list of workloads.Problem with identical topology; rom_ops: list (one per instance) of
    {subdomain index: {"Phi", "Phi_S", "K", "H", "B", "c"[, "C"]}} for the ROM subdomains (or None; "C"
    makes the ROM cubic).
    """

    def __init__(self, specs, rom_ops=None, precision: int = FP64, scatter: int = SCATTER_AUTO, device: int = 0,
                 stream=None, graph: bool = True):
        L = load()
        specs = list(specs)
        rom_ops = rom_ops or [None] * len(specs)
        self.specs = specs
        self._keep = []
        descs = (ProblemDesc * len(specs))()
        self.rank = {}
        for n, (spec, ops_n) in enumerate(zip(specs, rom_ops)):
            ops_n = ops_n or {}
            nsd = len(spec.subdomains)
            subs = (SubdomainDesc * nsd)()
            self._keep.append(subs)
            for i, sd in enumerate(spec.subdomains):
                d = subs[i]
                d.kind = FOM if sd.kind == "fom" else ROM
                d.nx, d.ny, d.nz = sd.dims
                d.h = sd.h
                d.origin = (C.c_double * 3)(*sd.origin)
                d.material = _MAT[sd.material]
                d.integrator = {"explicit": EXPLICIT, "implicit": IMPLICIT}[getattr(sd, "integrator", "explicit")]
                d.n_substeps = int(getattr(sd, "n_substeps", 0) or 0)
                d.lambda_, d.mu, d.rho = sd.lam, sd.mu, sd.rho
                arrs = {"lambda_e": _f64(sd.lam_e), "mu_e": _f64(sd.mu_e), "dirichlet": _u8(sd.dirichlet),
                        "u0": _f64(sd.u0), "v0": _f64(sd.v0)}
                if sd.kind == "rom":
                    ops = ops_n[i]
                    for k in ("Phi", "Phi_S", "K", "H", "B", "c"):
                        arrs[k] = _f64(ops[k])
                    if ops.get("C") is not None:
                        arrs["C"] = _f64(ops["C"])
                    d.r = int(ops["Phi"].shape[1])
                    d.r_s = int(ops["Phi_S"].shape[1])
                    self.rank[(n, i)] = d.r
                for k, a in arrs.items():
                    self._keep.append(a)
                    setattr(d, k, _ptr(a))
            cpls = (CouplingDesc * max(1, len(spec.couplings)))()
            self._keep.append(cpls)
            for k, cp in enumerate(spec.couplings):
                m = _u8(cp.nodes)
                self._keep.append(m)
                cpls[k].dst, cpls[k].src, cpls[k].nodes = cp.dst, cp.src, _ptr(m)
            desc = descs[n]
            desc.n_subdomains = nsd
            desc.subdomains = subs
            desc.n_couplings = len(spec.couplings)
            desc.couplings = cpls
            desc.dt = spec.dt
            desc.n_substeps = spec.n_substeps
            desc.tol_abs, desc.tol_rel = spec.tol_abs, spec.tol_rel
            desc.max_iters = spec.max_iters
            desc.precision = precision
            desc.scatter = scatter
            desc.stream = _stream_handle(stream)
            desc.device = device
            desc.schwarz = ADDITIVE if getattr(spec, "schwarz", "multiplicative") == "additive" else MULTIPLICATIVE
        h = _vp()
        _check(L.osam_batch_init(len(specs), descs, C.byref(h)), None)
        self.h = h
        self.n = len(specs)
        self._keep = None  # the library copied everything it needs
        if not graph:
            self._c(L.osam_set_graph(self.h, 0))

    def close(self):
        if getattr(self, "h", None):
            load().osam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, code):
        return _check(code, self.h)

    def set_graph(self, enable: bool):
        self._c(load().osam_set_graph(self.h, int(enable)))

    def step(self):
        """One controller step of every instance: (per-instance reports, aggregate report)."""
        reps = (StepReport * self.n)()
        tot = StepReport()
        rc = self._c(load().osam_batch_step(self.h, reps, C.byref(tot)))
        per = [{"status": r.status, "iterations": r.iterations, "cnum": r.cnum, "cden": r.cden,
                "element_updates": r.element_updates, "elapsed_ms": r.elapsed_ms} for r in reps]
        return per, {"status": rc, "iterations": tot.iterations, "cnum": tot.cnum, "cden": tot.cden,
                     "element_updates": tot.element_updates, "elapsed_ms": tot.elapsed_ms}

    def tuning(self):
        sc, eb, rc, tl = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._c(load().osam_tuning(self.h, C.byref(sc), C.byref(eb), C.byref(rc), C.byref(tl)))
        return {"scatter": "atomic" if sc.value == SCATTER_ATOMIC else "gather", "element_block": eb.value,
                "register_cap": rc.value, "tiled": bool(tl.value)}

    def profile(self, enable=True):
        """Start (and reset) kernel-level accounting of the internal-force launches."""
        self._c(load().osam_profile(self.h, int(enable)))

    def profile_read(self) -> dict:
        ms = C.c_double()
        fl, fe, kl = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self._c(load().osam_profile_read(self.h, C.byref(ms), C.byref(fl), C.byref(fe), C.byref(kl)))
        return {"force_ms": ms.value, "force_launches": fl.value, "force_elements": fe.value,
                "kernel_launches": kl.value}

    def implicit_profile(self) -> dict:
        """Tangent-action time / launches / elements and Newton / CG counts of the implicit subdomains
        since the last profile() call (time only while profiling is enabled)."""
        ms = C.c_double()
        v = [C.c_longlong() for _ in range(4)]
        self._c(load().osam_implicit_profile(self.h, C.byref(ms), *[C.byref(x) for x in v]))
        return {"tangent_ms": ms.value, "tangent_launches": v[0].value, "tangent_elements": v[1].value,
                "newton_steps": v[2].value, "cg_iterations": v[3].value}

    def sizes(self, i, inst=0):
        """Node, element, free-dof and Schwarz-node counts of subdomain i (fixed at initialisation, so
        asked of the library once per subdomain: its free-dof count is a pass over the masks)."""
        cache = self.__dict__.setdefault("_sizes", {})
        if (i, inst) not in cache:
            v = [C.c_int() for _ in range(4)]
            self._c(load().osam_instance_sizes(self.h, inst, i, *[C.byref(x) for x in v]))
            cache[(i, inst)] = {"n_nodes": v[0].value, "n_elements": v[1].value, "n_free": v[2].value,
                                "n_schwarz": v[3].value}
        return dict(cache[(i, inst)])

    def state(self, i, out=None, fields=(0, 1, 2), inst=0):
        """(u, v, a) of subdomain i of instance inst as [nodes, 3] arrays (numpy unless `out` arrays /
        tensors are given; fields not listed are returned as None)."""
        n = self.sizes(i, inst)["n_nodes"]
        if out is None:
            out = tuple(np.zeros((n, 3)) if f in fields else None for f in range(3))
        self._c(load().osam_instance_get_state(self.h, inst, i, *[_ptr(x) for x in out]))
        return out

    def set_state(self, i, u, v=None, a=None, inst=0):
        u, v, a = _f64(u), _f64(v), _f64(a)
        self._c(load().osam_instance_set_state(self.h, inst, i, _ptr(u), _ptr(v), _ptr(a)))

    def reduced_state(self, i, inst=0):
        r = self.rank[(inst, i)]
        outs = tuple(np.zeros(r) for _ in range(3))
        self._c(load().osam_instance_get_reduced_state(self.h, inst, i, *[_ptr(x) for x in outs]))
        return outs

    def set_reduced_state(self, i, q, qd=None, qdd=None, inst=0):
        q, qd, qdd = _f64(q), _f64(qd), _f64(qdd)
        self._c(load().osam_instance_set_reduced_state(self.h, inst, i, _ptr(q), _ptr(qd), _ptr(qdd)))


class Problem(Batch):
    """A single coupled O-SAM problem on the GPU (a batch of one), built from a workloads.Problem spec.

    rom_ops: {subdomain index: {"Phi", "Phi_S", "K", "H", "B", "c"}} for the ROM subdomains.
    """

    def __init__(self, spec, rom_ops: Optional[Dict[int, dict]] = None, precision: int = FP64,
                 scatter: int = SCATTER_AUTO, device: int = 0, stream=None, graph: bool = True):
        super().__init__([spec], [rom_ops], precision=precision, scatter=scatter, device=device, stream=stream,
                         graph=graph)
        self.spec = spec
        self.rank = {i: r for (_, i), r in self.rank.items()}

    def step(self) -> dict:
        rep = StepReport()
        rc = self._c(load().schwarz_step(self.h, C.byref(rep)))
        return {"status": rc, "iterations": rep.iterations, "cnum": rep.cnum, "cden": rep.cden,
                "element_updates": rep.element_updates, "elapsed_ms": rep.elapsed_ms}

    def reduced_state(self, i, inst=0):
        r = self.rank[i]
        outs = tuple(np.zeros(r) for _ in range(3))
        self._c(load().osam_instance_get_reduced_state(self.h, inst, i, *[_ptr(x) for x in outs]))
        return outs

    def advance(self, i):
        self._c(load().subdomain_advance(self.h, i))

    def transfer(self, src, dst):
        self._c(load().transfer_overlap(self.h, src, dst))

    def begin_interval(self):
        self._c(load().osam_begin_interval(self.h))

    def restore_interval(self):
        self._c(load().osam_restore_interval(self.h))

    def criterion(self):
        a, b = C.c_double(), C.c_double()
        self._c(load().osam_criterion(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def scatter_mode(self):
        return load().osam_scatter_mode(self.h)


# ---------------------------------------------------------------------------------------------
# element-level operators (device tensors)
# ---------------------------------------------------------------------------------------------
def hex8_force(dims, h, material, lam, mu, u, f, lam_e=None, mu_e=None, stream=None):
    """f = internal force of displacement u (both CUDA float64 tensors [nodes, 3])."""
    nx, ny, nz = dims
    _check(load().osam_hex8_force(nx, ny, nz, h, _MAT[material], lam, mu, _ptr(lam_e), _ptr(mu_e), _ptr(u), _ptr(f),
                                  _stream_handle(stream)))


def hex8_force_vjp(dims, h, material, lam, mu, u, ybar, ubar, lam_bar=None, mu_bar=None, lam_e=None, mu_e=None,
                   stream=None):
    nx, ny, nz = dims
    _check(load().osam_hex8_force_vjp(nx, ny, nz, h, _MAT[material], lam, mu, _ptr(lam_e), _ptr(mu_e), _ptr(u),
                                      _ptr(ybar), _ptr(ubar), _ptr(lam_bar), _ptr(mu_bar), _stream_handle(stream)))


# ---------------------------------------------------------------------------------------------
# offline OpInf fit
# ---------------------------------------------------------------------------------------------
def _fit_outputs(n, nsd, ns, r, rs_cols, cubic):
    out = {"Phi": np.zeros((n, r)), "Phi_S": np.zeros((max(nsd, 1), rs_cols)), "K": np.zeros((r, r)),
           "H": np.zeros((r, r * (r + 1) // 2)), "B": np.zeros((r, rs_cols)), "c": np.zeros(r),
           "sigma": np.zeros(ns), "sigma_s": np.zeros(ns)}
    if cubic:
        out["C"] = np.zeros((r, r * (r + 1) * (r + 2) // 6))
    return out


def opinf_fit(U, A, S, r, lam, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, quadratic=True, device=0, stream=None,
              cubic=False):
    """U, A: [n_snap, n_dof]; S: [n_snap, n_sdof] snapshots (host or device float64).  Returns numpy
    operators {Phi [n_dof, r], Phi_S [n_sdof, r_s], K, H, (C,) B [r, r_s], c, sigma, sigma_s, r_s}."""
    U, A, S = _f64(U), _f64(A), _f64(S)
    ns, n = U.shape
    nsd = S.shape[1] if S is not None else 0
    rs_cols = max(r_s_max, r_s)
    out_arrs = _fit_outputs(n, nsd, ns, r, rs_cols, cubic)
    fi = FitInput(n_dof=n, n_snap=ns, n_sdof=nsd, U=_ptr(U), A=_ptr(A), S=_ptr(S), r=r, r_s=r_s, energy_s=energy_s,
                  r_s_max=r_s_max, lambda_=lam, quadratic=int(quadratic), stream=_stream_handle(stream), device=device,
                  cubic=int(cubic))
    fo = FitOutput(**{k: _ptr(v) for k, v in out_arrs.items()}, r_s=0)
    rc = load().opinf_fit(C.byref(fi), C.byref(fo))
    if rc < 0:
        raise OsamError(rc, load().osam_fit_last_error().decode())
    rs = fo.r_s
    out_arrs["Phi_S"] = out_arrs["Phi_S"][:, :rs].copy()
    out_arrs["B"] = out_arrs["B"][:, :rs].copy()
    out_arrs["r_s"] = rs
    return out_arrs


def opinf_select(U, A, S, v0, r, lambdas, dt, substeps, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, quadratic=True,
                 device=0, stream=None, cubic=False):
    """Schwarz-aware regularisation selection (Algorithm 3) on the GPU.  U, A: [n_snap, n_dof];
    S: [n_snap, n_sdof]; v0: [n_dof] velocity of the first snapshot (or None); lambdas: candidates.
    Returns the operators at the selected lambda (as opinf_fit) plus "errors", "best" and "lambda"."""
    U, A, S, v0 = _f64(U), _f64(A), _f64(S), _f64(v0)
    lams = np.ascontiguousarray(lambdas, dtype=np.float64)
    ns, n = U.shape
    nsd = S.shape[1] if S is not None else 0
    rs_cols = max(r_s_max, r_s)
    out_arrs = _fit_outputs(n, nsd, ns, r, rs_cols, cubic)
    fi = FitInput(n_dof=n, n_snap=ns, n_sdof=nsd, U=_ptr(U), A=_ptr(A), S=_ptr(S), r=r, r_s=r_s, energy_s=energy_s,
                  r_s_max=r_s_max, lambda_=0.0, quadratic=int(quadratic), stream=_stream_handle(stream), device=device,
                  cubic=int(cubic))
    si = SelectInput(lambdas=lams.ctypes.data, n_lambda=len(lams), v0=_ptr(v0), dt=dt, substeps=substeps)
    fo = FitOutput(**{k: _ptr(v) for k, v in out_arrs.items()}, r_s=0)
    errors = np.zeros(len(lams))
    best = C.c_int(-1)
    rc = load().opinf_select(C.byref(fi), C.byref(si), errors.ctypes.data_as(_dp), C.byref(best), C.byref(fo))
    if rc < 0:
        raise OsamError(rc, load().osam_fit_last_error().decode())
    rs = fo.r_s
    out_arrs["Phi_S"] = out_arrs["Phi_S"][:, :rs].copy()
    out_arrs["B"] = out_arrs["B"][:, :rs].copy()
    out_arrs.update(r_s=rs, errors=errors, best=best.value, **{"lambda": float(lams[best.value])})
    return out_arrs


# ---------------------------------------------------------------------------------------------
# adjoint rollout
# ---------------------------------------------------------------------------------------------
def adjoint(dims, h, material, lam_e, mu_e, rho, dirichlet, u0, v0, dt, n_steps, w, checkpoint_every=50, device=0,
            stream=None):
    """J = w . u_T and its gradients w.r.t. u0, v0, lambda_e, mu_e (numpy outputs)."""
    nx, ny, nz = dims
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    ne = nx * ny * nz
    lam_e, mu_e, u0, v0, w = _f64(lam_e), _f64(mu_e), _f64(u0), _f64(v0), _f64(w)
    dm = _u8(dirichlet)
    d = AdjointDesc(nx=nx, ny=ny, nz=nz, h=h, material=_MAT[material], lambda_e=_ptr(lam_e), mu_e=_ptr(mu_e), rho=rho,
                    dirichlet=_ptr(dm), u0=_ptr(u0), v0=_ptr(v0), dt=dt, n_steps=n_steps,
                    checkpoint_every=checkpoint_every, w=_ptr(w), stream=_stream_handle(stream), device=device)
    gu, gv, gl, gm = np.zeros((nn, 3)), np.zeros((nn, 3)), np.zeros(ne), np.zeros(ne)
    o = AdjointOut(J=0.0, grad_u0=_ptr(gu), grad_v0=_ptr(gv), grad_lambda=_ptr(gl), grad_mu=_ptr(gm), elapsed_ms=0.0)
    rc = load().osam_adjoint(C.byref(d), C.byref(o))
    if rc < 0:
        msg = load().osam_last_error(None)
        raise OsamError(rc, msg.decode() if msg else "")
    return {"J": o.J, "grad_u0": gu, "grad_v0": gv, "grad_lambda": gl, "grad_mu": gm, "elapsed_ms": o.elapsed_ms}


def fp64_peak_gflops(device=0) -> float:
    """Measured FP64 FMA throughput of the device (GFLOP/s)."""
    g = C.c_double()
    _check(load().osam_fp64_peak(device, C.byref(g)))
    return g.value


def fp64_probe(kind=0, repeats=10, device=0):
    """FP64 throughput probe: (TFLOP/s, ms) of each of `repeats` launches; kind 0 FMA, 1 tensor-core
    MMA (m8n8k4), 2 both interleaved in the same warps."""
    t = np.zeros(repeats)
    ms = np.zeros(repeats)
    _check(load().osam_fp64_probe(device, kind, repeats, t.ctypes.data_as(_dp), ms.ctypes.data_as(_dp)))
    return t, ms


def fp64_issue_probe(warps=1, lanes=32, device=0):
    """ns per FP64 warp-instruction of one warp, one block of `warps` warps with `lanes` active lanes
    each alone on one SM."""
    ns = C.c_double()
    _check(load().osam_fp64_issue_probe(device, warps, lanes, C.byref(ns)))
    return ns.value


def fit_profile(enable: bool) -> dict:
    """Turn the accounting of the fit's GEMMs on (resetting it) or off; returns the totals so far."""
    ms, fl, n = C.c_double(), C.c_double(), C.c_longlong()
    _check(load().osam_fit_profile(int(enable), C.byref(ms), C.byref(fl), C.byref(n)))
    return {"gemm_ms": ms.value, "gemm_flops": fl.value, "gemm_launches": n.value}
