"""Thin ctypes binding of the C ABI declared in include/cahn.h.

Argument marshalling only: every step of the solver runs in libcahn.so's
CUDA kernels.  There is no CPU path; if the library is missing or fails to
load, `load()` raises.

The functions take raw device pointers (ints, e.g. `tensor.data_ptr()` of
contiguous float64 CUDA tensors of shape [ny+1, nx]) and a CUDA stream
handle (e.g. `torch.cuda.current_stream().cuda_stream`).
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcahn.so")

CAHN_OK = 0
CAHN_ERR_ARG = -1
CAHN_ERR_CUDA = -2
CAHN_ERR_NOMEM = -3
CAHN_ERR_DOMAIN = -4
CAHN_ERR_NAN = -5
CAHN_ERR_NOT_CONVERGED = -6
SYS_PHI, SYS_U, SYS_V, SYS_P, SYS_C = 0, 1, 2, 3, 4
SYS_UV = 5      # the coupled momentum system (stacked [u; v]; statistics in the U slot)
MOM_SPLIT, MOM_IMPLICIT = 0, 1
NSYS = 5
PC_MG, PC_JACOBI, PC_SCHWARZ = 0, 1, 2

_I32, _I64, _F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class cahn_params(ctypes.Structure):
    _fields_ = [
        ("nx", _I32), ("ny", _I32), ("lx", _F64), ("ly", _F64), ("eps", _F64),
        ("mobility", _F64), ("chi", _F64), ("n_poly", _F64), ("stab_s", _F64),
        ("eta_water", _F64), ("eta_biofilm", _F64), ("rho_water", _F64),
        ("rho_biofilm", _F64), ("gamma_cap", _F64), ("flow_mode", _I32),
        ("u_max", _F64), ("dt", _F64), ("precision", _I32), ("krylov", _I32),
        ("restart", _I32), ("mg_levels", _I32), ("max_iters", _I32), ("rtol", _F64),
        ("energy", _I32), ("gamma2", _F64), ("precond", _I32), ("use_graph", _I32),
        ("nutrient", _I32), ("diff_s", _F64), ("growth_mu", _F64), ("growth_kc", _F64),
        ("growth_eps", _F64), ("consume_a", _F64), ("c_bulk", _F64), ("nutrient_bc", _I32),
        ("momentum", _I32),
    ]


class cahn_stats(ctypes.Structure):
    _fields_ = [
        ("steps", _I64), ("iters", _I32 * NSYS), ("outer", _I32 * NSYS), ("resid", _F64 * NSYS),
        ("mass_drift", _F64), ("failed_system", _I32), ("status", _I32),
    ]

    def as_dict(self):
        return {"steps": self.steps, "iters": list(self.iters), "outer": list(self.outer),
                "resid": list(self.resid), "mass_drift": self.mass_drift,
                "failed_system": self.failed_system, "status": self.status}


# the functions the header declares, with their ctypes signatures
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "cahn_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _I32,
                                 ctypes.POINTER(cahn_params), _PP, _PP, _PP, _PP,
                                 ctypes.c_void_p]),
    "cahn_step": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.POINTER(cahn_stats)]),
    "cahn_step_host": (ctypes.c_int, [ctypes.c_void_p, _I32, _PP, _PP, _PP, _PP,
                                      ctypes.POINTER(cahn_stats)]),
    "cahn_solve": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.POINTER(cahn_stats)]),
    "cahn_apply": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, ctypes.c_void_p, ctypes.c_void_p]),
    "cahn_apply32": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, ctypes.c_void_p, ctypes.c_void_p]),
    "cahn_mg_down32": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "cahn_smooth32": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, _I32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cahn_vjp": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, _I32, _I32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(_F64), ctypes.POINTER(cahn_stats)]),
    "cahn_solve_p_noalloc": (ctypes.c_int, [_I32, _I32, _F64, _F64, _F64, _I32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(cahn_stats)]),
    "cahn_noalloc_last_error": (ctypes.c_char_p, []),
    "cahn_lap5_coarse_inverse": (ctypes.c_int, [_I32, _I32, _I32, _F64, _F64, _F64,
                                                ctypes.c_void_p]),
    "cahn_get_history": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(_F64)]),
    "cahn_set_history": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, _F64]),
    "cahn_attach_nutrient": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "cahn_get_nutrient_history": (ctypes.c_int, [ctypes.c_void_p, _I32, ctypes.c_void_p]),
    "cahn_tile_height": (ctypes.c_int, [ctypes.c_void_p, _I32, _I32, _I32]),
    "cahn_free": (ctypes.c_int, [ctypes.c_void_p]),
    "cahn_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "cahn_abi_version": (ctypes.c_int, []),
    "cahn_last_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
}

_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libcahn.so (build it first with `build()`); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class CahnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def make_params(prm: "inputs.Params", precond: int = PC_JACOBI, use_graph: int = 0) -> cahn_params:
    q = cahn_params()
    for name, _ in cahn_params._fields_:
        if name == "precond":
            q.precond = getattr(prm, "precond", precond)
        elif name == "use_graph":
            q.use_graph = getattr(prm, "use_graph", use_graph)
        else:
            setattr(q, name, getattr(prm, name))
    return q


def _ptr_array(ptrs: Sequence[int]):
    arr = (ctypes.c_void_p * len(ptrs))()
    for k, p in enumerate(ptrs):
        arr[k] = p
    return arr


def cahn_init(params: Sequence[cahn_params], phi: Sequence[int], u: Sequence[int],
              v: Sequence[int], p: Sequence[int], stream: int = 0) -> int:
    lib = load()
    n = len(params)
    parr = (cahn_params * n)(*params)
    ctx = ctypes.c_void_p()
    code = lib.cahn_init(ctypes.byref(ctx), n, parr, _ptr_array(phi), _ptr_array(u),
                         _ptr_array(v), _ptr_array(p), ctypes.c_void_p(stream))
    if code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(None).decode())
    return ctx.value


def cahn_step(ctx: int, nsteps: int, batch: int = 1, check: bool = True):
    lib = load()
    st = (cahn_stats * batch)()
    code = lib.cahn_step(ctypes.c_void_p(ctx), nsteps, st)
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code, [s.as_dict() for s in st]


def cahn_step_host(ctx: int, nsteps: int, phi: Sequence[int], u: Sequence[int],
                   v: Sequence[int], p: Sequence[int], check: bool = True):
    lib = load()
    st = (cahn_stats * len(phi))()
    code = lib.cahn_step_host(ctypes.c_void_p(ctx), nsteps, _ptr_array(phi), _ptr_array(u),
                              _ptr_array(v), _ptr_array(p), st)
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code, [s.as_dict() for s in st]


def cahn_solve(ctx: int, instance: int, system: int, rhs: int, x: int, check: bool = True):
    lib = load()
    st = cahn_stats()
    code = lib.cahn_solve(ctypes.c_void_p(ctx), instance, system, ctypes.c_void_p(rhs),
                          ctypes.c_void_p(x), ctypes.byref(st))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code, st.as_dict()


def cahn_apply(ctx: int, instance: int, system: int, x: int, y: int, check: bool = True) -> int:
    lib = load()
    code = lib.cahn_apply(ctypes.c_void_p(ctx), instance, system, ctypes.c_void_p(x),
                          ctypes.c_void_p(y))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_vjp(ctx: int, instance: int, phi0: int, u0: int, v0: int, p0: int, nsteps: int,
             checkpoint: int, phiN_bar: int, phi0_bar: int, check: bool = True):
    """Adjoint of nsteps steps (see include/cahn.h): writes dJ/dphi0 into
    phi0_bar and returns (code, (dJ/dchi, dJ/dM), stats)."""
    lib = load()
    st = cahn_stats()
    theta = (_F64 * 2)()
    code = lib.cahn_vjp(ctypes.c_void_p(ctx), instance, ctypes.c_void_p(phi0), ctypes.c_void_p(u0),
                        ctypes.c_void_p(v0), ctypes.c_void_p(p0), nsteps, checkpoint,
                        ctypes.c_void_p(phiN_bar), ctypes.c_void_p(phi0_bar), theta,
                        ctypes.byref(st))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code, (theta[0], theta[1]), st.as_dict()


def cahn_solve_p_noalloc(nx: int, ny: int, lx: float, ly: float, rtol: float, max_iters: int,
                         rhs: int, x: int, stream: int = 0, check: bool = True):
    """The allocation-free pressure solve (see include/cahn.h)."""
    lib = load()
    st = cahn_stats()
    code = lib.cahn_solve_p_noalloc(nx, ny, lx, ly, rtol, max_iters, ctypes.c_void_p(rhs),
                                    ctypes.c_void_p(x), ctypes.c_void_p(stream), ctypes.byref(st))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_noalloc_last_error().decode())
    return code, st.as_dict()


def cahn_lap5_coarse_inverse(nx: int, ny: int, walls: int, c0: float, cx: float, cy: float,
                             check: bool = True):
    """The dense coarsest-level solve P of a constant-coefficient 5-point
    operator (host only; see include/cahn.h): returns (code, P) with P an
    (n, n) float64 array, n = nx (ny + 1)."""
    import numpy as np
    lib = load()
    n = nx * (ny + 1)
    P = np.zeros((n, n) if n <= 4096 and n > 0 else (1, 1), dtype=np.float64)
    code = lib.cahn_lap5_coarse_inverse(nx, ny, walls, c0, cx, cy,
                                        ctypes.c_void_p(P.ctypes.data))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(None).decode())
    return code, P


def cahn_smooth32(ctx: int, instance: int, system: int, k: int, x: int, b: int, d: int, y: int,
                  check: bool = True) -> int:
    """Step k of the system's FP32 fine-level smoother (device pointers)."""
    lib = load()
    code = lib.cahn_smooth32(ctypes.c_void_p(ctx), instance, system, k, ctypes.c_void_p(x),
                             ctypes.c_void_p(b), ctypes.c_void_p(d), ctypes.c_void_p(y))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_mg_down32(ctx: int, instance: int, system: int, b: int, x: int,
                   check: bool = True) -> int:
    """The V-cycle's first pass on the fine grid of a 5-point system: the
    pre-smoothing steps from x = 0 and the restricted residual (device
    pointers)."""
    lib = load()
    code = lib.cahn_mg_down32(ctypes.c_void_p(ctx), instance, system, ctypes.c_void_p(b),
                              ctypes.c_void_p(x))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_apply32(ctx: int, instance: int, system: int, x: int, y: int, check: bool = True) -> int:
    lib = load()
    code = lib.cahn_apply32(ctypes.c_void_p(ctx), instance, system, ctypes.c_void_p(x),
                            ctypes.c_void_p(y))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_get_history(ctx: int, instance: int, phi_prev: int, u_prev: int, v_prev: int,
                     check: bool = True):
    """Copy the previous levels into the given device arrays; returns (code, m0)."""
    lib = load()
    m0 = _F64()
    code = lib.cahn_get_history(ctypes.c_void_p(ctx), instance, ctypes.c_void_p(phi_prev),
                                ctypes.c_void_p(u_prev), ctypes.c_void_p(v_prev), ctypes.byref(m0))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code, m0.value


def cahn_set_history(ctx: int, instance: int, phi_prev: int, u_prev: int, v_prev: int,
                     m0: float, check: bool = True) -> int:
    lib = load()
    code = lib.cahn_set_history(ctypes.c_void_p(ctx), instance, ctypes.c_void_p(phi_prev),
                                ctypes.c_void_p(u_prev), ctypes.c_void_p(v_prev), m0)
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_attach_nutrient(ctx: int, instance: int, c: int, c_prev: int = 0,
                         check: bool = True) -> int:
    """Register the device nutrient array c (and optionally c^{n-1})."""
    lib = load()
    code = lib.cahn_attach_nutrient(ctypes.c_void_p(ctx), instance, ctypes.c_void_p(c),
                                    ctypes.c_void_p(c_prev or None))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_get_nutrient_history(ctx: int, instance: int, c_prev: int, check: bool = True) -> int:
    lib = load()
    code = lib.cahn_get_nutrient_history(ctypes.c_void_p(ctx), instance, ctypes.c_void_p(c_prev))
    if check and code != CAHN_OK:
        raise CahnError(code, lib.cahn_last_error(ctypes.c_void_p(ctx)).decode())
    return code


def cahn_tile_height(ctx: int, instance: int, system: int, level: int) -> int:
    return load().cahn_tile_height(ctypes.c_void_p(ctx), instance, system, level)


def tile_heights(ctx: int, instance: int = 0) -> dict:
    """{system name: [tile height per multigrid level]} chosen by the tuner."""
    out = {}
    for name, sysid in (("phi", SYS_PHI), ("u", SYS_U), ("v", SYS_V), ("p", SYS_P),
                        ("c", SYS_C)):
        hs = []
        while True:
            h = cahn_tile_height(ctx, instance, sysid, len(hs))
            if h < 0:
                break
            hs.append(h)
        if hs or sysid != SYS_C:
            out[name] = hs
    return out


def cahn_free(ctx: int) -> int:
    return load().cahn_free(ctypes.c_void_p(ctx))


def cahn_last_error(ctx: Optional[int]) -> str:
    return load().cahn_last_error(ctypes.c_void_p(ctx) if ctx else None).decode()


def cahn_abi_version() -> int:
    return load().cahn_abi_version()


def cahn_last_launch_count(ctx: int) -> int:
    return load().cahn_last_launch_count(ctypes.c_void_p(ctx))


# --------------------------------------------------------------------------
class Simulation:
    """Convenience owner of the device state (torch float64 CUDA tensors) of
    one or more instances plus their library context.  A state is (phi, u,
    v, p), or (phi, u, v, p, c) for an instance with the nutrient on (c
    defaults to the bulk value everywhere)."""

    def __init__(self, prms: List["inputs.Params"], states, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.prms = prms
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.fields = []
        for q, st in zip(prms, states):
            st = list(st)
            if getattr(q, "nutrient", 0) and len(st) == 4:
                st.append(inputs.initial_nutrient(q))
            self.fields.append([torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous()
                                for a in st])
        ptr = lambda k: [f[k].data_ptr() for f in self.fields]
        torch.cuda.synchronize(self.device)
        self.ctx = cahn_init([make_params(q) for q in prms], ptr(0), ptr(1), ptr(2), ptr(3),
                             self.stream.cuda_stream)
        for k, f in enumerate(self.fields):
            if len(f) == 5:
                cahn_attach_nutrient(self.ctx, k, f[4].data_ptr())

    def step(self, nsteps: int, check: bool = True):
        return cahn_step(self.ctx, nsteps, len(self.fields), check=check)

    def solve(self, instance: int, system: int, rhs, x0=None, check: bool = True):
        torch = self.torch
        b = torch.as_tensor(rhs, dtype=torch.float64).to(self.device).contiguous()
        x = (torch.zeros_like(b) if x0 is None   # SYS_UV: stacked [2 (ny+1), nx]
             else torch.as_tensor(x0, dtype=torch.float64).to(self.device).contiguous())
        torch.cuda.synchronize(self.device)
        code, st = cahn_solve(self.ctx, instance, system, b.data_ptr(), x.data_ptr(), check=check)
        return x, code, st

    def apply(self, instance: int, system: int, x):
        torch = self.torch
        xt = torch.as_tensor(x, dtype=torch.float64).to(self.device).contiguous()
        y = torch.empty_like(xt)
        cahn_apply(self.ctx, instance, system, xt.data_ptr(), y.data_ptr())
        torch.cuda.synchronize(self.device)
        return y

    def vjp(self, instance: int, phi0, u0, v0, p0, nsteps: int, checkpoint: int, phiN_bar,
            check: bool = True):
        """(dJ/dphi0 tensor, (dJ/dchi, dJ/dM), stats) of nsteps steps from a
        fresh start at (phi0, u0, v0, p0), for dJ/dphi^N = phiN_bar."""
        torch = self.torch
        dev = lambda a: torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous()
        ins = [dev(a) for a in (phi0, u0, v0, p0, phiN_bar)]
        out = torch.empty_like(ins[0])
        torch.cuda.synchronize(self.device)
        code, theta, st = cahn_vjp(self.ctx, instance, *[t.data_ptr() for t in ins[:4]], nsteps,
                                   checkpoint, ins[4].data_ptr(), out.data_ptr(), check=check)
        return out, theta, st

    def checkpoint(self, instance: int = 0):
        """The full state of an instance (host arrays): phi, u, v, p [, c],
        the previous levels phi^-, u^-, v^- [, c^-] and m0 (the mass
        target)."""
        torch = self.torch
        prev = [torch.empty_like(self.fields[instance][0]) for _ in range(3)]
        torch.cuda.synchronize(self.device)
        _, m0 = cahn_get_history(self.ctx, instance, *[t.data_ptr() for t in prev])
        if len(self.fields[instance]) == 5:
            cp = torch.empty_like(self.fields[instance][0])
            cahn_get_nutrient_history(self.ctx, instance, cp.data_ptr())
            prev.append(cp)
        return {"fields": self.numpy(instance), "prev": [t.cpu().numpy() for t in prev], "m0": m0}

    def resume(self, instance: int, ckpt):
        """Install a checkpoint's previous levels and m0 (the context must
        have been created from the checkpoint's fields)."""
        torch = self.torch
        prev = [torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous()
                for a in ckpt["prev"]]
        torch.cuda.synchronize(self.device)
        cahn_set_history(self.ctx, instance, *[t.data_ptr() for t in prev[:3]], ckpt["m0"])
        if len(prev) == 4:
            f = self.fields[instance]
            cahn_attach_nutrient(self.ctx, instance, f[4].data_ptr(), prev[3].data_ptr())
            torch.cuda.synchronize(self.device)

    def numpy(self, instance: int = 0):
        return [f.cpu().numpy() for f in self.fields[instance]]

    def close(self):
        if self.ctx:
            cahn_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
