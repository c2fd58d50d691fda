"""The vectorised fine-grid tiles (128 columns, 16-byte loads) against the
general tiles of the same operators, selected with CAHN_VEC=0, through the
C ABI: every node of an apply is evaluated alike, so FP64 and FP32 applies
agree bit for bit on grids with a full and a ragged tile in x and y;
multigrid-preconditioned solves and whole steps, whose Krylov dot products
are summed in another order, agree to rounding.  Parity of the vectorised
path with the FP64 oracle is in test_gpu_parity.py and test_gpu_nutrient.py
(the 160x70 and 1024x1024 grids)."""
import os

import numpy as np
import pytest

from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu

VGRIDS = {
    "128x64": dict(nx=128, ny=64, lx=2.0, ly=1.0),
    "160x70": dict(nx=160, ny=70, lx=2.0, ly=1.0),
    "384x130": dict(nx=384, ny=130, lx=3.0, ly=1.0),
    "1024x1024": dict(nx=1024, ny=1024, lx=4.0, ly=1.0),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    binding.load()


def _with_vec(flag, fn):
    old = os.environ.get("CAHN_VEC")
    if flag is None:
        os.environ.pop("CAHN_VEC", None)
    else:
        os.environ["CAHN_VEC"] = flag
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop("CAHN_VEC", None)
        else:
            os.environ["CAHN_VEC"] = old


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def _setup(grid, nutrient=0, nutrient_bc=0, **kw):
    prm = inputs.config_small()[0].replace(**VGRIDS[grid])
    prm = prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny), nutrient=nutrient,
                      nutrient_bc=nutrient_bc, **kw)
    geo = inputs.Protrusions(h_b=0.3, centres=(0.4 * prm.lx, 0.7 * prm.lx), radius=0.15,
                             noise=1e-3, seed=4)
    state = list(inputs.initial_state(prm, geo))
    if nutrient:
        c = prm.c_bulk * (0.6 + 0.3 * inputs.random_field(prm, seed=21, lo=0.0, hi=1.0))
        state.append(c)
    return prm, state


@pytest.mark.parametrize("grid", list(VGRIDS))
@pytest.mark.parametrize("nutrient_bc", [None, 0, 1])
def test_applies_bitwise(grid, nutrient_bc):
    """cahn_apply (FP64) and cahn_apply32 (FP32) of every system: identical
    with and without the vectorised tiles."""
    import torch
    nut = nutrient_bc is not None
    prm, state = _setup(grid, nutrient=int(nut), nutrient_bc=nutrient_bc or 0,
                        precision=inputs.MIXED)
    sim = binding.Simulation([prm], [state])
    x = torch.as_tensor(inputs.random_field(prm, seed=9), device="cuda").contiguous()
    x32 = x.float()
    systems = [binding.SYS_C] if nut else [binding.SYS_PHI, binding.SYS_U, binding.SYS_P]

    def run():
        out = []
        for s in systems:
            out.append(sim.apply(0, s, x).cpu().numpy())
            y32 = torch.empty_like(x32)
            binding.cahn_apply32(sim.ctx, 0, s, x32.data_ptr(), y32.data_ptr())
            torch.cuda.synchronize()
            out.append(y32.cpu().numpy())
        return out

    vec = _with_vec(None, run)
    gen = _with_vec("0", run)
    sim.close()
    for k, (a, b) in enumerate(zip(vec, gen)):
        assert np.array_equal(a, b), (k, np.max(np.abs(a - b)))


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.MIXED])
@pytest.mark.parametrize("grid", ["160x70", "1024x1024"])
def test_mg_solves_match(grid, precision):
    """V-cycle-preconditioned solves of every system (the smoother steps with
    fused zero-guess and prolongation loads, the residual epilogues): the same
    solution to rounding, in the same number of iterations (+-1)."""
    prm, state = _setup(grid, rtol=1e-13, max_iters=4000, precision=precision)
    rhs = inputs.random_field(prm, seed=11)

    def run():
        sim = binding.Simulation([prm], [state])
        out = [sim.solve(0, s, rhs) for s in range(4)]
        res = [(x.cpu().numpy(), st["iters"][s]) for s, (x, code, st) in enumerate(out)]
        assert all(code == 0 for _, code, _ in out)
        sim.close()
        return res

    vec = _with_vec(None, run)
    gen = _with_vec("0", run)
    for s, ((xa, ia), (xb, ib)) in enumerate(zip(vec, gen)):
        assert rel(xa, xb) <= 1e-11, (s, rel(xa, xb))
        assert abs(ia - ib) <= 1, (s, ia, ib)


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.MIXED])
def test_steps_match(precision):
    """Five graph-mode steps of a 384x130 instance with the nutrient on."""
    prm, state = _setup("384x130", nutrient=1, rtol=1e-12, precision=precision, use_graph=1,
                        dt=2e-4)

    def run():
        sim = binding.Simulation([prm], [state])
        sim.step(5)
        out = sim.numpy(0)
        sim.close()
        return out

    vec = _with_vec(None, run)
    gen = _with_vec("0", run)
    for name, a, b in zip(("phi", "u", "v", "p", "c"), vec, gen):
        assert rel(a, b) <= 1e-10, (name, rel(a, b))


@pytest.mark.parametrize("system", ["phi", "u", "p"])
def test_smooth32_step(system):
    """cahn_smooth32, step k of the FP32 fine-level smoother: y - x = d' and
    d' = c1 d + c2 D^-1 (b - A x) with one pair (c1, c2) for the whole grid
    (c1 = 0 at k = 0); D is the operator's diagonal, from the oracle's
    probing (phi) or its closed form (5-point rows); the predictor's wall rows
    of y are zero."""
    import torch
    from oracle import cahn_oracle as O
    prm, state = _setup("160x70", precision=inputs.MIXED)
    sysid = {"phi": binding.SYS_PHI, "u": binding.SYS_U, "p": binding.SYS_P}[system]
    sim = binding.Simulation([prm], [state])
    g = O.grid_of(prm)
    if system == "phi":
        a, _ = O.ch_coefficient(prm, O.init_state(prm, *state))
        D = O.probe_diagonal(lambda v: O.ch_apply(prm, g, a, v), g.shape)
    elif system == "u":
        D = O.probe_diagonal(lambda v: O.helm_apply(prm, g, v), g.shape, radius=1)
    else:
        D = O.probe_diagonal(lambda v: O.lap(g, v), g.shape, radius=1)
    dev = lambda f: torch.as_tensor(f, dtype=torch.float32, device="cuda").contiguous()
    x = dev(inputs.random_field(prm, seed=31))
    b = dev(inputs.random_field(prm, seed=32))
    d0 = inputs.random_field(prm, seed=33)
    ax = torch.empty_like(x)
    binding.cahn_apply32(sim.ctx, 0, sysid, x.data_ptr(), ax.data_ptr())
    rows = slice(1, -1) if system == "u" else slice(None)
    for k in (0, 2):
        d = dev(d0)
        y = torch.empty_like(x)
        binding.cahn_smooth32(sim.ctx, 0, sysid, k, x.data_ptr(), b.data_ptr(), d.data_ptr(),
                              y.data_ptr())
        torch.cuda.synchronize()
        yn, xn, dn = (t.cpu().numpy().astype(np.float64) for t in (y, x, d))
        r = (b - ax).cpu().numpy().astype(np.float64)
        step = (yn - xn)[rows]
        assert np.max(np.abs(step - dn[rows])) <= 1e-6 * np.max(np.abs(yn)), k
        z = (r / D)[rows]
        cols = [z.ravel()] if k == 0 else [z.ravel(), d0[rows].ravel()]
        coef, *_ = np.linalg.lstsq(np.stack(cols, 1), step.ravel(), rcond=None)
        fit = np.stack(cols, 1) @ coef
        assert np.linalg.norm(fit - step.ravel()) <= 1e-5 * np.linalg.norm(step), (k, coef)
        assert coef[0] > 0
        if system == "u":
            assert np.all(yn[[0, -1]] == 0.0)
    sim.close()
