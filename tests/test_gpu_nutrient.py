"""GPU parity of the nutrient transport and network production (Eq. 2.5-2.7)
through the C ABI against the FP64 CPU oracle: the nutrient operator
(FP64 and FP32), single solves, whole steps in host-loop, graph and batched
graph mode, FP64 and mixed precision, checkpoint/resume and the argument
checks, for both wall conditions (zero flux on both walls, the default;
c = c_bulk on the top wall).  FP64 bar: relative L2 error <= 1e-10 per
field."""
import dataclasses

import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-6
NAMES = ("phi", "u", "v", "p", "c")
BCS = {"flux": O.NUT_BC_ZERO_FLUX, "top": O.NUT_BC_BULK_TOP}

GRIDS = {
    "64x64": dict(nx=64, ny=64, lx=2.0, ly=1.0),
    "40x22": dict(nx=40, ny=22, lx=2.0, ly=1.0),     # ragged tiles in x and y
    "4x4": dict(nx=4, ny=4, lx=2.0, ly=1.0),         # smaller than one tile
    "96x130": dict(nx=96, ny=130, lx=1.0, ly=1.0),   # dy < dx, 5 tile rows
    # the vectorised 128-column tiles: one full and one ragged tile in x,
    # ragged 16- and 8-row tiles in y
    "160x70": dict(nx=160, ny=70, lx=2.0, ly=1.0),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    binding.load()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def _prm(grid="64x64", **kw):
    prm = inputs.config_nutrient()[0].replace(**GRIDS[grid])
    return prm.replace(eps=max(prm.eps, 2 * prm.ly / prm.ny), **kw)


def _state(prm, seed=3):
    geo = inputs.Protrusions(h_b=0.3, centres=(0.5 * prm.lx,), radius=0.2 * prm.ly,
                             noise=1e-3, seed=seed)
    phi, u, v, p = inputs.initial_state(prm, geo)
    # a nutrient field with structure in x and y (c_bulk on the top wall)
    c = prm.c_bulk * (0.6 + 0.3 * inputs.random_field(prm, seed=21, lo=0.0, hi=1.0))
    c[-1] = prm.c_bulk
    return phi, u, v, p, c


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("grid", list(GRIDS) + ["1024x1024"])
def test_nutrient_apply_parity(grid, bc):
    """K x through cahn_apply (FP64) and cahn_apply32 (FP32 shadow) against
    the oracle's operator with phi^{n+1} = phi^n = phi, elementwise."""
    import torch
    if grid == "1024x1024":
        prm, geo, _ = inputs.config_large()
        prm = prm.replace(nutrient=1, nutrient_bc=BCS[bc])
        phi, u, v, p = inputs.initial_state(prm, geo)
        state = (phi, u, v, p, inputs.initial_nutrient(prm))
    else:
        prm = _prm(grid, dt=1e-3, nutrient_bc=BCS[bc])
        state = _state(prm)
    g = O.grid_of(prm)
    x = inputs.random_field(prm, seed=9)
    ref = O.nut_apply(prm, g, state[0], state[0], x)
    scale = np.max(np.abs(ref))
    sim = binding.Simulation([prm], [state])
    y = sim.apply(0, binding.SYS_C, x).cpu().numpy()
    sim.close()
    assert np.max(np.abs(y - ref)) <= 1e-13 * scale, np.max(np.abs(y - ref)) / scale
    sim = binding.Simulation([prm.replace(precision=inputs.MIXED)], [state])
    x32 = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    y32 = torch.empty_like(x32)
    torch.cuda.synchronize()
    binding.cahn_apply32(sim.ctx, 0, binding.SYS_C, x32.data_ptr(), y32.data_ptr())
    torch.cuda.synchronize()
    sim.close()
    err = np.max(np.abs(y32.cpu().numpy().astype(np.float64) - ref)) / scale
    assert err <= 2e-6, err


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("pc", ["mg", "jacobi"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", list(GRIDS))
def test_nutrient_solve_parity(grid, precision, pc, bc):
    prm = _prm(grid, rtol=1e-13, max_iters=20000, dt=1e-3, precond=0 if pc == "mg" else 1,
               precision=inputs.MIXED if precision == "mixed" else inputs.FP64,
               nutrient_bc=BCS[bc])
    state = _state(prm)
    rhs = inputs.random_field(prm, seed=11)
    sim = binding.Simulation([prm], [state])
    x, code, st = sim.solve(0, binding.SYS_C, rhs)
    heights = binding.tile_heights(sim.ctx)
    sim.close()
    assert code == 0, st
    assert st["iters"][binding.SYS_C] > 0
    if pc == "mg":   # the V-cycle must actually precondition (per refinement sweep)
        assert len(heights["c"]) >= 2 or grid == "4x4", heights
        assert st["iters"][binding.SYS_C] <= 40 * max(1, st["outer"][binding.SYS_C]), st
    ref = O.solve_system(prm, O.init_state(prm, *state), "c", rhs)
    assert rel(x.cpu().numpy(), ref) <= TOL_FP64, rel(x.cpu().numpy(), ref)
    if bc == "top":
        np.testing.assert_allclose(x.cpu().numpy()[-1], rhs[-1] * prm.dt, rtol=1e-15)


def _run_both(prm, state, nsteps):
    sim = binding.Simulation([prm], [state])
    _, st = sim.step(nsteps)
    got = sim.numpy(0)
    prev = [sim.torch.empty_like(sim.fields[0][0]) for _ in range(3)]
    _, m_gpu = binding.cahn_get_history(sim.ctx, 0, *[t.data_ptr() for t in prev])
    sim.close()
    ref = O.run(prm, *state[:4], nsteps, c0=state[4])
    return got, ref, st[0], m_gpu


def _check(got, ref, tol):
    for name, g, r in zip(NAMES, got, (ref.phi, ref.u, ref.v, ref.p, ref.c)):
        assert rel(g, r) <= tol, (name, rel(g, r))


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("mode", ["host", "graph"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nutrient_step_parity_20_steps(precision, mode, bc):
    """The 64^2 workload with the nutrient at the paper's D_s, mu, K_c, A:
    every field (c included) and the grown mass target against the oracle."""
    prm, geo, nsteps = inputs.config_nutrient()
    prm = prm.replace(use_graph=1 if mode == "graph" else 0, nutrient_bc=BCS[bc])
    if precision == "mixed":
        prm = prm.replace(precision=inputs.MIXED, rtol=1e-10)
    phi, u, v, p = inputs.initial_state(prm, geo)
    state = (phi, u, v, p, inputs.initial_nutrient(prm))
    got, ref, st, m_gpu = _run_both(prm, state, nsteps)
    _check(got, ref, TOL_FP64)
    assert st["iters"][binding.SYS_C] >= nsteps
    assert abs(m_gpu - ref.m0) <= 1e-12 * abs(ref.m0)
    assert ref.m0 > O.mass(O.grid_of(prm), phi)   # the production grew the mass
    assert abs(st["mass_drift"]) < 1e-9


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("grid", ["40x22", "96x130"])
def test_nutrient_step_parity_ragged(grid, bc):
    prm = _prm(grid, precond=1, rtol=1e-13, nutrient_bc=BCS[bc])
    state = _state(prm, seed=4)
    got, ref, _, _ = _run_both(prm, state, 6)
    _check(got, ref, TOL_FP64)


def test_nutrient_batch_graph_beside_a_plain_instance():
    """One batched graph advancing a nutrient instance and a plain one
    (refinement to the FP64 tolerance, so the FP64 bar applies)."""
    prm_n = _prm("64x64", use_graph=1, precision=inputs.MIXED, rtol=1e-12)
    prm_p = inputs.config_small()[0].replace(nx=40, ny=22, eps=2 / 22, use_graph=1,
                                             precision=inputs.MIXED, rtol=1e-12)
    st_n = _state(prm_n)
    st_p = _state(prm_p)[:4]
    sim = binding.Simulation([prm_n, prm_p], [st_n, st_p])
    _, stats = sim.step(8)
    got_n, got_p = sim.numpy(0), sim.numpy(1)
    sim.close()
    assert len(got_n) == 5 and len(got_p) == 4
    ref_n = O.run(prm_n, *st_n[:4], 8, c0=st_n[4])
    ref_p = O.run(prm_p, *st_p, 8)
    _check(got_n, ref_n, TOL_FP64)
    for name, g, r in zip(NAMES, got_p, (ref_p.phi, ref_p.u, ref_p.v, ref_p.p)):
        assert rel(g, r) <= TOL_FP64, (name, rel(g, r))
    assert stats[1]["iters"][binding.SYS_C] == 0


@pytest.mark.parametrize("mode", ["host", "graph"])
def test_nutrient_checkpoint_resume_is_exact(mode):
    """Steps 1..10 in one go equal steps 1..5, a checkpoint (c^{n-1} and the
    mass target included), a fresh context and steps 6..10, bit for bit."""
    prm = _prm("64x64", use_graph=1 if mode == "graph" else 0)
    state = _state(prm)
    a = binding.Simulation([prm], [state])
    a.step(10)
    want = a.numpy(0)
    a.close()
    b = binding.Simulation([prm], [state])
    b.step(5)
    ck = b.checkpoint(0)
    b.close()
    assert len(ck["prev"]) == 4
    c = binding.Simulation([prm], [tuple(ck["fields"])])
    c.resume(0, ck)
    c.step(5)
    got = c.numpy(0)
    c.close()
    for name, g, w in zip(NAMES, got, want):
        assert np.array_equal(g, w), name


def test_nutrient_argument_checks():
    import torch
    prm = _prm("64x64")
    phi, u, v, p, _ = _state(prm)
    t = [torch.as_tensor(f, device="cuda").contiguous() for f in (phi, u, v, p)]
    torch.cuda.synchronize()
    ctx = binding.cahn_init([binding.make_params(prm)], *[[f.data_ptr()] for f in t])
    try:
        code, _ = binding.cahn_step(ctx, 1, check=False)
        assert code == binding.CAHN_ERR_ARG          # no c registered
        assert "nutrient" in binding.cahn_last_error(ctx)
    finally:
        binding.cahn_free(ctx)
    plain = inputs.config_small()[0]
    sim = binding.Simulation([plain], [_state(plain)[:4]])
    _, code, _ = sim.solve(0, binding.SYS_C, np.zeros((plain.ny + 1, plain.nx)), check=False)
    assert code == binding.CAHN_ERR_ARG
    assert binding.cahn_attach_nutrient(sim.ctx, 0, t[0].data_ptr(), check=False) == \
        binding.CAHN_ERR_ARG
    sim.close()
    sim = binding.Simulation([prm], [_state(prm)])
    f = sim.fields[0]
    out = torch.empty_like(f[0])
    torch.cuda.synchronize()
    code, _, _ = binding.cahn_vjp(sim.ctx, 0, f[0].data_ptr(), f[1].data_ptr(), f[2].data_ptr(),
                                  f[3].data_ptr(), 1, 1, f[0].data_ptr(), out.data_ptr(),
                                  check=False)
    assert code == binding.CAHN_ERR_ARG
    sim.close()


@pytest.mark.parametrize("mode", ["host", "graph"])
def test_nutrient_domain_error_when_phi_reaches_one(mode):
    """A mass target that the correction reaches only with phi^{n+1} > 1: the
    step stops with CAHN_ERR_DOMAIN on the nutrient system before its solve
    (the solvent fraction 1 - phi vanishes, Eq. 2.6), leaves every field at
    its start value, and the oracle raises its domain error on the same
    state; a reachable target steps."""
    prm = inputs.config_nutrient()[0].replace(nx=16, ny=12, eps=0.2, dt=1e-4,
                                              use_graph=1 if mode == "graph" else 0)
    g = O.grid_of(prm)
    rng = np.random.default_rng(7)
    phi = 0.9995 + 1e-5 * rng.random(g.shape)
    z = np.zeros(g.shape)
    state = (phi, z, z.copy(), z.copy(), np.ones(g.shape))
    sw = float(np.sum(g.w))
    st0 = O.init_state(prm, *state)
    for shift, fails in ((2e-4, False), (2e-3, True)):
        sim = binding.Simulation([prm], [state])
        ck = sim.checkpoint(0)
        ck["m0"] = st0.m0 + shift * sw
        sim.resume(0, ck)
        code, st = sim.step(1, check=False)
        got = sim.numpy(0)
        sim.close()
        if fails:
            assert code == binding.CAHN_ERR_DOMAIN, code
            assert st[0]["failed_system"] == binding.SYS_C and st[0]["steps"] == 0, st[0]
            for a, b in zip(got, state):
                assert np.array_equal(a, b)
            with pytest.raises(O.DomainError):
                O.step(prm, dataclasses.replace(st0, m0=ck["m0"]))
        else:
            assert code == binding.CAHN_OK, code
            ref = O.step(prm, dataclasses.replace(st0, m0=ck["m0"]))
            assert rel(got[0], ref.phi) <= TOL_FP64 and rel(got[4], ref.c) <= TOL_FP64
