"""GPU discrete adjoint (cahn_vjp and the torch.autograd.Function over it)
against the oracle's FP64 adjoint on small grids, and against central
finite differences of the GPU forward at 256 x 256 (50 steps, checkpoints
every 10).

Tolerances.  Against the oracle: both sides solve every system to ~1e-13
relative residual (the oracle's adjoint solves are dense, exact), and the
step maps are well conditioned (A_phi is dominated by I/dt), so the
gradients agree to ~1e-11; the test asserts 1e-8.  Against central
differences with h = 1e-6 relative: truncation O(h^2) and rounding of the
forward ~1e-16 / (h |dJ/dtheta| / |J|); the bar is 1e-5 relative.  On the
256^2 workload J is the volume above y = 0.25 after 50 steps of 2.5e-5, and
its sensitivity to chi is |dJ/dchi| / |J| ~ 5e-8: with h = 1e-6 chi the
difference J(chi + h) - J(chi - h) is ~5e-14, about 2000 units in the last
place of J (~0.22), so one ulp of rounding in either value is a 5e-4 error
of the difference (measured: 5.1e-4 for chi).  chi and M are therefore
checked with Richardson-extrapolated central differences at h = 1e-2 theta
and h / 2 (error O(h^4) ~ 1e-8, rounding ~1e-7); the phi0 direction keeps
h = 1e-6 (there the difference is ~1e-8, far above rounding)."""
import numpy as np
import pytest

from oracle import cahn_adjoint as A
from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-8
TOL_FD = 1e-5


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


def _small(**kw):
    prm, _, _ = inputs.config_small()
    over = dict(nx=32, ny=32, eps=0.08, dt=2e-4, mobility=5e-3, u_max=1.0, rtol=1e-13,
                max_iters=4000)
    over.update(kw)
    prm = prm.replace(**over)
    geo = inputs.Protrusions(h_b=0.3, centres=(1.0,), radius=0.2, noise=1e-3, seed=1)
    return prm, inputs.initial_state(prm, geo)


def _gpu_vjp(prm, state, nsteps, checkpoint, jbar):
    sim = binding.Simulation([prm], [state])
    try:
        g, theta, st = sim.vjp(0, *state, nsteps, checkpoint, jbar)
        return g.cpu().numpy(), theta, st
    finally:
        sim.close()


CASES = {
    # name: (grid and physics overrides, steps, checkpoint)
    "fh_poiseuille_mg": (dict(), 6, 4),
    "fh_poiseuille_jacobi": (dict(precond=1), 5, 2),
    "dw_shear_stab": (dict(nx=12, ny=10, energy=O.ENERGY_DOUBLE_WELL, gamma2=2.0, stab_s=1.0,
                           flow_mode=O.FLOW_SHEAR, u_max=0.5), 4, 3),
    "ragged_40x22": (dict(nx=40, ny=22), 3, 1),
}


@pytest.mark.parametrize("case", list(CASES))
def test_vjp_matches_oracle_adjoint(case):
    over, nsteps, ck = CASES[case]
    prm, state = _small(**over)
    if "energy" in over:
        state = inputs.initial_state(prm, inputs.Protrusions(h_b=0.3, centres=(1.0,), radius=0.2,
                                                             seed=2))
    jbar = A.objective_weights(prm)
    _, phi0_b, chi_b, mob_b = A.gradient(prm, *state, nsteps, jbar=jbar)
    g, (chi_g, mob_g), st = _gpu_vjp(prm, state, nsteps, ck, jbar)
    assert st["status"] == 0, st
    assert st["steps"] == nsteps
    e_phi = rel(g, phi0_b)
    e_mob = abs(mob_g - mob_b) / abs(mob_b)
    assert e_phi <= TOL_ORACLE, (e_phi, st)
    assert e_mob <= TOL_ORACLE, (mob_g, mob_b)
    if over.get("energy", 0) == 0:
        e_chi = abs(chi_g - chi_b) / abs(chi_b)
        assert e_chi <= TOL_ORACLE, (chi_g, chi_b)
    else:
        assert chi_g == 0.0 and chi_b == 0.0


def test_vjp_random_cotangent_matches_oracle():
    """A cotangent on every node (wall rows included) of phi^N."""
    prm, state = _small(nx=24, ny=16)
    jbar = inputs.random_field(prm, seed=77)
    _, phi0_b, chi_b, mob_b = A.gradient(prm, *state, 3, jbar=jbar)
    g, (chi_g, mob_g), st = _gpu_vjp(prm, state, 3, 2, jbar)
    assert rel(g, phi0_b) <= TOL_ORACLE
    assert abs(chi_g - chi_b) <= TOL_ORACLE * abs(chi_b)
    assert abs(mob_g - mob_b) <= TOL_ORACLE * abs(mob_b)


def test_vjp_checkpoint_spacing_is_bitwise_invariant():
    """Recomputed segments repeat the forward bit for bit, so the result
    does not depend on the checkpoint spacing."""
    prm, state = _small(nx=32, ny=32)
    jbar = A.objective_weights(prm)
    ref = _gpu_vjp(prm, state, 6, 6, jbar)
    for ck in (1, 4, 100):
        g, theta, _ = _gpu_vjp(prm, state, 6, ck, jbar)
        assert np.array_equal(g, ref[0]), ck
        assert theta == ref[1], ck


def test_vjp_zero_steps_is_identity():
    prm, state = _small(nx=16, ny=16)
    jbar = inputs.random_field(prm, seed=3)
    g, theta, st = _gpu_vjp(prm, state, 0, 10, jbar)
    assert np.array_equal(g, jbar)
    assert theta == (0.0, 0.0)


@pytest.mark.parametrize("graph", [0, 1])
def test_vjp_leaves_the_instance_unchanged(graph):
    """step 3, vjp, step 3 == step 6, bit for bit (host and graph mode)."""
    prm, state = _small(nx=32, ny=32, use_graph=graph)
    jbar = A.objective_weights(prm)
    a = binding.Simulation([prm], [state])
    a.step(3)
    before = [f.clone() for f in a.fields[0]]
    a.vjp(0, *state, 4, 2, jbar)
    assert all(np.array_equal(x.cpu().numpy(), y.cpu().numpy())
               for x, y in zip(before, a.fields[0]))
    a.step(3)
    b = binding.Simulation([prm], [state])
    b.step(6)
    for x, y in zip(a.numpy(), b.numpy()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_vjp_argument_errors():
    prm, state = _small(nx=16, ny=16)
    sim = binding.Simulation([prm], [state])
    import torch
    t = [torch.as_tensor(s, dtype=torch.float64).cuda().contiguous() for s in state]
    out = torch.empty_like(t[0])
    for args in [(0, -1, 1), (0, 2, 0), (1, 2, 1)]:
        inst, n, ck = args
        code, _, _ = binding.cahn_vjp(sim.ctx, inst, *[x.data_ptr() for x in t], n, ck,
                                      t[0].data_ptr(), out.data_ptr(), check=False)
        assert code == binding.CAHN_ERR_ARG, args
    code, _, _ = binding.cahn_vjp(sim.ctx, 0, 0, t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(),
                                  1, 1, t[0].data_ptr(), out.data_ptr(), check=False)
    assert code == binding.CAHN_ERR_ARG
    sim.close()


def test_autograd_function_matches_vjp():
    import torch
    from paper_1811_11842_gb300 import autograd as AG
    prm, state = _small(nx=32, ny=32)
    dev = torch.device("cuda:0")
    phi0 = torch.as_tensor(state[0], dtype=torch.float64, device=dev).requires_grad_(True)
    chi = torch.tensor(prm.chi, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(prm.mobility, dtype=torch.float64, requires_grad=True)
    u0, v0, p0 = (torch.as_tensor(s, dtype=torch.float64, device=dev) for s in state[1:])
    wts = AG.detached_volume_weights(prm, device=dev)
    phiN = AG.phase_field_steps(phi0, chi, mob, prm, u0, v0, p0, 5, checkpoint=2)
    J = (wts * phiN).sum()
    J.backward()
    jbar = A.objective_weights(prm)
    assert np.array_equal(wts.cpu().numpy(), jbar)
    g, (chi_g, mob_g), _ = _gpu_vjp(prm, state, 5, 2, jbar)
    assert np.array_equal(phi0.grad.cpu().numpy(), g)
    assert chi.grad.item() == chi_g and mob.grad.item() == mob_g
    # the forward value is the GPU step's
    sim = binding.Simulation([prm], [state])
    sim.step(5)
    assert np.array_equal(phiN.detach().cpu().numpy(), sim.numpy()[0])
    sim.close()


def _gpu_objective(prm, state, nsteps, jbar):
    sim = binding.Simulation([prm], [state])
    sim.step(nsteps)
    phi = sim.numpy()[0]
    sim.close()
    return float(np.sum(jbar * phi))


def test_gradient_matches_central_differences_256():
    """256 x 256 intervals, the 256^2 workload's setup, 50 FP64 steps,
    checkpoints every 10: chi, M and a unit-RMS direction in phi0 against
    central differences with h = 1e-6 (relative for chi and M)."""
    prm, geo, _ = inputs.config_medium()
    prm = prm.replace(rtol=1e-13, max_iters=4000)
    state = inputs.initial_state(prm, geo)
    nsteps, ck = 50, 10
    jbar = A.objective_weights(prm)
    g, (chi_g, mob_g), st = _gpu_vjp(prm, state, nsteps, ck, jbar)
    assert st["status"] == 0, st
    d = inputs.random_field(prm, seed=31)
    d /= np.sqrt(np.mean(d * d))
    fd = {}
    for name in ("chi", "mobility"):
        v = getattr(prm, name)

        def central(h):
            jp = _gpu_objective(prm.replace(**{name: v + h}), state, nsteps, jbar)
            jm = _gpu_objective(prm.replace(**{name: v - h}), state, nsteps, jbar)
            return (jp - jm) / (2 * h)

        h = 1e-2 * abs(v)
        fd[name] = (4.0 * central(h / 2) - central(h)) / 3.0
    h = 1e-6
    sp = (state[0] + h * d,) + tuple(state[1:])
    sm = (state[0] - h * d,) + tuple(state[1:])
    fd["phi0"] = (_gpu_objective(prm, sp, nsteps, jbar) - _gpu_objective(prm, sm, nsteps, jbar)) / (2 * h)
    ad = {"chi": chi_g, "mobility": mob_g, "phi0": float(np.sum(g * d))}
    errs = {k: abs(ad[k] - fd[k]) / abs(fd[k]) for k in fd}
    print("adjoint vs FD at 256^2:", {k: (ad[k], fd[k], errs[k]) for k in fd})
    assert all(e <= TOL_FD for e in errs.values()), (ad, fd, errs)


def test_vjp_graph_instance_matches_host_instance_bitwise():
    """A graph-mode instance replays its captured step in the forward passes;
    the gradient is the host-loop one, bit for bit."""
    prm, state = _small(nx=32, ny=32)
    jbar = A.objective_weights(prm)
    g0, t0, _ = _gpu_vjp(prm, state, 5, 2, jbar)
    g1, t1, _ = _gpu_vjp(prm.replace(use_graph=1), state, 5, 2, jbar)
    assert np.array_equal(g0, g1)
    assert t0 == t1
