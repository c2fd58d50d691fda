"""The oracle on the paper's own parameter set (§5: Re_s, Re_n, Lambda,
Gamma1, Gamma2, the shear flow of §5.1) -- a stiffness stress test of the
scheme (viscosity ratio 4.3e5, Gamma2 = 1.25e6).  CPU only.  Pins: the
conservation form of Eq. 2.4 keeps <phi, 1>_W to the solver tolerance, the
linear Couette profile is an exact discrete steady state at these
viscosities, and ten steps stay inside (0, 1) with a bounded velocity."""
import numpy as np

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs as I


def test_paper_set_conserves_mass_and_stays_in_domain():
    prm, geo, _ = I.config_paper(48)
    g = O.grid_of(prm)
    st = O.init_state(prm, *I.initial_state(prm, geo))
    m0 = st.m0
    worst = 0.0
    for _ in range(10):
        b, a, _ = O.ch_rhs(prm, g, st)
        phi_new, _ = O.solve_phi(prm, g, a, b, x0=st.phi)
        worst = max(worst, abs(O.mass(g, phi_new) - O.mass(g, st.phi)) / m0)
        st = O.step(prm, st)
        assert 0.0 < st.phi.min() and st.phi.max() < 1.0
        assert np.max(np.abs(st.u)) <= 0.1 + 1e-9
    assert worst <= 1e-12, worst


def test_paper_set_couette_is_steady():
    """Uniform phi under the shear u = 0.1 of §5.1: u = 0.1 y/Ly is kept to
    roundoff (linear profiles are differenced exactly), p stays 0."""
    prm, _, _ = I.config_paper(32)
    u0, v0, p0 = I.initial_velocity(prm)
    phi = 0.3 * np.ones_like(u0)
    st = O.run(prm, phi, u0, v0, p0, 4)
    assert np.max(np.abs(st.u - u0)) < 1e-12
    assert np.max(np.abs(st.v)) < 1e-12 and np.max(np.abs(st.p)) < 1e-12
    assert np.max(np.abs(st.phi - 0.3)) < 1e-13
