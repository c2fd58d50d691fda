"""Temporal order of the oracle's whole step (§4: Crank-Nicolson on the
linear stiff terms, the n+1/2 extrapolation q* = (3 q^n - q^{n-1})/2 for the
rest).  Without flow (u_max = 0, no capillary force) the velocity stays zero
and the step is the phase-field scheme plus the nutrient scheme, both second
order in time: the differences between runs at dt, dt/2, dt/4, dt/8 to the
same final time shrink by 4 per halving.  A first-order slip anywhere in the
time discretisation (an unextrapolated term, a CN weight off 1/2, a wrong
time level of a coefficient) drives the ratio towards 2.
"""
import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import inputs


def _final(prm, state, c0, dt, t_end):
    n = int(round(t_end / dt))
    st = O.run(prm.replace(dt=dt), *state, n, c0=c0)
    return st.phi, st.c


@pytest.mark.parametrize("energy", [O.ENERGY_FLORY_HUGGINS, O.ENERGY_DOUBLE_WELL])
def test_step_is_second_order_in_time_without_flow(energy):
    prm = inputs.Params(nx=16, ny=16, lx=2.0, ly=1.0, eps=0.1, mobility=1e-2, u_max=0.0,
                        gamma_cap=0.0, energy=energy, gamma2=2.0, nutrient=1, diff_s=0.5,
                        growth_mu=1.0, consume_a=10.0, c_bulk=0.8)
    geo = inputs.Protrusions(h_b=0.3, centres=(1.0,), radius=0.25, noise=0.0, seed=0)
    state = inputs.initial_state(prm, geo)
    x, y = inputs.grid_coords(prm)
    c0 = 0.5 + 0.3 * np.cos(np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    t_end = 0.032
    runs = [_final(prm, state, c0, dt, t_end) for dt in (4e-3, 2e-3, 1e-3, 5e-4)]
    for k, name in ((0, "phi"), (1, "c")):
        d = [np.linalg.norm(runs[i][k] - runs[i + 1][k]) for i in range(3)]
        assert d[2] > 0 and d[0] > 1e-9, (name, d)    # the runs really differ
        r1, r2 = d[0] / d[1], d[1] / d[2]
        assert 3.4 < r1 < 4.6 and 3.6 < r2 < 4.4, (name, d, r1, r2)
