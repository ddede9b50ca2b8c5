"""Pin of the oracle's pressure force on a nonlinear field: the Gresho-Chan
vortex (section 4.2, Eqs. gc-az and gc-p) is a steady inviscid balance, so
the momentum rate of pass B must equal the centripetal acceleration
-u_phi^2 / r (radially) wherever the fields are smooth, with the error of a
second-order kernel interpolation: it must shrink about fourfold when the
spacing halves.  A dropped term, a wrong sign or a wrong pressure reading
(C3) shows up as an O(1) error."""
import numpy as np

import oracle
from paper_2107_01276_gb300 import workloads as wl


def _error(nx):
    g = wl.gresho_chan(nx=nx, adaptive=False)
    P = oracle.params(**g["params"])
    pt = g["particles"]
    r = oracle.rhs(P, oracle.dt(P, pt["h"]), oracle.make_state(pt))
    x, y = pt["x"], pt["y"]
    rr = np.hypot(x, y)
    up = wl.gresho_chan_exact(x, y)
    rs = np.where(rr > 0, rr, 1.0)
    ax, ay = -(up ** 2 / rs) * x / rs, -(up ** 2 / rs) * y / rs
    err = np.hypot(r["dudt"] - ax, r["dvdt"] - ay)
    h = 3.0 * pt["h"][0]                      # kernel support
    smooth = (rr > h) & (np.abs(rr - 0.2) > h) & (np.abs(rr - 0.4) > h)
    return err[smooth].max() / np.hypot(ax, ay).max()


def test_gresho_chan_pressure_balance_converges():
    e50, e100 = _error(50), _error(100)
    assert e100 < 5e-3
    assert e50 / e100 > 3.0
