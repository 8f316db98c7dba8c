"""Physics pin of the oracle (no GPU): the self-similar resistive current sheet
of Sec. 4.2. For p >> B^2 the field obeys the diffusion equation with
eta = 1/sigma, whose solution is B_y = B0 erf(x sqrt(sigma/t)/2). Started from
the exact profile at t = 1 and run for 9 time units (sigma = 100, p = 50,
rho = 1), the oracle's B_y approaches the profile at t = 10 as N grows."""
import math

import numpy as np

import oracle as O
from paper_1808_09721_gb300 import workloads as WL


def _run(n):
    wl = WL.current_sheet(nx=n)
    sim = O.Sim(O.MODEL_SF, wl.nx, 1, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    sim.set_prims(wl.prims)
    T = 9.0
    nst = int(math.ceil(T / wl.dt))
    sim.step(T / nst, nst)
    x = wl.xlim[0] + (np.arange(n) + 0.5) * (wl.xlim[1] - wl.xlim[0]) / n
    exact = np.array([math.erf(0.5 * xx * math.sqrt(wl.sigma / 10.0)) for xx in x])
    return np.mean(np.abs(sim.prims()[6, 0] - exact))


def test_current_sheet_diffuses_like_erf():
    e50, e100, e200 = _run(50), _run(100), _run(200)
    assert e100 < 2e-3
    assert e50 > 3.0 * e100 > 3.0 * e200 * 1.0
    assert e200 < e100
