"""Why the steady march (Sec. 5.2, Eq. cfl) stalls on the bump channel: the channel's parallel
slip walls, pinned on the oracle.

A flat channel (no bump: the steady state is the free stream) at Ma 0.5 starts from the free
stream plus a seeded Gaussian density/pressure blob and marches with PCEXP, local time steps
and the CFL ramp of Eq. cfl capped at 10 (m = 20):

* with far-field faces on all four sides, P1: the density residual drops 10 decades within
  150 iterations, and its late iterations contract by about 0.88 each;
* the same channel with slip walls top and bottom (the bump case's boundaries), P1: after
  150 iterations it has dropped less than 4.5 decades, and its tail contracts by more than
  0.97 per iteration: the part of the perturbation that bounces between the walls leaves only
  slowly, and the P1 scheme damps it only through its small numerical dissipation;
* the walled channel at P0 (far more dissipative) drops 10 decades within 50 iterations.

So the stall of the full-size bump march is the walls' (and the order's), not the bump's
facets nor the Krylov error of the large steps: the paper's steady cases (an airfoil, a
sphere) are external flows with far-field boundaries all around.
"""
import dataclasses

import numpy as np

import workloads as W


def _blob(x):
    r2 = (x[..., 0] - 0.5) ** 2 + (x[..., 1] - 0.5) ** 2
    g = np.exp(-r2 / 0.1 ** 2)
    rho, p = 1.0 + 0.02 * g, 1.0 + 0.02 * g
    u = 0.5 * np.sqrt(1.4)
    return np.stack([rho, rho * u, 0.0 * rho, p / 0.4 + 0.5 * rho * u * u], axis=-1)


def _march(mesh, p, iters):
    from oracle import pcexp
    from oracle.dg import DGOracle
    dg = DGOracle(mesh, p, W.Freestream(0.5, 0.0))
    _, hist = pcexp.steady_march(dg, dg.project(_blob), 10.0, 10.0, iters, 20, dg.area.sum(), scheme="pcexp")
    return hist


def _tail_factor(hist, a, b):
    return (hist[b] / hist[a]) ** (1.0 / (b - a))


def test_open_channel_converges_walled_channel_stalls():
    walled = W.bump_channel(12, 4, 0.0, 1, bump_h=0.0)
    open_ = dataclasses.replace(walled, btags=np.full(len(walled.btags), W.BC_FARFIELD, np.int32))
    ho = _march(open_, 1, 150)
    assert ho[-1] <= 1e-10 * ho[0] and len(ho) <= 150
    assert _tail_factor(ho, len(ho) - 21, len(ho) - 1) < 0.95
    hw = _march(walled, 1, 150)
    assert len(hw) == 150 and hw[-1] > 10 ** -4.5 * hw[0]
    assert _tail_factor(hw, 100, 149) > 0.97
    h0 = _march(walled, 0, 50)
    assert h0[-1] <= 1e-10 * h0[0]
