"""Pins of the complex step through whole oracle PCEXP steps (the gradient reference of the
adjoint, Sec. 8c of the scope: derivatives of the step map as computed).

Im F(u + i h delta) / h with h = 1e-30 is the exact directional derivative of the step map F
(no cancellation); it must agree with central differences of the real step to their O(h^2)
accuracy, for a state direction and for the free-stream Mach number and angle entering
through the far-field ghost state and the projected initial state.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import pcexp
from oracle.cases import freestream_state
from oracle.dg import DGOracle


def _setup(free):
    mesh = W.bump_channel(8, 4, 0.15, 1)
    dg = DGOracle(mesh, 1, free)
    return mesh, dg


def _J(dg, u, steps, dt=0.02, m=8):
    for _ in range(steps):
        u, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, m)
    return dg.wall_force(u, (1.0, 0.0))


def test_complex_step_state_direction_matches_central_differences():
    free = W.Freestream(0.5, 2.0)
    mesh, dg = _setup(free)
    u0 = dg.project(lambda x: freestream_state(x, free)).reshape(-1)
    u0 = u0 * (1.0 + 0.01 * W.uniform_pm(3, u0.size))
    delta = W.random_coeffs(4, (dg.K,)) * np.abs(u0)
    cs = np.imag(_J(dg, u0 + 1e-30j * delta, 2)) / 1e-30
    h = 1e-6
    fd = (_J(dg, u0 + h * delta, 2) - _J(dg, u0 - h * delta, 2)) / (2 * h)
    assert abs(cs - fd) <= 1e-6 * abs(fd), (cs, fd)


@pytest.mark.parametrize("name,h", [("mach", 1e-5), ("alpha_deg", 1e-3)])
def test_complex_step_freestream_parameter_matches_central_differences(name, h):
    free = W.Freestream(0.5, 2.0)

    def J_of(fr):
        mesh, dg = _setup(fr)
        u0 = dg.project(lambda x: freestream_state(x, fr)).reshape(-1)
        u0 = u0 + 0.03 * W.random_coeffs(5, u0.shape)  # a fixed perturbation (|.| is not analytic)
        return _J(dg, u0, 2)

    th = getattr(free, name)
    cs = np.imag(J_of(dataclasses.replace(free, **{name: th + 1e-30j}))) / 1e-30
    fd = (J_of(dataclasses.replace(free, **{name: th + h})) - J_of(dataclasses.replace(free, **{name: th - h}))) / (2 * h)
    assert abs(cs - fd) <= 1e-5 * abs(fd), (cs, fd)
