"""Rigid-body oscillator of §2.3.2 (oracle, FP64).

Eq. (12):  m wdd + c wd + k w = F   per translational degree of freedom,
integrated with the classical fourth-order Runge-Kutta method, the force
held at its value from the fluid step (weak coupling, N = 1 in Algorithm 1).

Reading: the paper prints k = 2 m (2 pi f_n)^2; the natural-frequency relation
of a spring-mass system is k = m (2 pi f_n)^2, so the factor is a parameter
(k_factor, 1 by default).  c = 2 m (2 pi f_n) zeta.

Parity: pinned against the closed-form free vibration y0 cos(omega t) with
fourth-order convergence in dt and the static offset F / k under a constant
force (tests/test_oracle_body.py).
"""
import math

import torch


class RigidParams:
    def __init__(self, m, k, c=0.0, active=(False, True)):
        self.m = float(m)
        self.k = k if torch.is_tensor(k) else torch.tensor(float(k), dtype=torch.float64)
        self.c = float(c)
        self.active = tuple(bool(a) for a in active)

    @staticmethod
    def from_reduced(mass_ratio, reduced_velocity, U, D, zeta=0.0, rho=1.0, k_factor=1.0,
                     active=(False, True)):
        """m = m* rho pi D^2 / 4, f_n = U / (U_r D), k = k_factor m (2 pi f_n)^2, c = 2 m 2 pi f_n zeta."""
        m = mass_ratio * rho * math.pi * D * D / 4.0
        fn = U / (reduced_velocity * D)
        k = k_factor * m * (2.0 * math.pi * fn) ** 2
        c = 2.0 * m * 2.0 * math.pi * fn * zeta
        return RigidParams(m, k, c, active)


def rk4(params, w, wd, F, dt):
    """One RK4 step of Eq. (12) for each active DOF; inactive DOFs stay at rest."""
    m, k, c = params.m, params.k, params.c
    w_new, wd_new = [], []
    for d in range(2):
        if not params.active[d]:
            w_new.append(w[d] * 0.0)
            wd_new.append(wd[d] * 0.0)
            continue
        acc = lambda x, v: (F[d] - c * v - k * x) / m  # noqa: E731
        k1x, k1v = wd[d], acc(w[d], wd[d])
        k2x, k2v = wd[d] + 0.5 * dt * k1v, acc(w[d] + 0.5 * dt * k1x, wd[d] + 0.5 * dt * k1v)
        k3x, k3v = wd[d] + 0.5 * dt * k2v, acc(w[d] + 0.5 * dt * k2x, wd[d] + 0.5 * dt * k2v)
        k4x, k4v = wd[d] + dt * k3v, acc(w[d] + dt * k3x, wd[d] + dt * k3v)
        w_new.append(w[d] + dt / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x))
        wd_new.append(wd[d] + dt / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v))
    return torch.stack(w_new), torch.stack(wd_new)
