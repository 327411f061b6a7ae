"""Seeded synthetic workloads: which problems to run, with which parameters.

Only problem descriptions live here (grid sizes, Mach and Reynolds numbers,
arrival times); the flow fields themselves are set by the solver's own
initialisation kernels.  No arithmetic of the method is in this module.
"""
import math

import numpy as np

GAMMA = 1.4
PR = 0.72
OMEGA = 0.7
VISC_POWER = 1


def tgv_solver_kwargs(Ma, Re, gamma=GAMMA):
    """Solver keyword arguments of a Taylor-Green vortex (Section 5.1): unit
    velocity and density scale, mean pressure 1/(gamma Ma^2), power-law
    viscosity mu = (1/Re) (T/T0)^0.7 with T0 the mean temperature p0/rho0."""
    p0 = 1.0 / (gamma * Ma * Ma)
    return dict(visc=(VISC_POWER, 1.0 / Re, p0, OMEGA), Pr=PR, gamma=gamma)


def batch_tgv_problems(count=64, seed=64, sizes=(24, 32, 48, 64, 96)):
    """The batched Taylor-Green workload: each problem draws its three grid
    sizes independently from `sizes`, Ma ~ U[0.1, 0.5] and Re log-uniform on
    [400, 3200].  Returns a list of ((nx, ny, nz), Ma, Re)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.choice(sizes, size=3))
        Ma = float(rng.uniform(0.1, 0.5))
        Re = float(math.exp(rng.uniform(math.log(400.0), math.log(3200.0))))
        out.append((n, Ma, Re))
    return out
