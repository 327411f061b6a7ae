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
    """Solver keyword arguments of a Taylor-Green vortex (Sec. 4.1): unit
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


def channel_solver_kwargs(Ma=0.5, Reb=2800.0, Re_tau=180.0, gamma=GAMMA):
    """Solver keyword arguments of the compressible channel (Sec. 4.2):
    box 2pi x 2 x pi, y in [-1, 1] stretched with b = 2, isothermal walls at
    the bulk temperature 1/(gamma Ma^2), power-law viscosity 1/Re_b at that
    temperature, Pr 0.7, and a constant streamwise body force
    (Re_tau / Re_b)^2 in place of the paper's flow-rate controller."""
    Tw = 1.0 / (gamma * Ma * Ma)
    return dict(lengths=(2 * math.pi, 2.0, math.pi), origin=(0.0, -1.0, 0.0), y_stretch_b=2.0,
                visc=(VISC_POWER, 1.0 / Reb, Tw, OMEGA), Pr=0.7, bc_lo=(0, 1, 0), bc_hi=(0, 1, 0), T_wall=Tw,
                body_force=((Re_tau / Reb) ** 2, 0.0, 0.0), gamma=gamma)


def serve_requests(count=500, seed=500, tgv_share=0.6, tgv_sizes=(32, 48, 64, 96, 128, 160, 192),
                   channel_sizes=(64, 96, 128), steps=(20, 200)):
    """The serving workload: a Poisson stream of solve requests.  Each request
    is a Taylor-Green vortex (Ma 0.1, Re 1600) with probability tgv_share,
    else a channel (Ma_b 0.5, Re_b 2800), on a cubic grid drawn from the
    sizes, for a step count uniform on [steps[0], steps[1]].  Arrival times
    are in units of the mean inter-arrival time (unit-rate exponential gaps);
    divide by the arrival rate to get seconds."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0))
        if rng.uniform() < tgv_share:
            n = int(rng.choice(tgv_sizes))
            req = dict(id=i, arrival=t, kind="tgv", n=(n, n, n), Ma=0.1, Re=1600.0)
        else:
            n = int(rng.choice(channel_sizes))
            req = dict(id=i, arrival=t, kind="channel", n=(n, n, n), Ma=0.5, Re=2800.0, seed=2800 + i)
        req["steps"] = int(rng.integers(steps[0], steps[1] + 1))
        out.append(req)
    return out


def request_work(req):
    """Cell-updates a request asks for."""
    return int(np.prod(req["n"])) * int(req["steps"])
