"""Write the oracle's diagnostic histories used by the long-run GPU parity tests.

Calls only the CPU oracle (`oracle/`).  Each case steps one problem with the
oracle and records, after every step, the time, the time step and the
diagnostics of Sec. 4.1 (kinetic energy, enstrophy, compressible dissipation,
totals, maximum Mach number, wall shear), plus the conservative variables of a
seeded sample of cells at a few checkpoint steps, with the per-component scale
max |Q| of the whole state at that step.

Cases (parameters restate the workloads; R = 1, gamma = 1.4):
  tgv64    Taylor-Green vortex (Sec. 4.1) on [0, 2 pi]^3, 64^3 cells, Ma 0.1,
           Re 1600, Pr 0.72, mu = (1/Re) (T/T0)^0.7, 200 steps at CFL 0.5.
  channel  Compressible channel (Sec. 4.2 set-up with Ma_b 0.5, Re_b 2800):
           2 pi x 2 x pi, 32 x 48 x 24 cells, y stretched with b = 2, isothermal
           no-slip walls, body force (180/2800)^2, 10 % seeded velocity noise
           (seed 2800), 200 steps at CFL 0.5.
  tgv256   The Taylor-Green vortex above at 256^3 cells, 2 steps at CFL 0.5
           (the full-size workload; about half an hour per step on 8 cores).
  tgv32long  The Taylor-Green vortex above at 32^3 cells, 1200 steps at CFL
           0.5 (t ~ 11 convective times: through the transition, where the
           flow is chaotic and rounding differences grow).

Usage: python tests/golden/make_histories.py tgv64 [channel tgv256 ...]
"""
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ref  # noqa: E402

GAMMA = 1.4


def tgv_case(n, steps, checkpoints):
    p0 = 1.0 / (GAMMA * 0.1 * 0.1)
    kw = dict(gamma=GAMMA, Pr=0.72, visc=(ref.VISC_POWER, 1.0 / 1600.0, p0, 0.7))
    return dict(kind="tgv", n=(n, n, n), solver=kw, init=dict(Ma=0.1, U0=1.0, rho0=1.0),
                steps=steps, cfl=0.5, checkpoints=checkpoints)


def channel_case(n, steps, checkpoints):
    Ma, Reb = 0.5, 2800.0
    Tw = 1.0 / (GAMMA * Ma * Ma)
    kw = dict(gamma=GAMMA, lengths=(2 * math.pi, 2.0, math.pi), origin=(0.0, -1.0, 0.0), y_stretch_b=2.0,
              visc=(ref.VISC_POWER, 1.0 / Reb, Tw, 0.7), Pr=0.7, bc_lo=(0, 1, 0), bc_hi=(0, 1, 0),
              T_wall=Tw, body_force=((180.0 / Reb) ** 2, 0.0, 0.0))
    return dict(kind="channel", n=n, solver=kw, init=dict(Ma_b=Ma, noise_amp=0.1, seed=2800),
                steps=steps, cfl=0.5, checkpoints=checkpoints)


CASES = {
    "tgv64": tgv_case(64, 200, (10, 100, 200)),
    "channel": channel_case((32, 48, 24), 200, (10, 100, 200)),
    "tgv256": tgv_case(256, 2, (1, 2)),
    "tgv32long": tgv_case(32, 1200, (10, 100, 400, 800, 1200)),
}
SAMPLES = 384


def run(name):
    case = CASES[name]
    n = tuple(case["n"])
    s = ref.RefSolver(n, **case["solver"])
    if case["kind"] == "tgv":
        s.init_tgv(**case["init"])
    else:
        s.init_channel(**case["init"])
    ncell = n[0] * n[1] * n[2]
    rng = np.random.default_rng(20701173)
    cells = np.sort(rng.choice(ncell, size=min(SAMPLES, ncell), replace=False)).astype(np.int64)
    history, checks = [], {}
    t0 = time.time()
    for k in range(1, case["steps"] + 1):
        s.step(1, case["cfl"])
        st = s.stats()
        history.append(st)
        if k in case["checkpoints"]:
            q = s.get_state().reshape(5, -1)
            checks[str(k)] = dict(scale=[float(v) for v in np.abs(q).max(axis=1)],
                                  values=[[float(v) for v in q[:, c]] for c in cells])
        print("%s step %d/%d  t=%.6e Ek=%.15e  (%.0f s)" % (name, k, case["steps"], st["t"], st["Ek"],
                                                           time.time() - t0), flush=True)
    out = dict(
        source="written by tests/golden/make_histories.py from the CPU oracle (oracle/hgks_ref.c)",
        case=name, kind=case["kind"], n=list(n), solver={k: list(v) if isinstance(v, tuple) else v
                                                           for k, v in case["solver"].items()},
        init=case["init"], cfl=case["cfl"], steps=case["steps"],
        sample_cells=[int(c) for c in cells], history=history, checkpoints=checks,
        oracle_seconds=round(time.time() - t0, 1))
    path = os.path.join(HERE, "history_%s.json" % name)
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
    os.replace(path + ".tmp", path)
    print("wrote", path)


if __name__ == "__main__":
    for name in sys.argv[1:] or ["tgv64", "channel"]:
        run(name)
