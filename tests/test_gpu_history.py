"""Long-run parity of the CUDA path with the oracle: diagnostic histories.

The oracle's histories are stored under tests/golden/ (written by
tests/golden/make_histories.py, which calls only the CPU oracle): after every
step the time, the time step and the diagnostics of Sec. 4.1, plus the
conservative variables of a seeded sample of cells at checkpoint steps.

Tolerances:
  * FP64 path: every entry of the E_k / enstrophy / eps_com / wall-shear
    histories within 1e-6 relative (the stated bound for longer runs); in
    practice the two FP64 codes differ only in rounding order, so the test
    also records the largest difference and holds it well below 1e-9.  The
    sampled cells after 10 steps within 1e-11 relative (per component,
    momenta sharing one normaliser, the scale being max |Q| of the whole
    oracle state), as for the short parity runs; later checkpoints within
    1e-9 (rounding differences grow slowly with the steps).
  * Mixed path: its statistical error against the same oracle histories,
    printed and bounded.  FP32 rounding (6e-8) of the flux terms, amplified
    by the cancellation of neighbouring face fluxes (about L/h), leaves a
    per-cell state error near 1e-6 of the state; E_k, a volume average of
    the state, keeps about 1e-8.  Enstrophy and dissipation square
    fourth-order velocity differences: for the Taylor-Green vortex these are
    smooth and keep the state's relative error (bound 1e-7), while in the
    channel they are dominated by the grid-scale seeded noise, whose
    differences are ~10x smaller than the velocity, so the relative error
    grows by that factor (bound 3e-5; measured 1.2e-6 and 7.6e-6 over 200
    steps).  The mixed run takes its own CFL steps, so its times drift from
    the oracle's by the same relative amount as the states.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def golden(name):
    path = os.path.join(HERE, "golden", "history_%s.json" % name)
    if not os.path.exists(path):
        pytest.fail("missing golden history %s (run tests/golden/make_histories.py %s)" % (path, name))
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def hg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2207_01173_gb300 as hg
    return hg


def solver_for(hg, g, precision):
    kw = {k: tuple(v) if isinstance(v, list) else v for k, v in g["solver"].items()}
    s = hg.Solver(tuple(g["n"]), precision=precision, **kw)
    if g["kind"] == "tgv":
        s.init_tgv(**g["init"])
    else:
        s.init_channel(**g["init"])
    return s


def sampled_err(q, chk, cells):
    """Relative error of the sampled cells, per component, momenta sharing
    the largest momentum scale."""
    scale = np.array(chk["scale"])
    scale[1:4] = scale[1:4].max()
    ref = np.array(chk["values"])             # [ncells][5]
    got = q.reshape(5, -1)[:, cells].T        # [ncells][5]
    return (np.abs(got - ref) / scale).max(axis=0)


def run_history(hg, g, precision):
    s = solver_for(hg, g, precision)
    cells = np.array(g["sample_cells"], dtype=np.int64)
    hist, errs = [], {}
    for k in range(1, g["steps"] + 1):
        s.step(1, g["cfl"])
        hist.append(s.stats())
        if str(k) in g["checkpoints"]:
            errs[k] = sampled_err(s.get_state(), g["checkpoints"][str(k)], cells)
    s.close()
    return hist, errs


KEYS = {"tgv": ("Ek", "enstrophy", "eps_com"), "channel": ("Ek", "enstrophy", "eps_com", "wall_shear")}


def history_rel(hist, g, keys):
    out = {}
    for key in keys + ("t", "dt", "mass", "energy"):
        a = np.array([h[key] for h in hist])
        b = np.array([h[key] for h in g["history"]])
        out[key] = float((np.abs(a - b) / np.maximum(np.abs(b), 1e-300)).max())
    return out


# the oracle histories stored under tests/golden/
HISTORIES = ["tgv64", "channel"]


@pytest.mark.parametrize("name", HISTORIES)
def test_fp64_history_matches_oracle(hg, name):
    g = golden(name)
    hist, errs = run_history(hg, g, hg.FP64)
    assert [h["step"] for h in hist] == list(range(1, g["steps"] + 1))
    rel = history_rel(hist, g, KEYS[g["kind"]])
    print("FP64 vs oracle, %s, %d steps: %s" % (name, g["steps"], rel))
    for key in KEYS[g["kind"]]:
        assert rel[key] < 1e-6, (key, rel[key])
        assert rel[key] < 1e-9, (key, rel[key])
    assert rel["t"] < 1e-12 and rel["dt"] < 1e-12
    # totals are sums over every cell taken in different orders (a tree on the
    # GPU, serial in the oracle): rounding of order sqrt(N) eps, N = 64^3
    # (measured 2.2e-13)
    assert rel["mass"] < 1e-12 and rel["energy"] < 1e-12
    for k, e in errs.items():
        print("  sampled cells after %d steps: %s" % (k, e))
        assert e.max() < (1e-11 if k <= 10 else 1e-9), (k, e)


MIXED_BOUNDS = {"tgv": {"Ek": 1e-7, "enstrophy": 1e-7, "eps_com": 1e-7},
                "channel": {"Ek": 1e-7, "enstrophy": 3e-5, "eps_com": 3e-5, "wall_shear": 1e-5}}


@pytest.mark.parametrize("name", HISTORIES)
def test_mixed_history_against_oracle(hg, name):
    """The mixed path's statistical error against the oracle's FP64 history."""
    g = golden(name)
    hist, errs = run_history(hg, g, hg.MIXED)
    rel = history_rel(hist, g, KEYS[g["kind"]])
    print("mixed vs oracle, %s, %d steps: %s; sampled cells: %s" % (
        name, g["steps"], rel, {k: float(e.max()) for k, e in errs.items()}))
    bounds = MIXED_BOUNDS[g["kind"]]
    for key, b in bounds.items():
        assert rel[key] < b, (key, rel[key], b)
    # the update stays FP64, but mass passes the channel walls (the mirror
    # ghosts' densities differ from the interior's) through FP32 wall fluxes
    assert rel["mass"] < 1e-9
    for k, e in errs.items():
        assert e.max() < 1e-5, (k, e)


def test_fp64_full_size_tgv256_two_steps(hg):
    """The full-size Taylor-Green workload (256^3, the benchmark's) against
    two oracle steps: time steps and the sampled cells within the short-run
    bounds (measured 7e-15).  The diagnostics are held to 1e-9: at 16.7 M
    cells the oracle's serial summation, not the states, sets their
    difference (its total mass differs by the same 2.4e-10 while every cell
    agrees to 1e-14)."""
    g = golden("tgv256")
    hist, errs = run_history(hg, g, hg.FP64)
    rel = history_rel(hist, g, KEYS["tgv"])
    print("FP64 vs oracle, tgv256, 2 steps: %s; sampled cells: %s"
          % (rel, {k: float(e.max()) for k, e in errs.items()}))
    for key in KEYS["tgv"]:
        assert rel[key] < 1e-9, (key, rel[key])
    assert rel["dt"] < 1e-12 and rel["t"] < 1e-12
    assert sorted(errs) == [1, 2]
    for k, e in errs.items():
        assert e.max() < 1e-11, (k, e)


def test_fp64_through_the_transition_tgv32(hg):
    """A longer, chaotic run: the Taylor-Green vortex at 32^3 over 1200 steps
    (t ~ 10.6 convective times, through the transition to small-scale
    motion), FP64 against the oracle's stored history.  Rounding differences
    between the two FP64 codes grow once the flow becomes chaotic; the kinetic
    energy and enstrophy histories must stay within 1e-6 relative over the
    whole run (the stated bound for longer chaotic runs)."""
    g = golden("tgv32long")
    hist, errs = run_history(hg, g, hg.FP64)
    ek = np.array([h["Ek"] for h in hist]), np.array([h["Ek"] for h in g["history"]])
    en = np.array([h["enstrophy"] for h in hist]), np.array([h["enstrophy"] for h in g["history"]])
    rek = np.abs(ek[0] - ek[1]) / np.abs(ek[1])
    ren = np.abs(en[0] - en[1]) / np.abs(en[1])
    for k in (100, 400, 800, 1200):
        print("step %d t %.3f: E_k rel %.2e, enstrophy rel %.2e" % (k, g["history"][k - 1]["t"], rek[:k].max(),
                                                                    ren[:k].max()))
    print("sampled cells: %s" % {k: float(e.max()) for k, e in errs.items()})
    assert rek.max() < 1e-6 and ren.max() < 1e-6
