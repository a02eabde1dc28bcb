"""Pins of the exact mean first-passage time (Eq. 5-7) on the tiny state space
of one vacancy and one Cu atom in a 3^3-cell Fe lattice (pair model, 2862
states), absorbing set: the vacancy and the Cu farther apart than second
neighbours.  Independent checks: Monte Carlo first-passage times of oracle
trajectories, a one-step closed form, translation invariance, and Eq. 7 with
the exact potential."""
import numpy as np
import pytest

import oracle
import oracle.mfpt as MF
import synth

L, T = 3, 563.0


@pytest.fixture(scope="module")
def chain(model):
    vs, cs, sp = synth.vacancy_solute_states(L)
    desc = synth.VoxelDesc(L, 1, (0.0, 0.0, 0.0), T, synth.PAIR_MODEL, synth.PREC_FP64, seed=5, uid=5)
    rates = MF.oracle_rates(model, desc, sp, vs)
    succ = MF.successors(vs, cs, L)
    r2 = np.array([MF.min_image_r2(int(v), int(c), L) for v, c in zip(vs, cs)])
    absorbing = r2 > 4
    tau = MF.solve_mfpt(rates, succ, absorbing)
    return dict(vs=vs, cs=cs, sp=sp, rates=rates, succ=succ, absorbing=absorbing, tau=tau, r2=r2, desc=desc)


def test_state_space(chain):
    assert chain["vs"].size == 54 * 53
    assert chain["absorbing"].any() and (~chain["absorbing"]).any()
    assert (chain["tau"][chain["absorbing"]] == 0).all()
    assert (chain["tau"][~chain["absorbing"]] > 0).all()


def test_one_step_closed_form(chain):
    # absorbing set = every state but s0: the first hop always absorbs
    s0 = int(np.flatnonzero(~chain["absorbing"])[7])
    ab = np.ones_like(chain["absorbing"])
    ab[s0] = False
    tau = MF.solve_mfpt(chain["rates"], chain["succ"], ab)
    assert tau[s0] == pytest.approx(1.0 / chain["rates"][s0].sum(), rel=1e-13)


def test_translation_invariance(chain):
    # tau depends only on the relative vacancy-solute vector
    rel = {}
    for i, (v, c) in enumerate(zip(chain["vs"], chain["cs"])):
        d = MF.half_coords(int(c), L) - MF.half_coords(int(v), L)
        d = tuple(((d + L) % (2 * L)).tolist())
        rel.setdefault(d, []).append(chain["tau"][i])
    for vals in rel.values():
        vals = np.array(vals)
        assert np.allclose(vals, vals[0], rtol=1e-10, atol=0)


def test_eq7_with_exact_potential(chain):
    tau, rates, succ = chain["tau"], chain["rates"], chain["succ"]
    u = MF.potential(tau, rates)
    gt = rates.sum(axis=1)
    dt = MF.delta_tau(tau, succ)
    tr = np.flatnonzero(~chain["absorbing"])
    est = (u[tr, None] - (gt[tr, None] / gt[succ[tr]]) * u[succ[tr]]) / gt[tr, None]
    np.testing.assert_allclose(est, dt[tr], rtol=1e-10, atol=1e-12 * tau.max())
    # the mean increment over the event distribution is the mean residence time
    mean_inc = (rates[tr] * dt[tr]).sum(axis=1) / gt[tr]
    np.testing.assert_allclose(mean_inc, 1.0 / gt[tr], rtol=1e-9)


def test_monte_carlo_first_passage(model, chain):
    vs, cs, sp = chain["vs"], chain["cs"], chain["sp"]
    starts = [int(i) for i in np.flatnonzero(chain["r2"] == 3)[:1]] + \
             [int(i) for i in np.flatnonzero(chain["r2"] == 4)[:1]]
    runs = 1500
    for s in starts:
        times = np.empty(runs)
        for k in range(runs):
            d = synth.VoxelDesc(L, 1, (0.0, 0.0, 0.0), T, synth.PAIR_MODEL, synth.PREC_FP64, seed=77, uid=1000 + k)
            v = oracle.Voxel(d, model)
            v.load(sp[s], np.array([vs[s]], np.int32))
            vp, cp, t = int(vs[s]), int(cs[s]), 0.0
            while MF.min_image_r2(vp, cp, L) <= 4:
                log, dts = v.step(1, log=True, dt=True)
                e = int(log[0])
                X = MF.half_coords(vp, L)
                m = MF.site_of(X + np.array([-1 if e & 1 else 1, -1 if e & 2 else 1, -1 if e & 4 else 1]), L)
                if m == cp:
                    cp = vp
                vp = m
                t += float(dts[0])
            times[k] = t
        se = times.std(ddof=1) / np.sqrt(runs)
        assert abs(times.mean() - chain["tau"][s]) < 4 * se, (s, times.mean(), chain["tau"][s], se)
