"""Pins of the oracle's WINDOW stop rule (Sec. 3.4: the equilibrium test on
the last n_fit = 20 sweeps of the energy series, every n_f = 5 sweeps, first
after n_fit + n_f = 25).

  * the slope numerator is the least-squares slope of the window (numpy's
    polyfit) times 2 sum (j - mean j)^2, and n (n^2 - 1) c / 6 on a line of
    slope c;
  * on constructed energy series the stop sweeps are the ones derived by
    hand: a ramp that levels off stops at the first test whose window is
    flat, a series that turns back stops at the first test that sees the
    turn, sigma = 0 stops at the first test, and blocks without sample bonds
    close with the targeted blocks;
  * a whole simulation's stop sweeps follow from its own energy trace by
    polyfit slopes.
"""
import numpy as np
import pytest

import oracle
from test_oracle_mc import _stop_problem


def ring(trace_fn, t, n_fit, nblk):
    """The ring the caller keeps: e_b(s) at row s mod n_fit for s <= t."""
    h = np.zeros((n_fit, nblk))
    for s in range(max(1, t - n_fit + 1), t + 1):
        h[s % n_fit] = trace_fn(s)
    return h


@pytest.mark.parametrize("n_fit", [20, 7])
def test_slope_numerator_is_the_least_squares_slope(n_fit):
    rng = np.random.default_rng(n_fit)
    o = oracle.Oracle(4, 4, 2, n_fit=n_fit)
    nblk = o.nblk
    series = rng.normal(size=(200, nblk)).cumsum(axis=0)
    for t in (n_fit, n_fit + 13, 150):
        h = ring(lambda s: series[s], t, n_fit, nblk)
        x = np.arange(n_fit)
        for b in range(nblk):
            y = series[t - n_fit + 1: t + 1, b]
            slope = np.polyfit(x, y, 1)[0]
            want = 2.0 * slope * np.sum((x - x.mean()) ** 2)
            assert o.window_slope(t, h, b) == pytest.approx(want, rel=1e-9, abs=1e-9)
    c = 0.37
    h = ring(lambda s: np.full(nblk, 1.5 + c * s), 40, n_fit, nblk)
    assert o.window_slope(40, h, 0) == pytest.approx(n_fit * (n_fit ** 2 - 1) * c / 6, rel=1e-12)


def run_rule(o, traces, sigma, Nsp, n_max=80):
    """Stop sweeps of the WINDOW rule on given e_b(t) series (t = 1 ..)."""
    nblk = o.nblk
    st = oracle.BlockStats(Es=np.zeros(nblk), Nsp=np.asarray(Nsp, np.int64),
                           Nb=np.ones(nblk, np.int64), mean_angle=np.zeros(nblk),
                           n_gap=np.ones(nblk, np.int64), n_sample=np.ones(nblk, np.int64),
                           global_mean=0.0)
    sig = np.asarray(sigma, np.int8)
    active = np.ones(nblk, np.uint8)
    stop = np.full(nblk, -1, np.int32)
    h = np.zeros((o.m.n_fit, nblk))
    for t in range(1, n_max + 1):
        h[t % o.m.n_fit] = traces(t)
        if o.stop_update_window(t, n_max, st, sig, h, active, stop) == 0:
            break
    return stop


def test_constructed_series_stop_where_derived():
    o = oracle.Oracle(4, 8, 2, n_fit=20, n_f=5)     # 8 blocks
    assert o.nblk == 8

    def tr(t):
        ramp_up = 0.01 * min(t, 27)                    # levels off at t = 27
        ramp_dn = -0.01 * min(t, 27)
        turn = 0.01 * t if t <= 30 else 0.3 - 0.02 * (t - 30)   # turns at t = 30
        noise_free_flat = 0.0
        return np.array([ramp_up, ramp_dn, turn, ramp_up, noise_free_flat, 0.01 * t,
                         ramp_up, -0.01 * t])

    sigma = [+1, -1, +1, -1, +1, +1, 0, -1]
    Nsp = [5, 5, 5, 5, 5, 5, 5, 0]
    stop = run_rule(o, tr, sigma, Nsp, n_max=80)
    # A ramp that levels off at 27: the windows ending at 25 .. 45 still rise
    # (the window 26..45 holds 26 -> 27), the one ending at 50 is flat (slope
    # 0, and sigma * 0 <= 0 stops).
    assert stop[0] == 50 and stop[1] == 50
    # Rising until 30, then falling twice as fast: the window ending at 35
    # (16..35: 15 sweeps up, 5 down) still has a positive least-squares slope,
    # the one ending at 40 (21..40: 10 up, 10 down twice as fast) a negative
    # one.
    x = np.arange(20)
    slope35 = np.polyfit(x, [tr(s)[2] for s in range(16, 36)], 1)[0]
    slope40 = np.polyfit(x, [tr(s)[2] for s in range(21, 41)], 1)[0]
    assert slope35 > 0 > slope40
    assert stop[2] == 40
    # Moving away from the target (sigma -1, rising): stops at the first test.
    assert stop[3] == 25
    # A flat series: slope 0 stops at the first test; so does sigma = 0.
    assert stop[4] == 25 and stop[6] == 25
    # Still drifting towards the target: runs to n_max.
    assert stop[5] == 80
    # No sample bonds: closes when no targeted block runs (here at n_max,
    # because block 5 runs to the end).
    assert stop[7] == 80


def test_simulation_stops_follow_its_energy_trace():
    z, mask, lb = _stop_problem()
    H, W = mask.shape
    o = oracle.Oracle(H, W, lb, seed=9, stop_rule=1, n_fit=20, n_f=5)
    phi, *_ = o.transform(z, mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    T = np.random.default_rng(1).uniform(0.02, 0.6, o.nblk)
    n_max = 90
    _, stop, n, tr = o.simulate_one(phi0, mask, T, st, n_max, r=2, trace=True)
    es = st.es
    sigma = np.sign(es - tr[0])
    targeted = (st.Nsp > 0) & (st.n_gap > 0)
    x = np.arange(20)
    for b in np.where(targeted)[0]:
        want = n_max
        for t in range(25, n_max + 1, 5):
            slope = np.polyfit(x, tr[t - 19: t + 1, b], 1)[0]
            if sigma[b] * slope <= 0:
                want = t
                break
        assert stop[b] == want, (b, stop[b], want)
    assert np.all(stop[st.n_gap == 0] == 0)
    others = (st.Nsp == 0) & (st.n_gap > 0)
    if targeted.any():
        assert np.all(stop[others] == stop[targeted].max())
    assert n == stop.max()
