"""Table-driven checks of the shrink-and-expand strategies (Algorithms 6
and 7, Eqs. ckslope / ckslopek, warm-up rule) on scripted residual
histories.  The expected event lists are worked out by hand from the
rules, so they pin the oracle's state machine exactly."""
import pytest

from oracle.strategy import Strategy

NES, NEX = 5, 8


def drive(strategy, rs):
    """Run the decision points of Algorithm 3 over a scripted r^(j) list:
    record r^(j), ifexpand() before the Rayleigh-Ritz step, ifshrink() after."""
    nnow = NEX
    widths = []
    for j, r in enumerate(rs, start=1):
        strategy.record(j, r)
        if strategy.ifexpand(j, nnow):
            nnow = NEX
        widths.append(nnow)
        if strategy.ifshrink(j, nnow):
            nnow = NES
    return strategy.events, widths


def geometric(n, start=1.0, factor=0.5):
    return [start * factor ** j for j in range(n)]


def test_none_never_changes_width():
    ev, widths = drive(Strategy("none", NES, NEX), geometric(40))
    assert ev == [] and set(widths) == {NEX}


def test_warmup_gate_needs_both_conditions():
    # r <= 1e-4 first at j = 15 (0.5^14 = 6.1e-5); j_warm = 5 already met
    ev, _ = drive(Strategy("fix", NES, NEX), geometric(16))
    assert ev == [(15, "shrink")]
    # residual small from the start: gate opens at j_warm = 5
    ev, _ = drive(Strategy("fix", NES, NEX), [1e-6] * 6)
    assert ev == [(5, "shrink")]


def test_fix_schedule_relative_to_first_shrink():
    rs = [1e-5] * 60
    ev, widths = drive(Strategy("fix", NES, NEX, je=12, js=2), rs)
    # first shrink at j0 = 5; expansions at j0 + je - js + i je = 15, 27, 39, 51;
    # shrinks js = 2 iterations after each expansion.
    assert ev == [(5, "shrink"), (15, "expand"), (17, "shrink"), (27, "expand"), (29, "shrink"),
                  (39, "expand"), (41, "shrink"), (51, "expand"), (53, "shrink")]
    assert widths[4] == NEX and widths[5] == NES and widths[14] == NEX and widths[16] == NEX
    assert widths[17] == NES


def test_slope_expands_when_rate_drops_by_mu():
    # steady slope 1.0 per iteration, then it drops to 0.5 at j = 12
    logs = [0.0]
    for j in range(2, 30):
        logs.append(logs[-1] - (1.0 if j < 12 else 0.5))
    rs = [10 ** (l - 3) for l in logs]   # r^(5) = 1e-7 <= 1e-4
    ev, _ = drive(Strategy("slope", NES, NEX, mu=1.1, js=2), rs)
    # shrink at 5 (warm-up); c_max = 1.0; c^(12) = 0.5 -> 1.1*0.5 < 1.0: expand at 12;
    # shrink at 14; after that every slope is 0.5 = c_max -> no expansion.
    assert ev == [(5, "shrink"), (12, "expand"), (14, "shrink")]


def test_slope_expands_on_residual_increase():
    rs = [1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 2e-10, 1e-11, 1e-12, 1e-13]
    ev, _ = drive(Strategy("slope", NES, NEX, mu=1.1, js=2), rs)
    # shrink at 5; c^(6) = 1 -> c_max = 1; c^(7) = -0.30 < 0: expand at 7;
    # shrink at 9 (js = 2 after the expansion)
    assert ev == [(5, "shrink"), (6 + 1, "expand"), (9, "shrink")]


def test_slope_first_post_shrink_increase_expands_immediately():
    rs = [1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 2e-9, 1e-10, 1e-11]
    ev, _ = drive(Strategy("slope", NES, NEX, mu=1.1, js=2), rs)
    # c^(6) < 0 is the first slope after the shrink: c_max = c, mu c < c
    assert ev[:2] == [(5, "shrink"), (6, "expand")]


def test_slopek_uses_window_average():
    # oscillating residual: increments of log10 r alternate -2, +0.5
    logs = [-5.0]
    for j in range(2, 30):
        logs.append(logs[-1] + (-2.0 if j % 2 == 0 else 0.5))
    rs = [10.0 ** l for l in logs]
    ev_k, _ = drive(Strategy("slopek", NES, NEX, mu=1.1, js=2, jp=2), rs)
    ev_s, _ = drive(Strategy("slope", NES, NEX, mu=1.1, js=2), rs)
    # slope: shrink at 5, c^(6) = 2 = c_max, c^(7) = -0.5 -> expand at 7,
    # shrink at 9, c^(10) = 2, c^(11) = -0.5 -> expand at 11, ...
    assert ev_s[:5] == [(5, "shrink"), (7, "expand"), (9, "shrink"), (11, "expand"), (13, "shrink")]
    # slopek (jp = 2): every windowed slope is 0.75 = c_max -> never expands
    assert ev_k == [(5, "shrink")]


def test_slopek_needs_jp_history():
    rs = [1e-5] * 12
    s = Strategy("slopek", NES, NEX, jp=10)
    for j, r in enumerate(rs, start=1):
        s.record(j, r)
    assert s.slope(9) is None
    assert s.slope(10) is None          # needs r^(0)
    assert s.slope(11) == 0.0


@pytest.mark.parametrize("kind", ["fix", "slope", "slopek"])
def test_no_decision_before_warmup(kind):
    rs = [1.0] * 30
    ev, widths = drive(Strategy(kind, NES, NEX), rs)
    assert ev == [] and set(widths) == {NEX}


def test_aggressive_warmup_gates_on_the_first_pair():
    """warm_first (closing remarks of the paper): the gate reads the first
    Ritz pair's residual, not r^(j); with r_warm = 1e-1 the first shrink comes
    at j_warm = 5 although r^(j) is still far above the threshold."""
    r = [1.0] * 3 + [0.5] * 30           # r^(j): never below 1e-1
    r1 = [1.0, 0.5, 0.05] + [0.01] * 30  # first pair: below 1e-1 from j = 3
    st = Strategy("fix", NES, NEX, r_warm=1e-1, warm_first=True)
    nnow = NEX
    for j, (a, b) in enumerate(zip(r, r1), start=1):
        st.record(j, a, b)
        if st.ifexpand(j, nnow):
            nnow = NEX
        if st.ifshrink(j, nnow):
            nnow = NES
    assert st.events[:3] == [(5, "shrink"), (15, "expand"), (17, "shrink")]
    # the same history without warm_first never opens the gate
    st = Strategy("fix", NES, NEX, r_warm=1e-1)
    for j, (a, b) in enumerate(zip(r, r1), start=1):
        st.record(j, a, b)
        assert not st.ifshrink(j, NEX)
    assert st.events == []
