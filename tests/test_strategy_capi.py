"""The shrink-and-expand decision rule of the library's solve loop (C ABI
``eig_strategy_trace``: host code, no device work) against the oracle's
state machine (oracle/strategy.py, pinned by the hand-worked tables of
test_strategy.py).  On those tables and on seeded random residual histories
the event lists and the active widths must be identical."""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle.strategy import KINDS, Strategy


@pytest.fixture(scope="module")
def lib():
    from paper_2409_05572_gb300 import _lib, build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    _lib.load()
    return _lib


def oracle_trace(kind, nes, nex, rs, r1=None, **params):
    """The decision points of one iteration in the solve's order: record
    r^(j) (and the first pair's residual), expand?, width of iteration j,
    shrink?"""
    st = Strategy(kind, nes, nex, **params)
    nnow, widths = nex, []
    for j, r in enumerate(rs, start=1):
        st.record(j, r, None if r1 is None else r1[j - 1])
        if st.ifexpand(j, nnow):
            nnow = nex
        widths.append(nnow)
        if st.ifshrink(j, nnow):
            nnow = nes
    return st.events, widths


def random_history(rng, m):
    """log10 r^(j): a noisy descent with occasional increases and plateaus."""
    logs = [0.0]
    for _ in range(m - 1):
        u = rng.random()
        if u < 0.15:
            step = rng.uniform(0.0, 0.3)        # residual increase
        elif u < 0.25:
            step = 0.0                          # plateau (slope exactly 0)
        else:
            step = -rng.uniform(0.02, 0.5)
        logs.append(logs[-1] + step)
    return [10.0 ** x for x in logs]


TABLES = [
    ("none", [0.5 ** j for j in range(40)], {}),
    ("fix", [0.5 ** j for j in range(16)], {}),
    ("fix", [1e-6] * 6, {}),
    ("fix", [1e-5] * 60, dict(je=12, js=2)),
    ("slope", [10.0 ** -(j + (0.0 if j < 12 else 0.5 * (j - 11))) for j in range(30)], {}),
    ("slope", [1e-5 * 10.0 ** (-0.3 * j) for j in range(10)] + [1e-7] * 3 + [3e-7] + [1e-8] * 10, {}),
    ("slopek", [1e-5 * 10.0 ** (-0.2 * j) for j in range(40)], dict(jp=4)),
]


@pytest.mark.parametrize("kind,rs,params", TABLES)
def test_trace_matches_oracle_on_tables(lib, kind, rs, params):
    got = lib.eig_strategy_trace(kind, 5, 8, rs, **params)
    want = oracle_trace(kind, 5, 8, rs, **params)
    assert got == want


@pytest.mark.parametrize("seed", range(48))
def test_trace_matches_oracle_on_random_histories(lib, seed):
    rng = np.random.default_rng(seed)
    kind = KINDS[seed % 4]
    params = dict(je=int(rng.choice([6, 12, 15])), js=int(rng.choice([1, 2, 3])),
                  jp=int(rng.choice([3, 10])), mu=float(rng.choice([1.05, 1.1, 1.5])),
                  j_warm=int(rng.choice([1, 5, 9])), r_warm=float(rng.choice([1e-2, 1e-4])))
    nes, nex = (69, 128) if seed % 3 else (5, 8)
    rs = random_history(rng, 150)
    got_events, got_widths = lib.eig_strategy_trace(kind, nes, nex, rs, **params)
    want_events, want_widths = oracle_trace(kind, nes, nex, rs, **params)
    assert got_events == want_events
    assert got_widths == want_widths
    if kind != "none" and min(rs) <= params["r_warm"] and len(rs) > params["j_warm"]:
        assert got_events, "the warm-up gate opened, so at least the first shrink must happen"


@pytest.mark.parametrize("seed", range(24))
def test_trace_matches_oracle_with_first_pair_warmup(lib, seed):
    """warm_first: the gate reads the first pair's residual history, which
    runs ahead of r^(j) by a random factor."""
    rng = np.random.default_rng(1000 + seed)
    kind = KINDS[1 + seed % 3]
    params = dict(je=int(rng.choice([6, 12])), js=int(rng.choice([1, 2])), jp=int(rng.choice([3, 10])),
                  mu=float(rng.choice([1.05, 1.1])), j_warm=int(rng.choice([1, 5])),
                  r_warm=float(rng.choice([1e-1, 1e-4])), warm_first=int(seed % 2 == 0))
    rs = random_history(rng, 120)
    r1 = [x * 10.0 ** -rng.uniform(0.0, 3.0) for x in rs]
    got = lib.eig_strategy_trace(kind, 69, 128, rs, r1=r1, **params)
    want = oracle_trace(kind, 69, 128, rs, r1=r1, **params)
    assert got == want
    # without the option the first pair's history changes nothing
    if not params["warm_first"]:
        assert got == lib.eig_strategy_trace(kind, 69, 128, rs, **params)


def test_trace_defaults_and_zero_residual(lib):
    # r^(j) = 0 is valid (log10 clamped at 1e-300 in both)
    rs = [1.0, 1e-3, 1e-5, 0.0, 0.0, 1e-9, 1e-9, 0.0] + [1e-10] * 30
    for kind in KINDS:
        assert lib.eig_strategy_trace(kind, 5, 8, rs) == oracle_trace(kind, 5, 8, rs)
    assert lib.eig_strategy_trace("fix", 5, 8, []) == ([], [])


def test_trace_rejects_bad_arguments(lib):
    with pytest.raises(lib.EigError):
        lib.eig_strategy_trace("fix", 8, 8, [1.0])            # nes must be below nex
    with pytest.raises(lib.EigError):
        lib.eig_strategy_trace("fix", 5, 8, [1.0, -1e-3])     # negative residual
    with pytest.raises(lib.EigError):
        lib.eig_strategy_trace("fix", 5, 8, [1.0, math.nan])
    with pytest.raises(lib.EigError):
        lib.eig_strategy_trace("fix", 5, 8, [1.0], je=0)
    with pytest.raises(lib.EigError):
        lib.eig_strategy_trace("fix", 5, 8, [1.0, 0.5], r1=[1.0, -0.5])   # negative first-pair residual
    raw = lib.load()
    n = ctypes.c_int(0)
    assert raw.eig_strategy_trace(7, 5, 8, None, None, None, 0, None, None, 0, ctypes.byref(n)) == 1
