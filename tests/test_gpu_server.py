"""Batched steps and serving on the GPU.

* every result is the same alone and in the mix (continuous batching with a
  budget that forces queueing, FP32 and FP64 requests together, ragged sizes);
* a served request equals the oracle run of the same steps (rotation field,
  which both sides evaluate with the same IEEE operations);
* graph replay and plain launches give identical results;
* a request that fails mid-run (an injected CFL violation, or a device-side
  wait of the persistent schedule made to run out) or is cancelled stops with
  its status, and every other request's result is still the one it gets
  alone."""
import math

import numpy as np
import pytest

import oracle
from paper_2309_00338_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2309_00338_gb300 import ebit  # noqa: E402


def _mix():
    rng = W.Rng(2024)
    reqs = []
    specs = [(48, ebit.EBIT_FIELD_VORTEX, 0, 40), (64, ebit.EBIT_FIELD_CELLULAR, 1, 30),
             (97, ebit.EBIT_FIELD_ROTATION, 0, 25), (130, ebit.EBIT_FIELD_VORTEX, 1, 20),
             (33, ebit.EBIT_FIELD_CELLULAR, 0, 50), (80, ebit.EBIT_FIELD_ROTATION, 1, 35)]
    for n, field, prec, steps in specs:
        dx = 1.0 / n
        circles = W.place_circles(rng, 6, 3 * dx, 0.12, 2 * dx, lambda x, y, r: True, max_tries=50)
        reqs.append(dict(n=n, circles=circles, field=field, prec=prec, steps=steps, cfl=0.5,
                         period=steps * 0.5 * dx, omega=2 * math.pi, centre=(0.5, 0.5), drift=(0.1, -0.05)))
    return reqs


def _run(specs, budget, use_graphs=True, autotune=True, schedule=0, wait_budget_ms=0):
    s = ebit.ebit_server_create(budget, use_graphs=use_graphs, autotune=autotune, schedule=schedule,
                                wait_budget_ms=wait_budget_ms)
    keep, outs, tickets = [], [], []
    try:
        for sp in specs:
            C = np.zeros(sp["n"] * sp["n"], np.float64 if sp["prec"] == 0 else np.float32)
            r, k = ebit.make_request(C_out=C, **sp)
            keep.append(k)
            outs.append(C)
            tickets.append(ebit.ebit_submit(s, r))
        res = ebit.wait_all(s, tickets)
        stats = ebit.ebit_server_stats_get(s)
    finally:
        ebit.ebit_server_destroy(s)
    return [res[t] for t in tickets], outs, stats


def test_alone_equals_in_the_mix():
    specs = _mix()
    fps = [ebit.ebit_footprint(sp["n"], sp["n"], 1.0 / sp["n"], sp["prec"]) for sp in specs]
    budget = int(2.5 * max(fps)) + (8 << 20)       # only a few fit at once: requests queue
    mixed, Cm, stats = _run(specs, budget)
    assert stats["batch_steps"] < sum(sp["steps"] for sp in specs)   # steps were shared
    assert any(r["queue_ms"] > 0.0 for r in mixed)
    for sp, rm, cm in zip(specs, mixed, Cm):
        assert rm["status"] == 0 and rm["steps"] == sp["steps"]
        alone, Ca, _ = _run([sp], budget)
        ra = alone[0]
        assert ra["area"] == rm["area"] and ra["area0"] == rm["area0"]
        assert np.array_equal(Ca[0], cm)
        assert np.array_equal(ra["counters"], rm["counters"])
        assert rm["counters"][ebit.D_INVARIANT] == 0 and rm["counters"][ebit.D_CFL] == 0


_SOLO = {}


def _solo(i, sp, budget):
    """The result of spec i run alone (cached across tests)."""
    if i not in _SOLO:
        r, C, _ = _run([sp], budget)
        _SOLO[i] = (r[0], C[0])
    return _SOLO[i]


def _assert_unchanged(specs, results, outs, budget, skip=()):
    for i, (sp, rm, cm) in enumerate(zip(specs, results, outs)):
        if i in skip:
            continue
        ra, ca = _solo(i, sp, budget)
        assert rm["status"] == 0 and rm["steps"] == sp["steps"]
        assert ra["area"] == rm["area"] and np.array_equal(ca, cm)
        assert np.array_equal(ra["counters"], rm["counters"])


def test_failing_request_leaves_the_others_unchanged():
    """One request raises a CFL violation mid-run (fault injection: from its
    5th step its dt is 4x, taking markers up to two cells per sweep): it
    stops after that step with EBIT_ECFL, and every other request of the mix
    returns exactly its solo result."""
    specs = _mix()
    bad = dict(specs[1])
    bad.update(steps=40, fault_after=5, fault_dt_factor=4.0)
    mixed = specs + [bad]
    fps = [ebit.ebit_footprint(sp["n"], sp["n"], 1.0 / sp["n"], sp["prec"]) for sp in specs]
    budget = int(3.5 * max(fps)) + (8 << 20)
    res, outs, _ = _run(mixed, budget)
    rb = res[-1]
    assert rb["status"] == ebit.EBIT_ECFL
    assert rb["steps"] == 6 and rb["counters"][ebit.D_CFL] > 0
    _assert_unchanged(specs, res[:-1], outs[:-1], budget)


@pytest.mark.parametrize("sched", [ebit.EBIT_SCHED_PERSISTENT_LARGEST_FIRST,
                                   ebit.EBIT_SCHED_PERSISTENT_INTERLEAVED])
def test_wait_that_runs_out_stops_only_its_request(sched):
    """Persistent batch steps: from its 4th step one grid's second-sweep
    tiles wait for one more first-sweep tile than there are (fault
    injection from the host; nothing ever sets the count they wait for).
    Each wait gives up after the 20 ms budget, the tile is skipped, and the
    request stops after that step with EBIT_ETIMEOUT; the batch step ends,
    the context stays usable, and every other request of the mix returns
    exactly its solo result."""
    specs = _mix()
    bad = dict(specs[1])
    bad.update(steps=40, fault_after=3, fault_wait=True)
    fps = [ebit.ebit_footprint(sp["n"], sp["n"], 1.0 / sp["n"], sp["prec"]) for sp in specs]
    budget = int(3.5 * max(fps)) + (8 << 20)
    res, outs, stats = _run(specs + [bad], budget, autotune=False, schedule=sched, wait_budget_ms=20)
    assert stats["schedule"] == sched
    rb = res[-1]
    assert rb["status"] == ebit.EBIT_ETIMEOUT and rb["steps"] == 4
    _assert_unchanged(specs, res[:-1], outs[:-1], budget)


def test_cancel_queued_and_running_requests():
    """A request cancelled while queued never runs; one cancelled while
    running stops before the next batch step with the steps it has done; both
    report EBIT_ECANCELLED and the other requests return their solo
    results.  A finished or unknown ticket cannot be cancelled."""
    specs = _mix()
    long_run = dict(specs[0])
    long_run.update(steps=100000)   # runs until cancelled
    queued = dict(specs[2])
    fps = [ebit.ebit_footprint(sp["n"], sp["n"], 1.0 / sp["n"], sp["prec"]) for sp in specs]
    budget = int(1.5 * max(fps)) + (8 << 20)      # the last request waits in the queue
    s = ebit.ebit_server_create(budget)
    keep, outs, tickets = [], [], []
    try:
        for sp in [long_run] + specs + [queued]:
            C = np.zeros(sp["n"] * sp["n"], np.float64 if sp["prec"] == 0 else np.float32)
            r, k = ebit.make_request(C_out=C, **sp)
            keep.append(k)
            outs.append(C)
            tickets.append(ebit.ebit_submit(s, r))
        ebit.ebit_cancel(s, tickets[-1])           # still queued behind the budget
        import time
        t0 = time.time()
        while ebit.ebit_server_stats_get(s)["batch_steps"] < 5 and time.time() - t0 < 60:
            time.sleep(0.002)
        ebit.ebit_cancel(s, tickets[0])            # running
        res = ebit.wait_all(s, tickets)
        with pytest.raises(ebit.EbitError):
            ebit.ebit_cancel(s, tickets[1])        # finished
        with pytest.raises(ebit.EbitError):
            ebit.ebit_cancel(s, 987654321)         # unknown
    finally:
        ebit.ebit_server_destroy(s)
    r0, rq = res[tickets[0]], res[tickets[-1]]
    assert r0["status"] == ebit.EBIT_ECANCELLED and 0 < r0["steps"] < 100000
    assert rq["status"] == ebit.EBIT_ECANCELLED and rq["steps"] == 0
    _assert_unchanged(specs, [res[t] for t in tickets[1:-1]], outs[1:-1], budget)


def test_graphs_and_plain_launches_agree():
    specs = _mix()[:3]
    a, Ca, _ = _run(specs, 8 << 30, use_graphs=True)
    b, Cb, _ = _run(specs, 8 << 30, use_graphs=False)
    for ra, rb, ca, cb in zip(a, b, Ca, Cb):
        assert ra["area"] == rb["area"] and np.array_equal(ca, cb)


def test_results_do_not_depend_on_the_cta_schedule():
    """Every fixed CTA schedule and the autotuned one give identical results;
    with all grids admitted at once the autotuner times every schedule."""
    specs = _mix()
    for sp in specs:
        sp["steps"] = max(sp["steps"], 3 * ebit.EBIT_SCHED_COUNT)
    tuned, Ct, stats = _run(specs, 8 << 30, autotune=True)
    assert stats["tuned_sets"] >= 1
    assert all(t > 0.0 for t in stats["tune_ms"])
    assert 0 <= stats["schedule"] < ebit.EBIT_SCHED_COUNT
    for sched in range(ebit.EBIT_SCHED_COUNT):
        fixed, Cf, st = _run(specs, 8 << 30, autotune=False, schedule=sched)
        assert st["schedule"] == sched and st["tuned_sets"] == 0
        for rt, rf, ct, cf in zip(tuned, fixed, Ct, Cf):
            assert rt["area"] == rf["area"] and np.array_equal(ct, cf)
            assert np.array_equal(rt["counters"], rf["counters"])


def test_flagged_requests_do_not_depend_on_the_schedule():
    """Plain, straight-line (EBIT_FIT_LINE) and generalised-HF requests in
    both precisions, served together under each fixed schedule (two sweep
    launches or one persistent launch, three orders): every request's
    fractions, area and counters are the same under all six."""
    rng = W.Rng(4242)
    specs = []
    for prec in (0, 1):
        for flags, n in ((0, 70), (ebit.EBIT_FIT_LINE, 90), (ebit.EBIT_CURV_GHF, 110)):
            dx = 1.0 / n
            circles = W.place_circles(rng, 8, 3 * dx, 0.1, 2 * dx, lambda x, y, r: True, max_tries=80)
            specs.append(dict(n=n, circles=circles, field=ebit.EBIT_FIELD_ROTATION, prec=prec, steps=15,
                              cfl=0.5, period=1.0, omega=2 * math.pi, centre=(0.5, 0.5), drift=(0.1, 0.05),
                              flags=flags))
    base, Cb, _ = _run(specs, 8 << 30, autotune=False, schedule=ebit.EBIT_SCHED_LARGEST_FIRST)
    assert all(r["status"] == 0 and r["steps"] == 15 for r in base)
    for sched in range(1, ebit.EBIT_SCHED_COUNT):
        res, C, st = _run(specs, 8 << 30, autotune=False, schedule=sched)
        assert st["schedule"] == sched
        for rb, r, cb, c in zip(base, res, Cb, C):
            assert r["status"] == 0 and r["area"] == rb["area"] and np.array_equal(c, cb)
            assert np.array_equal(r["counters"], rb["counters"])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_served_rotation_matches_oracle(prec):
    n, steps, cfl = 72, 30, 0.5
    omega, centre, drift = 2 * math.pi, (0.5, 0.5), (0.3, 0.1)
    circles = np.array([[0.42, 0.55, 0.11], [0.6, 0.3, 0.07]])
    C = np.zeros(n * n, np.float64 if prec == 0 else np.float32)
    s = ebit.ebit_server_create(4 << 30)
    try:
        r, keep = ebit.make_request(n, circles, ebit.EBIT_FIELD_ROTATION, steps, cfl, prec,
                                    omega=omega, centre=centre, drift=drift, C_out=C)
        res = ebit.wait_all(s, [ebit.ebit_submit(s, r)])
        res = list(res.values())[0]
    finally:
        ebit.ebit_server_destroy(s)
    dx = 1.0 / n
    umax = 0.0
    for a in (0, 1):
        for b in (0, 1):
            umax = max(umax, abs(-omega * (b - centre[1]) + drift[0]), abs(omega * (a - centre[0]) + drift[1]))
    dt = cfl * dx / umax
    f = W.rotation_field(n, n, dx, omega, centre, drift)
    S = oracle.init(n, n, dx, W.circle_scene(circles), prec)
    _, A0 = oracle.fraction(S)
    for k in range(steps):
        out = oracle.step(S, f.u, f.v, dt)
    assert res["status"] == 0
    assert abs(res["area0"] - A0) <= 1e-12 * A0
    assert abs(res["area"] - out["area"]) <= 1e-12 * out["area"]
    got = C.reshape(n, n).astype(np.float64)
    if prec == 1:
        assert np.array_equal(got, out["C"])
    else:
        assert np.max(np.abs(got - out["C"])) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_served_degenerate_grid_sizes_match_oracle(prec):
    """Grids of 1, 2, 3, 31, 33 and 65 cells a side (a single tile, ragged
    tile edges, one past a tile) served together in one batch: each equals
    the oracle's run of the same rotation steps."""
    sides, steps, cfl = (1, 2, 3, 31, 33, 65), 6, 0.5
    omega, centre, drift = 2 * math.pi, (0.5, 0.5), (0.2, -0.1)
    circles = np.array([[0.5, 0.5, 0.3], [0.3, 0.7, 0.12]])
    outs, keep, tickets = [], [], []
    s = ebit.ebit_server_create(4 << 30)
    try:
        for n in sides:
            C = np.zeros(n * n, np.float64 if prec == 0 else np.float32)
            r, k = ebit.make_request(n, circles, ebit.EBIT_FIELD_ROTATION, steps, cfl, prec,
                                     omega=omega, centre=centre, drift=drift, C_out=C)
            keep.append(k)
            outs.append(C)
            tickets.append(ebit.ebit_submit(s, r))
        res = ebit.wait_all(s, tickets)
    finally:
        ebit.ebit_server_destroy(s)
    umax = 0.0
    for a in (0, 1):
        for b in (0, 1):
            umax = max(umax, abs(-omega * (b - centre[1]) + drift[0]), abs(omega * (a - centre[0]) + drift[1]))
    for n, t, C in zip(sides, tickets, outs):
        dx = 1.0 / n
        dt = cfl * dx / umax
        f = W.rotation_field(n, n, dx, omega, centre, drift)
        S = oracle.init(n, n, dx, W.circle_scene(circles), prec)
        for _ in range(steps):
            out = oracle.step(S, f.u, f.v, dt)
        r = res[t]
        assert r["status"] == 0 and r["steps"] == steps, n
        assert abs(r["area"] - out["area"]) <= 1e-12 * max(out["area"], 1e-300), n
        got = C.reshape(n, n).astype(np.float64)
        if prec == 1:
            assert np.array_equal(got, out["C"]), n
        else:
            assert np.max(np.abs(got - out["C"])) <= 1e-12, n


def test_vortex_request_returns_to_its_shape():
    """A time-reversed vortex request (period = steps * dt) comes back with a
    small area error, as in the single-grid tests."""
    n = 64
    steps = 128
    s = ebit.ebit_server_create(4 << 30)
    try:
        r, keep = ebit.make_request(n, [(0.5, 0.75, 0.15)], ebit.EBIT_FIELD_VORTEX, steps, 0.5, 0,
                                    period=steps * 0.5 / n)
        res = list(ebit.wait_all(s, [ebit.ebit_submit(s, r)]).values())[0]
    finally:
        ebit.ebit_server_destroy(s)
    assert res["status"] == 0 and res["e_area"] < 5e-2


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_served_generalised_hf_matches_oracle(prec):
    """A request with EBIT_CURV_GHF, served beside plain requests: its
    fractions equal the oracle's and its fallback counters (summed over the
    steps) equal the oracle's; the plain requests are unaffected."""
    n, steps, cfl = 96, 12, 0.5
    omega, centre, drift = 2 * math.pi, (0.5, 0.5), (0.2, -0.1)
    rng = W.Rng(77)
    dx = 1.0 / n
    circles = W.place_circles(rng, 60, 2.5 * dx, 5 * dx, 2 * dx, lambda x, y, r: True)
    C = np.zeros(n * n, np.float64 if prec == 0 else np.float32)
    Cp = np.zeros(n * n, np.float64 if prec == 0 else np.float32)
    s = ebit.ebit_server_create(4 << 30)
    try:
        r, keep = ebit.make_request(n, circles, ebit.EBIT_FIELD_ROTATION, steps, cfl, prec, omega=omega,
                                    centre=centre, drift=drift, C_out=C, flags=ebit.EBIT_CURV_GHF)
        rp, keep2 = ebit.make_request(n, circles, ebit.EBIT_FIELD_ROTATION, steps, cfl, prec, omega=omega,
                                      centre=centre, drift=drift, C_out=Cp)
        tg, tp = ebit.ebit_submit(s, r), ebit.ebit_submit(s, rp)
        res = ebit.wait_all(s, [tg, tp])
    finally:
        ebit.ebit_server_destroy(s)
    rg, rpl = res[tg], res[tp]
    assert rg["status"] == 0 and rpl["status"] == 0
    umax = 0.0
    for a in (0, 1):
        for b in (0, 1):
            umax = max(umax, abs(-omega * (b - centre[1]) + drift[0]), abs(omega * (a - centre[0]) + drift[1]))
    dt = cfl * dx / umax
    f = W.rotation_field(n, n, dx, omega, centre, drift)
    S = oracle.init(n, n, dx, W.circle_scene(circles), prec)
    tot = np.zeros(oracle.NCOUNTERS, np.int64)
    for k in range(steps):
        out = oracle.step(S, f.u, f.v, dt, ghf=True)
        tot += out["counters"]
    got = C.reshape(n, n).astype(np.float64)
    if prec == 1:
        assert np.array_equal(got, out["C"])
    else:
        assert np.max(np.abs(got - out["C"])) <= 1e-12
    assert np.array_equal(np.asarray(rg["counters"])[[ebit.D_HF_INVALID, ebit.D_HF_OTHER, ebit.D_HF_MIXED,
                                                      ebit.D_HF_MARKERS]],
                          tot[[ebit.D_HF_INVALID, ebit.D_HF_OTHER, ebit.D_HF_MIXED, ebit.D_HF_MARKERS]])
    assert tot[ebit.D_HF_MIXED] + tot[ebit.D_HF_MARKERS] > 0
    # the plain request: same fractions, no fallbacks counted
    assert np.array_equal(Cp, C)
    assert np.asarray(rpl["counters"])[ebit.D_HF_OTHER:ebit.D_HF_MARKERS + 1].sum() == 0
    assert rpl["counters"][ebit.D_HF_INVALID] == rg["counters"][ebit.D_HF_INVALID]
