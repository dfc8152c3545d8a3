"""Serving with continuous batching: each fit gives the same result alone and in the mix,
admission respects the pool budget, and served fits match one-at-a-time fits."""
import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D


def opts(kind):
    n = 4 if kind == M1 else 18
    lo, hi = np.zeros(n), np.zeros(n)
    hi[-1] = 1.0
    step = np.array([2.0, 1.0, 2e-4, 0.02]) if kind == M1 else np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    return dict(lo=lo, hi=hi, step=step, tol_edm=1e-12, strategy=1, hessian=1)


def make_requests(n, stream0):
    from paper_2505_12414_gb300.serve import Request

    rs = synth.Stream(stream0, 1)
    sizes = np.exp(np.log(1000) + (np.log(8000) - np.log(1000)) * rs.uniform(n)).astype(int)
    reqs = []
    for i in range(n):
        kind = M1 if i % 2 == 0 else M4
        cols = synth.mass1d(int(sizes[i]), stream=stream0 + i) if kind == M1 else synth.kstar4d(int(sizes[i]), stream=stream0 + i)
        th0 = (synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D) + 0.3 * opts(kind)["step"]
        reqs.append(Request(i, kind, cols, th0, 0.0))
    return reqs


def servers(g, slots, pool):
    return {k: g.Server(k, synth.RANGES_1D if k == M1 else synth.RANGES_4D, slots, pool, 1024, **opts(k))
            for k in (M1, M4)}


def test_results_are_the_same_alone_and_in_the_mix(gpu_lib):
    from paper_2505_12414_gb300.serve import serve

    mix = make_requests(10, 9100)
    srv = servers(gpu_lib, 8, 200000)
    serve(srv, mix, realtime=False)
    for s in srv.values():
        s.close()
    alone = make_requests(10, 9100)
    for r in alone:
        srv = servers(gpu_lib, 1, 20000)
        serve(srv, [r], realtime=False)
        for s in srv.values():
            s.close()
    for a, b in zip(mix, alone):
        assert a.result["status"] == 0 and b.result["status"] == 0
        assert np.array_equal(a.result["theta"], b.result["theta"]), (a.rid, a.result["theta"] - b.result["theta"])
        assert np.array_equal(a.result["err"], b.result["err"])
        assert a.result["nll"] == b.result["nll"]


def test_admission_by_pool_budget(gpu_lib):
    s = gpu_lib.Server(M1, synth.RANGES_1D, 4, 5000, 1024, **opts(M1))
    c1, c2 = synth.mass1d(3000, stream=1), synth.mass1d(3000, stream=2)
    id1 = s.submit(c1, synth.TRUTH_1D)
    assert id1 is not None
    assert s.submit(c2, synth.TRUTH_1D) is None  # 3000 + 3000 events exceed the 5000-event pool
    st = s.status()
    assert st["busy"] == 1 and st["free_slots"] == 3 and st["free_events"] == 2000
    done = []
    for _ in range(500):
        s.step(4)
        s.sync()  # poll does not wait for the steps in flight
        done += s.poll()
        if done:
            break
    assert [d[0] for d in done] == [id1] and done[0][1]["status"] == 0
    assert s.submit(c2, synth.TRUTH_1D) is not None
    s.close()


def test_served_fits_match_model_fits(gpu_lib):
    from paper_2505_12414_gb300.serve import serve

    reqs = make_requests(4, 9200)
    srv = servers(gpu_lib, 4, 100000)
    serve(srv, reqs, realtime=False)
    for r in reqs:
        m = gpu_lib.Model(r.kind, synth.RANGES_1D if r.kind == M1 else synth.RANGES_4D)
        m.load(r.columns)
        o = dict(opts(r.kind))
        o["tol_edm"] = 1e-14
        ref = m.fit(r.theta0, **o)
        m.close()
        pull = (r.result["theta"] - ref["theta"]) / ref["err"]
        assert np.max(np.abs(pull)) < 1e-4, pull  # served fits stop at EDM 1e-12
    for s in srv.values():
        s.close()


def opts_analytic(kind):
    o = opts(kind)
    o.update(strategy=2, hessian=2)
    return o


def test_analytic_served_fits(gpu_lib):
    # served fits with the analytic start matrix (at admission) and the polished analytic
    # covariance (at poll): each result is the same alone and in the mix, and matches the
    # single-sample analytic fit
    from paper_2505_12414_gb300.serve import serve

    def run(reqs, slots, pool):
        srv = {k: gpu_lib.Server(k, synth.RANGES_1D if k == M1 else synth.RANGES_4D, slots, pool, 1024,
                                 **opts_analytic(k)) for k in (M1, M4)}
        serve(srv, reqs, realtime=False)
        for s in srv.values():
            s.close()

    mix = make_requests(8, 9300)
    run(mix, 8, 200000)
    alone = make_requests(8, 9300)
    for r in alone:
        run([r], 1, 20000)
    for a, b in zip(mix, alone):
        assert a.result["status"] == 0 and b.result["status"] == 0
        assert np.array_equal(a.result["theta"], b.result["theta"])
        assert np.array_equal(a.result["err"], b.result["err"])
    for r in mix:
        ranges = synth.RANGES_1D if r.kind == M1 else synth.RANGES_4D
        m = gpu_lib.Model(r.kind, ranges).load(r.columns)
        s = m.fit(r.theta0, **opts_analytic(r.kind))
        m.close()
        assert s["status"] == 0
        assert np.max(np.abs((r.result["theta"] - s["theta"]) / s["err"])) < 1e-5
        np.testing.assert_allclose(r.result["err"], s["err"], rtol=1e-4)
        assert r.result["n_eval"] < 40


def test_admission_rejects_events_outside_the_ranges(gpu_lib):
    # the range check runs on the device at admission; a rejected request frees its pool range
    s = gpu_lib.Server(M4, synth.RANGES_4D, 2, 6000, 1024, **opts(M4))
    cols = [c.copy() for c in synth.kstar4d(3000, stream=77)]
    cols[2][1234] = 1.2  # cos theta_K outside [-1, 1]
    with pytest.raises(gpu_lib.NLLError) as e:
        s.submit(cols, synth.TRUTH_4D)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    st = s.status()
    assert st["busy"] == 0 and st["free_events"] == 6000
    cols[2][1234] = 0.2
    assert s.submit(cols, synth.TRUTH_4D) is not None
    s.close()


def test_progress_and_non_blocking_poll(gpu_lib):
    s = gpu_lib.Server(M1, synth.RANGES_1D, 4, 20000, 1024, **opts(M1))
    assert s.progress() == (0, 0) and s.poll() == []
    rid = s.submit(synth.mass1d(5000, stream=31), synth.TRUTH_1D)
    s.step(3)
    queued, finished = s.progress()
    assert 0 <= queued <= 3 and finished in (0, 1)
    done = []
    for _ in range(400):
        queued, finished = s.progress()
        if finished:
            done += s.poll()
            break
        if queued < 2:
            s.step(2)
    assert [d[0] for d in done] == [rid] and done[0][1]["status"] == 0
    assert s.progress()[1] == 0
    s.sync()
    assert s.progress() == (0, 0)
    s.close()


def test_cancel_frees_the_slot_and_the_pool_range(gpu_lib):
    s = gpu_lib.Server(M4, synth.RANGES_4D, 2, 12000, 1024, **opts(M4))
    c1, c2, c3 = (synth.kstar4d(5000, stream=k) for k in (41, 42, 43))
    r1 = s.submit(c1, synth.TRUTH_4D)
    r2 = s.submit(c2, synth.TRUTH_4D)
    assert s.submit(c3, synth.TRUTH_4D) is None  # both slots busy
    s.step(2)
    s.cancel(r1)  # withdrawn while its steps run
    st = s.status()
    assert st["busy"] == 1 and st["free_slots"] == 1 and st["free_events"] == 12000 - 5000
    with pytest.raises(gpu_lib.NLLError) as e:
        s.cancel(r1)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    r3 = s.submit(c3, synth.TRUTH_4D)  # the freed slot and range take the next request
    assert r3 is not None
    got = {}
    for _ in range(2000):
        s.step(2)
        s.sync()
        for rid, res in s.poll():
            got[rid] = res
        if len(got) == 2:
            break
    assert set(got) == {r2, r3} and all(v["status"] == 0 for v in got.values())
    # the fit admitted into the cancelled fit's slot gives what it gives alone
    alone = gpu_lib.Server(M4, synth.RANGES_4D, 1, 6000, 1024, **opts(M4))
    ra = alone.submit(c3, synth.TRUTH_4D)
    res = []
    for _ in range(2000):
        alone.step(2)
        alone.sync()
        res += alone.poll()
        if res:
            break
    assert np.array_equal(res[0][1]["theta"], got[r3]["theta"])
    alone.close()
    s.close()


def test_routing_by_size_class_gives_the_same_results(gpu_lib):
    # each fit's result depends on its own events only: serving the same requests with small
    # and large fits on separate servers gives the same bits as one server per model kind
    from paper_2505_12414_gb300.serve import by_kind_and_size, serve

    per_kind = make_requests(8, 9400)
    srv = servers(gpu_lib, 8, 200000)
    serve(srv, per_kind, realtime=False)
    for s_ in srv.values():
        s_.close()
    routed = make_requests(8, 9400)
    route = by_kind_and_size(3000)
    srv2 = {(k, small): gpu_lib.Server(k, synth.RANGES_1D if k == M1 else synth.RANGES_4D, 8, 200000, 1024, **opts(k))
            for k in (M1, M4) for small in (True, False)}
    serve(srv2, routed, realtime=False, route=route)
    for s_ in srv2.values():
        s_.close()
    assert len({route(r) for r in routed}) > 2  # both size classes took fits
    for a, b in zip(per_kind, routed):
        assert a.result["status"] == 0 and b.result["status"] == 0
        assert np.array_equal(a.result["theta"], b.result["theta"])
        assert np.array_equal(a.result["err"], b.result["err"])


@pytest.mark.parametrize("strategy", [3, 5])
def test_served_fits_with_estimated_start_matrices(gpu_lib, strategy):
    """Served fits whose start matrix comes from a subsample (strategy 3) or a single-precision
    pass (strategy 5): the same result alone and in the mix, and the minimum and covariance of
    the analytic served fit (strategy 2) to within the stopping tolerance."""
    from paper_2505_12414_gb300.serve import serve

    def run(reqs, slots, pool, st):
        srv = {k: gpu_lib.Server(k, synth.RANGES_1D if k == M1 else synth.RANGES_4D, slots, pool, 1024,
                                 **dict(opts_analytic(k), strategy=st, tol_edm=1e-14)) for k in (M1, M4)}
        serve(srv, reqs, realtime=False)
        for s in srv.values():
            s.close()

    mix = make_requests(8, 9400)
    run(mix, 8, 200000, strategy)
    alone = make_requests(8, 9400)
    for r in alone[:3]:
        run([r], 1, 20000, strategy)
    for a, b in zip(mix, alone[:3]):
        assert a.result["status"] == 0 and b.result["status"] == 0
        assert np.array_equal(a.result["theta"], b.result["theta"])
        assert np.array_equal(a.result["err"], b.result["err"])
    ref = make_requests(8, 9400)
    run(ref, 8, 200000, 2)
    for a, r in zip(mix, ref):
        assert r.result["status"] == 0
        # both stop at EDM 1e-14: within sqrt(2e-14) = 1.4e-7 of the uncertainty of the minimum
        assert np.max(np.abs(a.result["theta"] - r.result["theta"]) / r.result["err"]) < 1e-6
        np.testing.assert_allclose(a.result["err"], r.result["err"], rtol=1e-6)


def test_lone_request_takes_the_single_fit_path(gpu_lib):
    """With direct models, a request that finds the loop idle is fitted through fit_minimise
    (the same result as Model.fit, bitwise); requests that arrive together still go through the
    servers."""
    from paper_2505_12414_gb300.serve import serve

    srv = servers(gpu_lib, 4, 100000)
    models = {k: gpu_lib.Model(k, synth.RANGES_1D if k == M1 else synth.RANGES_4D) for k in (M1, M4)}
    direct = {k: (models[k], opts(k)) for k in (M1, M4)}
    lone = make_requests(1, 9500)
    phases = {}
    serve(srv, lone, realtime=False, direct=direct, phases=phases)
    assert phases["direct_fits"] == 1
    ref = gpu_lib.Model(lone[0].kind, synth.RANGES_1D).load(lone[0].columns)
    s = ref.fit(lone[0].theta0, **opts(lone[0].kind))
    ref.close()
    assert np.array_equal(lone[0].result["theta"], s["theta"]) and lone[0].result["nll"] == s["nll"]
    together = make_requests(4, 9510)
    phases = {}
    serve(srv, together, realtime=False, direct=direct, phases=phases)
    assert phases["direct_fits"] == 0
    assert all(r.result["status"] == 0 for r in together)
    for s_ in srv.values():
        s_.close()
    for m in models.values():
        m.close()
