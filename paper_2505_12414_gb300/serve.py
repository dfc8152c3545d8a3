"""Request loop for serving fits with continuous batching.

Requests (model kind, events, start point, arrival time) are admitted into the servers of
their model kind as slots and pool memory free up.  The loop keeps a couple of device steps
queued on every server with fits in it (servers run on their own CUDA streams, so their steps
overlap on the device) and collects finished fits as soon as their done flags are up, so the
device does not wait for the host between steps and admissions and collections overlap the
steps of the other fits.  The loop only schedules: all fitting runs in the library
(nll_server_*, or fit_minimise for a lone request on an idle loop).
"""
import collections
import time

import numpy as np


class Request:
    __slots__ = ("rid", "kind", "columns", "theta0", "arrival", "admitted", "done", "result")

    def __init__(self, rid, kind, columns, theta0, arrival):
        self.rid = rid
        self.kind = kind
        self.columns = columns
        self.theta0 = theta0
        self.arrival = arrival
        self.admitted = None
        self.done = None
        self.result = None


def by_kind(request):
    """Default routing: one server per model kind."""
    return request.kind


def by_kind_and_size(limit):
    """Routing by model kind and sample size: fits of at most `limit` events go to their own
    servers, so their steps (which cost about the events of all the fits in a server) stay
    short while the large fits run on the other servers' streams."""

    def route(request):
        return (request.kind, len(request.columns[0]) <= limit)

    return route


def serve(servers, requests, steps_per_iter=2, realtime=True, max_queued=2, phases=None, route=by_kind,
          admit_all=True, direct=None):
    """Run `requests` (sorted by arrival, seconds from start) through `servers` {key: Server},
    each request going to servers[route(request)].

    With realtime=True requests become visible at their arrival times on the wall clock;
    otherwise all are queued at once.  Every server with fits in it gets `steps_per_iter` more
    steps whenever fewer than `max_queued` of its steps are still in flight; the loop tops the
    step queues up between single admissions and collections, so that the device keeps
    working while the host admits and collects.  With admit_all every server takes as many
    waiting requests as it has room for in each pass of the loop (fits that start together
    share their steps); otherwise one per pass.  If `phases` is a dict, the host time spent in
    admission (submit), step queueing (step), progress queries and collection (poll) is added
    to it, in seconds, with the number of steps queued.  With `direct` ({key: (Model, fit
    keyword arguments)}, keyed as the servers), a request that finds every server idle and no
    other request waiting is fitted at once through the single-fit path of its key's model
    (nll_load_events + fit_minimise) instead of being admitted: a lone fit would otherwise pay
    the device loop's per-step latency for every step, where batching has nothing to share
    (the time goes to direct_s).  Returns the requests with admitted/done times and results
    filled in."""
    clock = time.perf_counter
    acc = phases if phases is not None else {}
    for key in ("admit_s", "step_s", "progress_s", "collect_s", "direct_s", "steps", "direct_fits"):
        acc.setdefault(key, 0.0)
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    queues = {k: collections.deque() for k in servers}
    inflight = {k: {} for k in servers}
    finished = {k: 0 for k in servers}
    left = len(requests)
    t0 = clock()

    def feed():
        """Top up the step queues of the servers with fits in them; note finished fits."""
        for k, srv in servers.items():
            if not inflight[k]:
                continue
            c0 = clock()
            queued, finished[k] = srv.progress()
            c1 = clock()
            acc["progress_s"] += c1 - c0
            if queued < max_queued:
                srv.step(steps_per_iter)
                acc["steps"] += steps_per_iter
                acc["step_s"] += clock() - c1

    while left:
        now = clock() - t0
        while pending and (not realtime or pending[0].arrival <= now):
            r = pending.popleft()
            queues[route(r)].append(r)
        if direct is not None and not any(inflight.values()) and sum(len(q) for q in queues.values()) == 1:
            k = next(k for k, q in queues.items() if q)
            if k in direct:  # the lone request: the single-fit path
                r = queues[k].popleft()
                model, kwargs = direct[k]
                c0 = clock()
                r.admitted = c0 - t0
                model.load(r.columns)
                r.result = model.fit(r.theta0, **kwargs)
                r.done = clock() - t0
                acc["direct_s"] += clock() - c0
                acc["direct_fits"] += 1
                left -= 1
                continue
        feed()
        for k, srv in servers.items():  # admissions, feeding the step queues after each
            q = queues[k]
            while q:
                c0 = clock()
                rid = srv.submit(q[0].columns, q[0].theta0)
                acc["admit_s"] += clock() - c0
                if rid is None:
                    break
                r = q.popleft()
                r.admitted = clock() - t0
                inflight[k][rid] = r
                feed()
                if not admit_all:
                    break
        for k, srv in servers.items():
            if finished[k]:
                c0 = clock()
                done = srv.poll()
                acc["collect_s"] += clock() - c0
                finished[k] = 0
                for rid, res in done:
                    r = inflight[k].pop(rid)
                    r.done = clock() - t0
                    r.result = res
                    left -= 1
                feed()
        if not any(inflight.values()) and pending and realtime:
            time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.01)))
    return requests


def serve_sequential(models, requests, fit_kwargs):
    """The plain path: one fit at a time in arrival order on the GPU ({kind: Model})."""
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        r.admitted = time.perf_counter() - t0
        m = models[r.kind]
        m.load(r.columns)
        r.result = m.fit(r.theta0, **fit_kwargs[r.kind])
        r.done = time.perf_counter() - t0
    return requests


def latency_summary(requests):
    lat = np.array([r.done - r.arrival for r in requests])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"n": len(requests), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "fits_per_s": len(requests) / span if span > 0 else None}
