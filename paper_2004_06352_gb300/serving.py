"""Driver for the native request loop (lens_server_* in the C ABI).

The scheduling -- admission by device memory, continuous admission onto
stream slots, retirement -- happens in the library; this module only builds
request streams, submits them at their arrival times, polls
lens_server_progress and summarises latencies.

Workload shape (mixed serving stream): 60 % Hessian maps with side drawn from
{512, 1024, 2048, 4096, 8192} and a resident model of 10-2000 potentials
(log-uniform), 40 % source-plane chi2 batches of 16-4096 parameter sets
(log-uniform); Poisson arrivals.
"""
from __future__ import annotations

import time

import numpy as np

from . import api
from . import inputs as I

MAP_SIDES = (512, 1024, 2048, 4096, 8192)


def poisson_arrivals(n, rate, seed):
    """Arrival times (s) of n requests at `rate` per second."""
    return np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, n))


def resident_models(n_models, seed, n_range=(10, 2000)):
    """Cluster-like models: 2 cluster-scale halos plus luminosity-scaled
    members, total potential count log-uniform in n_range."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_models):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        n = max(n, 3)
        m = I.cfg2_model(seed=1000 + k, n_members=n - 2)
        out.append(m)
    return out


def mixed_requests(n, seed, n_models, p_map=0.6, p_range=(16, 4096), sides=MAP_SIDES):
    """n request descriptors: ("map", model, side) or ("chi2", model, P, seed)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        mi = int(rng.integers(0, n_models))
        if rng.uniform() < p_map:
            reqs.append(("map", mi, int(sides[rng.integers(0, len(sides))])))
        else:
            P = int(round(np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1])))))
            reqs.append(("chi2", mi, P, int(rng.integers(0, 2**31))))
    return reqs


def percentiles(lat_ms):
    a = np.asarray(lat_ms, dtype=np.float64)
    if a.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)), "mean_ms": float(a.mean())}


class PinnedPool:
    """Reusable page-locked host buffers keyed by (shape, dtype).  `misses`
    counts buffers that had to be page-locked on demand (slow: the call
    blocks the submitting thread).  Vectors (chi2 results) come as the first
    n elements of a buffer of at least VEC_CAP, so that requests of any batch
    size share the same buffers."""

    VEC_CAP = 4096

    def __init__(self):
        self.free = {}
        self.misses = 0

    def take(self, shape, dtype):
        import torch
        key = (tuple(shape), dtype)
        lst = self.free.get(key)
        if lst:
            return lst.pop()
        self.misses += 1
        return torch.empty(shape, dtype=dtype, pin_memory=True)

    def take_vec(self, n, dtype):
        return self.take((max(n, self.VEC_CAP),), dtype)[:n]

    def give(self, t):
        if t._base is not None:  # a vector handed out by take_vec: its whole buffer
            t = t._base
        self.free.setdefault((tuple(t.shape), t.dtype), []).append(t)


class Session:
    """Resident models and constraint sets of a serving run."""

    def __init__(self, ctx, models, precision=api.LENS_MIXED):
        self.ctx = ctx
        self.models = models
        self.precision = precision
        self.mids = [ctx.model_upload(m) for m in models]
        self.csets = []
        for k, m in enumerate(models):
            cons = I.random_constraints(100, seed=500 + k, field=60)
            self.csets.append(ctx.cset_create(self.mids[k], cons, (0, 1)))

    def submit(self, server, req, pool):
        import torch
        if req[0] == "map":
            side = req[2]
            buf = pool.take((6, side, side), torch.float32 if self.precision == api.LENS_MIXED else torch.float64)
            t = server.submit_map(self.mids[req[1]], I.grid(side), 1.0, self.precision, True, buf)
        else:
            P = req[2]
            params = I.perturbed_params(self.models[req[1]], (0, 1), P, seed=req[3])
            buf = pool.take_vec(P, torch.float64)
            t = server.submit_chi2_source(self.csets[req[1]], params, 0, buf)
        return t, buf


def run_stream(server, session, reqs, arrivals=None, pool=None, timeout_s=600.0, max_outstanding=None,
               keep_results=True):
    """Submit reqs at their arrival times (as fast as allowed if arrivals is
    None: at most max_outstanding submitted and not yet completed), poll
    until every ticket completes.  Latency runs from the request's arrival
    (its submission when arrivals is None) to its completion: the library's
    submit-to-completion time plus how late this loop submitted it.  Returns
    (latencies_ms, wall_s, completions, buffers by ticket)."""
    pool = pool or PinnedPool()
    t0 = time.perf_counter()
    pending, bufs, done = {}, {}, []
    k = 0
    n = len(reqs)
    while k < n or pending:
        now = time.perf_counter() - t0
        while k < n and (arrivals is None or arrivals[k] <= now) and (
                max_outstanding is None or len(pending) < max_outstanding):
            late_ms = 0.0 if arrivals is None else 1e3 * max(0.0, time.perf_counter() - t0 - arrivals[k])
            t, buf = session.submit(server, reqs[k], pool)
            pending[t] = (buf, late_ms)
            k += 1
        for (ticket, status, qms, lms) in server.progress():
            if status != api.LENS_OK:
                raise RuntimeError(f"request {ticket} failed: {api.strerror(status)}")
            buf, late_ms = pending.pop(ticket)
            bufs[ticket] = buf
            done.append((ticket, qms, lms + late_ms))
            if keep_results is False:
                pool.give(bufs.pop(ticket))
        if now > timeout_s:
            raise TimeoutError(f"serving stream did not finish within {timeout_s} s")
        if not done or k < n:
            time.sleep(0)  # yield
    wall = time.perf_counter() - t0
    return [d[2] for d in done], wall, done, bufs
