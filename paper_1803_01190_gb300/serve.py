"""Continuous-batching server for many independent N-body simulations.

Requests (one simulation each: initial state, mode, eps, G, dt, number of
KDK steps) are admitted into a resident device pool (`Batch`, the
nbody_batch_* C ABI) as soon as a slot and a contiguous range of particles
are free, advanced together one step per tick in shared launches, and
retired when done; requests that arrive while others are on the GPU join at
the next tick.  All arithmetic runs in the library's CUDA kernels; this
module only schedules.

Autotuner: the launch shape of each mode's force launch (i-particles per
thread, j-segment length) is chosen per load bucket (the mode and the
tick's interactions to within a factor of 8) from the force-kernel time per
interaction measured with CUDA events on the ticks themselves: every
candidate is tried once per bucket, then the fastest is used, with a
periodic re-check of the runner-up.  A shape changes rounding order only.
"""
import collections
import ctypes
import math
import time

import numpy as np

from ._abi import F64E, FP64, MIXED, NbodyError, check, lib

MODES = {"fp64": FP64, "mixed": MIXED, "f64e": F64E}
_CLS = {"fp64": 0, "mixed": 1, "f64e": 2}
_ENOSPC = -6


def _host(a, shape):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(shape)


class Batch:
    """A device pool of `capacity` particles holding up to `max_sims` simulations."""

    def __init__(self, capacity, max_sims, stream=None):
        import torch
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        check(lib.nbody_batch_create(ctypes.byref(h), int(capacity), int(max_sims), ctypes.c_void_p(st)),
              "nbody_batch_create")
        self._h = h
        self.capacity = int(capacity)
        self.max_sims = int(max_sims)

    @staticmethod
    def bytes_per_particle():
        return int(lib.nbody_batch_bytes_per_particle())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.nbody_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, pos, vel, mass, mode="fp64", eps=0.01, G=1.0, dt=1e-3):
        """Slot of the admitted simulation, or None when the pool is full (ENOSPC)."""
        n = int(np.shape(mass)[0])
        pos = _host(pos, (n, 3))
        mass = _host(mass, (n,))
        vel = None if vel is None else _host(vel, (n, 3))
        slot = ctypes.c_int(-1)
        rc = lib.nbody_batch_admit(self._h, n, MODES[mode], float(eps), float(G), float(dt),
                                   ctypes.c_void_p(pos.ctypes.data),
                                   None if vel is None else ctypes.c_void_p(vel.ctypes.data),
                                   ctypes.c_void_p(mass.ctypes.data), 0, ctypes.byref(slot))
        if rc == _ENOSPC:
            return None
        check(rc, "nbody_batch_admit")
        return slot.value

    def evict(self, slot):
        check(lib.nbody_batch_evict(self._h, int(slot)), "nbody_batch_evict")

    def step(self, nticks=1):
        check(lib.nbody_batch_step(self._h, int(nticks)), "nbody_batch_step")

    def sync(self):
        check(lib.nbody_batch_sync(self._h), "nbody_batch_sync")

    def ready(self):
        """True when every queued tick and copy of this pool has finished (non-blocking)."""
        rc = lib.nbody_batch_query(self._h)
        if rc < 0:
            check(rc, "nbody_batch_query")
        return rc == 1

    def slot_info(self, slot):
        n, m, s = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        check(lib.nbody_batch_slot_info(self._h, int(slot), ctypes.byref(n), ctypes.byref(m),
                                        ctypes.byref(s)), "nbody_batch_slot_info")
        return n.value, m.value, s.value

    def get_state(self, slot):
        n = self.slot_info(slot)[0]
        pos, vel = np.empty((n, 3)), np.empty((n, 3))
        t, s = ctypes.c_double(), ctypes.c_int64()
        check(lib.nbody_batch_get_state(self._h, int(slot), ctypes.c_void_p(pos.ctypes.data),
                                        ctypes.c_void_p(vel.ctypes.data), ctypes.byref(t),
                                        ctypes.byref(s), 0), "nbody_batch_get_state")
        return pos, vel, t.value, s.value

    def get_accel(self, slot):
        n = self.slot_info(slot)[0]
        acc, pot = np.empty((n, 3)), np.empty(n)
        check(lib.nbody_batch_get_accel(self._h, int(slot), ctypes.c_void_p(acc.ctypes.data),
                                        ctypes.c_void_p(pot.ctypes.data), 0), "nbody_batch_get_accel")
        return acc, pot

    def diagnostics(self, slot):
        E, K, W = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        P, L = (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
        check(lib.nbody_batch_diagnostics(self._h, int(slot), ctypes.byref(E), ctypes.byref(K),
                                          ctypes.byref(W), P, L), "nbody_batch_diagnostics")
        return {"E": E.value, "K": K.value, "W": W.value, "P": np.array(P[:]), "L": np.array(L[:])}

    def info(self):
        a, u, f = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        check(lib.nbody_batch_info(self._h, ctypes.byref(a), ctypes.byref(u), ctypes.byref(f)),
              "nbody_batch_info")
        return {"active": a.value, "used": u.value, "largest_free": f.value}

    def set_launch(self, mode, ipt, seg):
        check(lib.nbody_batch_set_launch(self._h, MODES[mode], int(ipt), int(seg)),
              "nbody_batch_set_launch")

    def profile(self, enable=True):
        check(lib.nbody_batch_profile(self._h, int(bool(enable))), "nbody_batch_profile")

    def set_fp64_residency(self, blocks_per_sm):
        check(lib.nbody_batch_set_fp64_residency(self._h, int(blocks_per_sm)),
              "nbody_batch_set_fp64_residency")

    def profile_read(self, cap=4096):
        """(tick_ms (k,), force_ms (k,3), interactions (k,3)) for the ticks since the last read;
        columns: FP64, MIXED, F64E force launches."""
        tick = np.zeros(cap)
        force = np.zeros((cap, 3))
        inter = np.zeros((cap, 3))
        k = ctypes.c_int64()
        check(lib.nbody_batch_profile_read(self._h, cap, ctypes.c_void_p(tick.ctypes.data),
                                           ctypes.c_void_p(force.ctypes.data),
                                           ctypes.c_void_p(inter.ctypes.data), ctypes.byref(k)),
              "nbody_batch_profile_read")
        m = min(k.value, cap)
        return tick[:m], force[:m], inter[:m]

    @property
    def launch_count(self):
        return int(lib.nbody_batch_launch_count(self._h))


class Autotuner:
    """Chooses (ipt, seg) per (mode, load bucket) from measured ns per interaction."""

    def __init__(self, candidates=None, trials=1, recheck_every=64):
        self.candidates = candidates or [(ipt, seg) for ipt in (2, 1, 4) for seg in (8192, 2048)]
        self.trials = trials
        self.recheck_every = recheck_every
        self.stats = collections.defaultdict(lambda: collections.defaultdict(list))
        self.picks = collections.Counter()

    @staticmethod
    def bucket(mode, interactions):
        """Load bucket: the mode and the tick's interactions to within a factor of 8."""
        return (mode, int(math.log2(max(interactions, 1.0)) // 3))

    def choose(self, key):
        st = self.stats[key]
        for c in self.candidates:                 # explore: every candidate `trials` times
            if len(st[c]) < self.trials:
                return c
        self.picks[key] += 1
        best = self.best(key)
        if self.recheck_every and self.picks[key] % self.recheck_every == 0:
            ranked = sorted(self.candidates, key=lambda c: np.median(st[c]))
            return ranked[1] if len(ranked) > 1 else best   # re-measure the runner-up
        return best

    def best(self, key):
        st = self.stats[key]
        tried = [c for c in self.candidates if st[c]]
        return min(tried, key=lambda c: np.median(st[c])) if tried else self.candidates[0]

    def record(self, key, cand, ns_per_interaction):
        lst = self.stats[key][cand]
        lst.append(float(ns_per_interaction))
        if len(lst) > 16:
            del lst[0]


class Request:
    """One simulation request.  `make` returns (pos, vel, mass) when called (lazy
    initial conditions); or give pos/vel/mass directly."""

    __slots__ = ("id", "n", "mode", "eps", "G", "dt", "nsteps", "make", "t_arrive", "t_admit",
                 "t_done", "slot", "result", "diag")

    def __init__(self, id, n, mode, eps, G, dt, nsteps, make, t_arrive=0.0):
        self.id, self.n, self.mode, self.eps, self.G, self.dt = id, n, mode, eps, G, dt
        self.nsteps, self.make, self.t_arrive = nsteps, make, t_arrive
        self.t_admit = self.t_done = None
        self.slot = None
        self.result = None
        self.diag = None


class _Pool:
    def __init__(self, mode, capacity, max_sims, launch, kernel=None):
        import torch
        self.mode = mode
        self.kernel = kernel or mode       # the batch mode the pool's simulations run in
        # MIXED ticks are short: give their stream priority so that their blocks are
        # scheduled as soon as an SM has room next to the long FP64 blocks
        self.stream = torch.cuda.Stream(priority=-1 if mode == "mixed" else 0)
        self.batch = Batch(capacity, max_sims, stream=self.stream)
        self.batch.profile(True)
        self.batch.set_launch(self.kernel, *launch)
        self.queue = []
        self.active = {}
        self.inflight = False
        self.chosen = None
        self.ticks_ms = []
        self.ticks = 0


class Server:
    """Admit / tick / retire loop with one resident pool per precision mode.

    FP64 and MIXED simulations live in separate pools, each ticking on its own
    CUDA stream: an FP64 tick is bound by the FP64 pipe and a MIXED tick by
    FP32 issue, so the two run side by side on the same SMs, and the fast
    MIXED ticks do not wait for the slow FP64 ones.  Each pool admits queued
    requests of its mode between its own ticks (first fit by free range and
    slot, with a look-ahead past requests that do not fit yet).

    run(requests, duration) plays an arrival schedule (Request.t_arrive in
    seconds from the start) for at most `duration` seconds of wall time (or
    until every request is done) and returns metrics: per-mode tick latency
    p50/p99 (CUDA events), aggregate Ginteractions/s, admitted, completed and
    queued counts."""

    def __init__(self, capacity, max_sims, autotune=True, launch=None, lookahead=8, keep_state=True,
                 split=None, modes=("fp64", "mixed"), fp64_kernel="fp64"):
        """capacity: particles (split between the pools by `split`) or {mode: particles};
        max_sims: resident simulations per pool, an int or {mode: int}; fp64_kernel:
        "fp64" (binary64 FP64 pipe) or "f64e" (binary64-class float-float on the FP32
        pipes, within the same parity gate) for requests asking for FP64."""
        launch = launch or {"fp64": (2, 4096), "mixed": (2, 8192), "f64e": (2, 4096)}
        split = split or {m: 1.0 / len(modes) for m in modes}
        cap = capacity if isinstance(capacity, dict) else {m: max(1, int(capacity * split[m])) for m in modes}
        ms = max_sims if isinstance(max_sims, dict) else {m: max_sims for m in modes}
        kern = {m: (fp64_kernel if m == "fp64" else m) for m in modes}
        self.pools = {m: _Pool(m, cap[m], ms[m], launch[kern[m]], kern[m]) for m in modes}
        self.tuner = Autotuner() if autotune else None
        self.lookahead = lookahead
        self.keep_state = keep_state

    def close(self):
        for p in self.pools.values():
            p.batch.close()

    def _admit(self, P, now):
        tried = 0
        i = 0
        while i < len(P.queue) and tried < self.lookahead and len(P.active) < P.batch.max_sims:
            rq = P.queue[i]
            tried += 1
            if P.batch.info()["largest_free"] < -(-rq.n // 64) * 64:
                i += 1                       # does not fit yet: look further down the queue
                continue
            pos, vel, mass = rq.make()
            slot = P.batch.admit(pos, vel, mass, P.kernel, rq.eps, rq.G, rq.dt)
            if slot is None:
                i += 1
                continue
            rq.slot, rq.t_admit = slot, now
            P.active[slot] = rq
            del P.queue[i]

    def _finish_tick(self, P, t0, done):
        tick, force, inter = P.batch.profile_read()
        mi = _CLS[P.kernel]
        for k in range(len(tick)):
            P.ticks_ms.append(float(tick[k]))
            self._inter += float(inter[k].sum())
        if self.tuner and P.chosen and len(tick) and inter[-1, mi] > 0 and force[-1, mi] > 0:
            key, c = P.chosen
            self.tuner.record(key, c, force[-1, mi] * 1e6 / inter[-1, mi])
        for slot in list(P.active):
            rq = P.active[slot]
            if P.batch.slot_info(slot)[2] >= rq.nsteps:
                if self.keep_state:
                    rq.result = P.batch.get_state(slot)
                rq.t_done = time.perf_counter() - t0
                P.batch.evict(slot)
                del P.active[slot]
                done.append(rq)

    def _launch_tick(self, P):
        load = sum(float(rq.n) ** 2 for rq in P.active.values())
        P.chosen = None
        if self.tuner:
            key = Autotuner.bucket(P.kernel, load)
            c = self.tuner.choose(key)
            P.chosen = (key, c)
            P.batch.set_launch(P.kernel, *c)
        P.batch.step(1)
        P.inflight = True
        P.ticks += 1

    def run(self, requests, duration=None, max_ticks=None):
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        arrivals = collections.deque(reqs)
        done = []
        self._inter = 0.0
        l0 = sum(P.batch.launch_count for P in self.pools.values())
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            if duration is not None and now > duration:
                break
            if max_ticks is not None and sum(P.ticks for P in self.pools.values()) >= max_ticks:
                break
            while arrivals and arrivals[0].t_arrive <= now:
                rq = arrivals.popleft()
                self.pools[rq.mode].queue.append(rq)
            progress = False
            for P in self.pools.values():
                if P.inflight:
                    if not P.batch.ready():
                        continue
                    P.inflight = False
                    self._finish_tick(P, t0, done)
                    progress = True
                self._admit(P, now)
                if P.active:
                    self._launch_tick(P)
                    progress = True
            if not progress:
                idle = all(not P.inflight and not P.active and not P.queue for P in self.pools.values())
                if idle and not arrivals:
                    break
                wait = arrivals[0].t_arrive - now if (idle and arrivals) else 5e-5
                time.sleep(max(0.0, min(0.005, wait)))
        wall = time.perf_counter() - t0
        for P in self.pools.values():
            P.batch.sync()
            if P.inflight:
                P.inflight = False
                self._finish_tick(P, t0, done)
        lat = [r.t_done - r.t_arrive for r in done]
        out = {
            "ticks": sum(P.ticks for P in self.pools.values()),
            "wall_s": wall,
            "interactions": self._inter,
            "ginteractions_per_s": self._inter / wall / 1e9,
            "submitted": len(reqs),
            "admitted": len(done) + sum(len(P.active) for P in self.pools.values()),
            "completed": len(done),
            "queued_at_end": sum(len(P.queue) for P in self.pools.values()) + len(arrivals),
            "resident_at_end": sum(len(P.active) for P in self.pools.values()),
            "request_latency_s_p50": float(np.percentile(lat, 50)) if lat else None,
            "request_latency_s_p99": float(np.percentile(lat, 99)) if lat else None,
            "launches": sum(P.batch.launch_count for P in self.pools.values()) - l0,
            "done": done,
        }
        allt = []
        for m, P in self.pools.items():
            t = np.array(P.ticks_ms) if P.ticks_ms else np.zeros(1)
            allt += P.ticks_ms
            out[f"{m}_ticks"] = len(P.ticks_ms)
            out[f"{m}_tick_ms_p50"] = float(np.percentile(t, 50))
            out[f"{m}_tick_ms_p99"] = float(np.percentile(t, 99))
            P.ticks_ms = []
            P.ticks = 0
        t = np.array(allt) if allt else np.zeros(1)
        out["tick_ms_p50"] = float(np.percentile(t, 50))
        out["tick_ms_p99"] = float(np.percentile(t, 99))
        return out


def poisson_requests(count, rate, seed, n_range=(2 ** 10, 2 ** 16), nsteps=100, dt=5e-4,
                     modes=("fp64", "mixed")):
    """The serving workload: Poisson arrivals at `rate`/s, N log-uniform in
    n_range, Plummer (eps 0.01) or disk + halo (eps 0.02) 50/50, FP64 or MIXED
    50/50, `nsteps` KDK steps each.  Initial conditions are built lazily."""
    import nbody_ics
    g = np.random.default_rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, count))
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    ns = np.exp(g.uniform(lo, hi, count)).astype(int)
    kind = g.integers(0, 2, count)
    mode = g.integers(0, len(modes), count)
    seeds = g.integers(0, 2 ** 31, count)
    out = []
    for k in range(count):
        n, s = int(ns[k]), int(seeds[k])
        if kind[k] == 0:
            make = (lambda n=n, s=s: nbody_ics.plummer(n, s))
            eps = 0.01
        else:
            make = (lambda n=n, s=s: nbody_ics.disk_halo(n, s))
            eps = 0.02
        out.append(Request(k, n, modes[mode[k]], eps, 1.0, dt, nsteps, make, float(t[k])))
    return out


__all__ = ["Batch", "Autotuner", "Request", "Server", "poisson_requests", "NbodyError"]
