"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module holds no arithmetic of the QAOA method: it only draws random numbers and
turns them into graphs, angles and request streams.  Both sides of every parity test
consume the arrays produced here, so they always see identical graphs and angles.

Generator: xoshiro256** (Blackman & Vigna, 2018) seeded through SplitMix64.  A double in
[0, 1) is ``(x >> 11) * 2**-53``.  Independent streams use ``seed ^ (stream * 0x9E3779B97F4A7C15)``:
stream 0 = graph, 1 = angles, 2 = arrival times, 3 = request attributes.

Graph families (the paper times unweighted 3-regular benchmark graphs, §3.1 "u3R/w3R",
which are not distributed with it; these seeded graphs of the same family stand in):

* ``gnp(n, p, seed)``: Erdos-Renyi G(n, p); pairs u < v visited in lexicographic order,
  edge iff ``u01() < p``.
* ``regular3(n, seed)``: configuration model; 3n stubs (or 3(n-1)+2 for odd n, where a
  3-regular graph cannot exist by the handshake lemma, so vertex n-1 gets degree 2) are
  Fisher-Yates shuffled and paired consecutively; any self-loop or repeated edge rejects
  the draw and the shuffle is redrawn.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

STREAM_GRAPH = 0
STREAM_ANGLES = 1
STREAM_ARRIVALS = 2
STREAM_REQUESTS = 3


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** with SplitMix64 seeding (public-domain reference definition)."""

    def __init__(self, seed: int, stream: int = 0):
        s = (seed ^ ((stream * GOLDEN) & MASK64)) & MASK64
        st = []
        for _ in range(4):
            s = (s + GOLDEN) & MASK64
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
            st.append(z ^ (z >> 31))
        self.s = st

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s
        result = (_rotl((s1 * 5) & MASK64, 7) * 9) & MASK64
        t = (s1 << 17) & MASK64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return result

    def u01(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, k: int) -> int:
        """Uniform integer in [0, k) by Lemire's multiply-shift (k small, bias < 2**-50)."""
        return (self.next_u64() * k) >> 64

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.u01()

    def exponential(self, rate: float) -> float:
        return -math.log1p(-self.u01()) / rate


@dataclass
class Graph:
    """An undirected simple graph on vertices 0..n-1 with edges stored as u < v, sorted."""

    n: int
    edges: np.ndarray  # int32 [m, 2]
    weights: np.ndarray | None = None  # float64 [m] or None (unit weights)
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    def degrees(self) -> np.ndarray:
        d = np.zeros(self.n, dtype=np.int64)
        for u, v in self.edges:
            d[u] += 1
            d[v] += 1
        return d


def _canonical(n: int, pairs, name: str, weights=None) -> Graph:
    e = sorted((min(u, v), max(u, v)) for u, v in pairs)
    arr = np.array(e, dtype=np.int32).reshape(-1, 2)
    w = None if weights is None else np.asarray(weights, dtype=np.float64)
    return Graph(n=n, edges=arr, weights=w, name=name)


def gnp(n: int, p: float, seed: int = 0) -> Graph:
    rng = Xoshiro256ss(seed, STREAM_GRAPH)
    pairs = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.u01() < p]
    return _canonical(n, pairs, f"gnp(n={n},p={p},seed={seed})")


def regular3(n: int, seed: int = 0, max_tries: int = 100000) -> Graph:
    """Random 3-regular graph (near-3-regular, one degree-2 vertex, for odd n)."""
    if n < 4:
        raise ValueError("3-regular graphs need n >= 4")
    degs = [3] * n
    if n % 2 == 1:
        degs[n - 1] = 2
    stubs = [v for v in range(n) for _ in range(degs[v])]
    rng = Xoshiro256ss(seed, STREAM_GRAPH)
    for _ in range(max_tries):
        st = list(stubs)
        for i in range(len(st) - 1, 0, -1):
            j = rng.below(i + 1)
            st[i], st[j] = st[j], st[i]
        seen = set()
        ok = True
        for k in range(0, len(st), 2):
            u, v = st[k], st[k + 1]
            if u == v:
                ok = False
                break
            key = (min(u, v), max(u, v))
            if key in seen:
                ok = False
                break
            seen.add(key)
        if ok:
            tag = "near-3-regular" if n % 2 else "3-regular"
            return _canonical(n, seen, f"{tag}(n={n},seed={seed})")
    raise RuntimeError("configuration model did not produce a simple graph")


def complete(n: int) -> Graph:
    return _canonical(n, [(u, v) for u in range(n) for v in range(u + 1, n)], f"K{n}")


def ring(n: int) -> Graph:
    return _canonical(n, [(i, (i + 1) % n) for i in range(n)], f"ring{n}")


def star(n: int) -> Graph:
    return _canonical(n, [(0, v) for v in range(1, n)], f"star{n}")


def empty(n: int) -> Graph:
    return _canonical(n, [], f"empty{n}")


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return _canonical(10, outer + spokes + inner, "petersen")


def random_weights(g: Graph, seed: int = 0, lo: float = 0.1, hi: float = 2.0) -> Graph:
    """Attach seeded uniform edge weights (stream 3) to a graph."""
    rng = Xoshiro256ss(seed, STREAM_REQUESTS)
    w = np.array([rng.uniform(lo, hi) for _ in range(g.m)], dtype=np.float64)
    return Graph(n=g.n, edges=g.edges.copy(), weights=w, name=g.name + "+w")


def angles(p: int, seed: int = 0, gamma_hi: float = math.pi, beta_hi: float = math.pi / 2):
    """gamma_k ~ U[0, gamma_hi], beta_k ~ U[0, beta_hi], drawn alternately from stream 1."""
    rng = Xoshiro256ss(seed, STREAM_ANGLES)
    g = np.empty(p, dtype=np.float64)
    b = np.empty(p, dtype=np.float64)
    for k in range(p):
        g[k] = rng.uniform(0.0, gamma_hi)
        b[k] = rng.uniform(0.0, beta_hi)
    return g, b


def random_state(n: int, seed: int = 0) -> np.ndarray:
    """A seeded normalised complex128 state (numpy's PCG64; used only as a test input)."""
    r = np.random.default_rng(seed)
    v = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
    return v / np.linalg.norm(v)


@dataclass
class Request:
    """One evaluation request of a serving stream."""

    rid: int
    arrival_s: float
    graph: Graph
    gamma: np.ndarray
    beta: np.ndarray
    want_grad: bool


@dataclass
class RequestStream:
    requests: list = field(default_factory=list)


def request_stream(count: int = 4096, rate_hz: float = 2000.0, seed: int = 0,
                   n_lo: int = 14, n_hi: int = 28, p_lo: int = 1, p_hi: int = 6,
                   grad_prob: float = 0.25) -> RequestStream:
    """Poisson arrivals; n ~ U{n_lo..n_hi}; half 3-regular, half G(n, 0.3); p ~ U{p_lo..p_hi}."""
    arr = Xoshiro256ss(seed, STREAM_ARRIVALS)
    att = Xoshiro256ss(seed, STREAM_REQUESTS)
    t = 0.0
    out = []
    for i in range(count):
        t += arr.exponential(rate_hz)
        n = n_lo + att.below(n_hi - n_lo + 1)
        gseed = att.next_u64() & 0xFFFFFFFF
        if att.u01() < 0.5:
            g = regular3(n, seed=gseed)
        else:
            g = gnp(n, 0.3, seed=gseed)
        p = p_lo + att.below(p_hi - p_lo + 1)
        ga, be = angles(p, seed=att.next_u64() & 0xFFFFFFFF)
        want = att.u01() < grad_prob
        out.append(Request(rid=i, arrival_s=t, graph=g, gamma=ga, beta=be, want_grad=want))
    return RequestStream(out)


# Named workloads: the five evaluation configurations of the build, by what they are.
def workload_n10_regular3_p1():
    """3-regular n=10, seed 0, p=1, gamma=0.4, beta=0.3 (complex128)."""
    return regular3(10, 0), np.array([0.4]), np.array([0.3])


def workload_gnp26_p4():
    """G(26, 0.5), seed 0, p=4, seeded angles."""
    g = gnp(26, 0.5, 0)
    ga, be = angles(4, 0)
    return g, ga, be


def workload_regular3_n33_p8():
    """Near-3-regular n=33 (one degree-2 vertex), seed 0, p=8, seeded angles (complex64)."""
    g = regular3(33, 0)
    ga, be = angles(8, 0)
    return g, ga, be


def workload_gnp24_p10():
    """G(24, 0.5), seed 0, p=10, seeded angles (gradient workload)."""
    g = gnp(24, 0.5, 0)
    ga, be = angles(10, 0)
    return g, ga, be
