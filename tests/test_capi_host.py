"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry point
declared in include/qaoa.h, validates its inputs, and plans passes that apply every RX gate of
every level exactly once (Algorithm 1's mixer layer) with the cost phases in order."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2312_03019_b300 import build as B
from paper_2312_03019_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2312_03019_b300 import binding
    return binding


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(qaoa_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_index_checks_only_in_the_debug_build(lib):
    # the release library has no index checks: the call says so without touching a GPU
    with pytest.raises(lib.QAOAError) as ei:
        lib.qaoa_debug_bounds_read(0)
    assert ei.value.status == lib.QAOA_ERR_UNSUPPORTED


def test_state_bytes(lib):
    assert lib.qaoa_state_bytes(10, "c64") == 8 << 10
    assert lib.qaoa_state_bytes(33, "c64") == 8 << 33
    assert lib.qaoa_state_bytes(26, "c128") == 16 << 26
    assert lib.qaoa_state_bytes(0, "c64") == 0
    assert lib.qaoa_state_bytes(35, "c64") == 0


@pytest.mark.parametrize("edges,msg", [
    ([[0, 0]], "self loop"), ([[0, 1], [1, 0]], "repeated"), ([[0, 9]], "range"),
])
def test_invalid_graph_rejected_before_any_gpu_work(lib, edges, msg):
    g = I.Graph(4, np.array(edges, dtype=np.int32))
    with pytest.raises(lib.QAOAError) as ei:
        lib.qaoa_state_init(g, "c64", 1 << 20, 1 << 20, 0)
    assert ei.value.status == lib.QAOA_ERR_INVALID
    assert msg in str(ei.value)


@pytest.mark.parametrize("w,msg", [(np.nan, "non-finite"), (np.inf, "non-finite"), (-np.inf, "non-finite"),
                                   (1.5e12, "1e12")])
def test_invalid_weights_rejected_before_any_gpu_work(lib, w, msg):
    g = I.gnp(8, 0.5, 3)
    wts = np.linspace(0.5, 1.5, g.m)
    wts[g.m // 2] = w
    bad = I.Graph(n=g.n, edges=g.edges, weights=wts)
    with pytest.raises(lib.QAOAError) as ei:
        lib.qaoa_state_init(bad, "c64", 1 << 20, 1 << 20, 0)
    assert ei.value.status == lib.QAOA_ERR_INVALID
    assert msg in str(ei.value)


def test_invalid_sizes_rejected(lib):
    g = I.ring(5)
    with pytest.raises(lib.QAOAError):
        lib.qaoa_state_init(g, "c64", 1 << 20, 8, 0)  # buffer too small
    with pytest.raises(lib.QAOAError):
        lib.qaoa_state_init(g, "c64", (1 << 20) + 4, 1 << 20, 0)  # misaligned
    big = I.Graph(35, np.zeros((0, 2), dtype=np.int32))
    with pytest.raises(lib.QAOAError):
        lib.qaoa_state_init(big, "c64", 1 << 20, 1 << 40, 0)


def _parse_plan(d):
    Q, R, cmin, ng = d[0], d[1], d[2], d[3]
    pos = 4
    groups = []
    for _ in range(ng):
        sz = d[pos]
        groups.append(list(d[pos + 1: pos + 1 + sz]))
        pos += 1 + sz
    npass = d[pos]
    pos += 1
    passes = []
    for _ in range(npass):
        grp, nops = d[pos], d[pos + 1]
        pos += 2
        ops = [tuple(d[pos + 3 * i: pos + 3 * i + 3]) for i in range(nops)]
        pos += 3 * nops
        passes.append((grp, ops))
    assert pos == len(d)
    return Q, R, cmin, groups, passes


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [15, 16, 18, 20, 22, 23, 24, 26, 29, 30, 31, 33, 34])
@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_plan_applies_each_rx_once_per_level(lib, prec, n, p):
    if (prec == "c128" and n <= 13) or (prec == "c64" and n <= 14):
        pytest.skip("small-state kernel")
    d = lib.qaoa_plan_describe(n, prec, p)
    Q, R, cmin, groups, passes = _parse_plan(d)
    # groups partition [0, n); group 0 is a run [0, r) with r >= 8 plus bits at or above the
    # 2 MiB page boundary; high groups leave >= cmin row bits; the page-boundary bits are spread
    # evenly over all groups (group 0's share capped by r >= 8)
    cover = []
    for bits in groups:
        cover += bits
    assert sorted(cover) == list(range(n))
    page_bit = 18 if prec == "c64" else 17
    g0 = groups[0]
    r = 0
    while r < len(g0) and g0[r] == r:
        r += 1
    assert len(g0) == Q and r >= 8 and all(b >= page_bit for b in g0[r:])
    sizes = [len(b) for b in groups[1:]]
    assert all(sz <= Q - cmin for sz in sizes) and max(sizes) - min(sizes) <= 1
    high = [sum(1 for b in bits if b >= page_bit) for bits in groups]
    assert max(high[1:]) - min(high[1:]) <= 1
    assert high[0] == min(Q - 8, max(0, n - max(page_bit, Q)) // len(groups))
    assert max(high) - min(high) <= 1 or high[0] == Q - 8
    g = len(groups)
    assert len(passes) == p * (g - 1) + 1

    reg_lo = {0: Q - R, 1: Q - 2 * R, 2: 0}
    rx_seen = {k: [] for k in range(p)}
    phases = []
    expect_at = None
    events = []  # sequence of ("rx", level) / ("phase", level)
    for pi, (grp, ops) in enumerate(passes):
        bits = groups[grp]
        if grp == 0:  # rows of the low run, then group 0's page-boundary bits
            gpos = list(bits)
            target = (1 << Q) - 1
        else:
            cprime = Q - len(bits)
            gpos = list(range(cprime)) + bits
            target = ((1 << Q) - 1) & ~((1 << cprime) - 1)
        kind0, lay0, _ = ops[0]
        assert kind0 == (2 if pi == 0 else 1)  # synthesise |+> only in the first pass
        assert lay0 in (0, 1)
        assert ops[-1][0] == 7 and ops[-1][1] in (0, 1)  # store from a coalesced layout
        layout = lay0
        for kind, arg, mask in ops[1:-1]:
            if kind == 3:
                layout = arg
            elif kind == 4:
                regmask = ((1 << R) - 1) << reg_lo[layout]
                assert mask and (mask & ~regmask) == 0 and (mask & ~target) == 0
                for u in range(Q):
                    if (mask >> u) & 1:
                        rx_seen[arg].append(gpos[u])
                events.append(("rx", arg))
            elif kind == 5:
                phases.append(arg)
                events.append(("phase", arg))
            elif kind == 6:
                expect_at = (pi, len(events))
            else:
                raise AssertionError(f"unexpected op {kind}")
    for k in range(p):
        assert sorted(rx_seen[k]) == list(range(n)), f"level {k}"
    assert phases == list(range(p))
    # phase k after every RX of level k-1 and before any RX of level k
    for idx, (what, k) in enumerate(events):
        if what == "phase":
            assert all(kk < k for w, kk in events[:idx] if w == "rx")
            assert all(kk >= k for w, kk in events[idx + 1:] if w == "rx")
    assert expect_at == (len(passes) - 1, len(events))
    if g >= 3:  # group 0 is never a fused boundary pass
        for grp, ops in passes:
            if grp == 0:
                assert sum(1 for k, _, _ in ops if k == 5) == 0


def test_small_states_have_no_pass_plan(lib):
    assert lib.qaoa_plan_describe(14, "c64", 3) == []
    assert lib.qaoa_plan_describe(13, "c128", 3) == []
