"""Index checks of the CUDA path.  The debug build of the library (-DQAOA_DEBUG_BOUNDS,
libqaoa_b300_debug.so) checks in its kernels every state load and store, shared-memory exchange,
phase-table read, cut-value write and weighted-row read against the buffer it belongs to; a
failed check sets a bit in a device word and skips the access (no trap).  This runs the paths
through that build, in a child process, at many shapes (one CTA, two and three groups, ragged
groups, the largest states; forward, <C>, read-out, gradients, edge weights, cut tables, the
allocation-free <C>, the server) and requires that no check failed."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json
import numpy as np
import torch
from paper_2312_03019_b300 import binding as B, inputs as I

assert B.LIB_PATH.endswith("libqaoa_b300_debug.so"), B.LIB_PATH
B.qaoa_debug_bounds_read(0, True)
report = {}

def check(name):
    report[name] = B.qaoa_debug_bounds_read(0, True)

def graph(n, weighted=False):
    g = I.regular3(n, n) if n >= 4 and n % 2 == 0 else I.gnp(n, 0.4, n)
    return I.random_weights(g, seed=n, lo=-1.0, hi=2.0) if weighted else g

for prec in ("c64", "c128"):
    for n in (1, 3, 12, 13, 14, 17, 20, 22, 23, 24, 26, 28):
        gamma, beta = I.angles(3, n, beta_hi=np.pi)
        s = B.QAOAState(graph(n), prec)
        s.apply_layers(gamma, beta)
        s.expectation()
        if n <= 20:
            s.amplitudes()
        s.close()
        check(f"forward {prec} n={n}")
    # complex64 n = 24 and 28: the persistent sweep programs with the 6- and 8-bit group masks
    for n in (13, 16, 22, 25) + ((24, 28) if prec == "c64" else ()):
        gamma, beta = I.angles(3, n)
        s = B.QAOAState(graph(n), prec)
        s.gradient(gamma, beta)
        s.close()
        check(f"gradient {prec} n={n}")
    for n in (14, 20, 25):
        gamma, beta = I.angles(2, n)
        s = B.QAOAState(graph(n, True), prec)
        s.apply_layers(gamma, beta)
        s.expectation()
        s.gradient(gamma, beta)
        s.close()
        check(f"weighted {prec} n={n}")
    g = graph(20)
    groups = B.qaoa_plan_describe(20, prec, 1)[3]
    for grp in range(groups):
        for layout in range(3):
            B.qaoa_cut_table_geometry(g, prec, grp, layout)
    B.qaoa_cut_table_f64(graph(16, True), prec)
    check(f"cut tables {prec}")
    torch.cuda.empty_cache()

# the allocation-free <C> (its own kernel arguments, built outside the pass planner): one-CTA
# and tiled sizes, up to the largest its scratch allows
for prec, sizes in (("c64", (12, 21, 29)), ("c128", (11, 20, 28))):
    for n in sizes:
        gamma, beta = I.angles(2, 60 + n)
        s = B.QAOAState(graph(n), prec)
        s.apply_layers(gamma, beta)
        B.qaoa_expectation_static(graph(n), prec, s.buffer.data_ptr(), s.nbytes, s.stream.cuda_stream)
        s.close()
        torch.cuda.empty_cache()
        check(f"static <C> {prec} n={n}")

for n, p in ((33, 2), (34, 1)):
    gamma, beta = I.angles(p, n)
    s = B.QAOAState(graph(n), "c64")
    s.apply_layers(gamma, beta)
    s.expectation()
    s.close()
    torch.cuda.empty_cache()
    check(f"forward c64 n={n}")

sv = B.qaoa_server_create(hbm_budget_bytes=4 << 30, prec="c64")
try:
    tickets = []
    for i, n in enumerate((8, 11, 14, 18, 22, 9, 16)):
        gamma, beta = I.angles(2, 40 + i)
        tickets.append(B.qaoa_submit(sv, graph(n), gamma, beta, want_grad=(i % 2 == 1)))
    for i, n in enumerate((15, 15, 15, 20, 20, 22, 22)):  # packed mid-size launches
        gamma, beta = I.angles(3, 80 + i)
        tickets.append(B.qaoa_submit(sv, I.gnp(n, 0.3, 80 + i), gamma, beta))
    while tickets:
        tickets = [t for t in tickets if B.qaoa_poll(sv, t) is None]
finally:
    B.qaoa_server_destroy(sv)
check("server c64")
print(json.dumps(report))
'''


def test_no_index_check_fails_in_the_debug_build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03019_b300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, QAOA_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    report = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(report) >= 30, report
    failed = {k: v for k, v in report.items() if v}
    assert not failed, failed
