"""Writes stored expected values for the large parity cases, computed by the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py [names...]
The gate-level oracle (Algorithm 1 in complex128) needs minutes at n = 24..28, too long to
rerun in every test session, so its <C>, norm and a seeded sample of amplitudes are stored as
JSON here, and for the gradient cases (grad_*) the oracle's FP64 adjoint gradient d<C>/d gamma_k,
d<C>/d beta_k.  Nothing in this script touches the CUDA path.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2312_03019_b300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    "gnp26_p4": I.workload_gnp26_p4,
    "gnp24_p10": I.workload_gnp24_p10,
    "regular3_n22_p6": lambda: (I.regular3(22, 0), *I.angles(6, 0)),
}

# adjoint gradients at the sizes whose sweeps use each compiled sweep program (high groups of
# 6, 7, 8 and 9 bits)
GRAD_CASES = {
    "grad_regular3_n24_p3": lambda: (I.regular3(24, 0), *I.angles(3, 24)),
    "grad_regular3_n25_p3": lambda: (I.regular3(25, 0), *I.angles(3, 25)),
    "grad_regular3_n27_p2": lambda: (I.regular3(27, 0), *I.angles(2, 27)),
    "grad_regular3_n28_p2": lambda: (I.regular3(28, 0), *I.angles(2, 28)),
    "grad_regular3_n29_p2": lambda: (I.regular3(29, 0), *I.angles(2, 29)),
}


def sample_indices(n, count=512, seed=12345):
    r = np.random.default_rng(seed)
    idx = set(int(i) for i in r.integers(0, 1 << n, size=count))
    idx |= {0, 1, (1 << n) - 1, (1 << n) - 2, 1 << (n - 1)}
    return sorted(idx)


def make(name):
    g, gamma, beta = CASES[name]()
    t0 = time.time()
    psi = oracle.qaoa_state(g, gamma, beta)
    c, nrm = oracle.expectation(g, psi)
    idx = sample_indices(g.n)
    rec = {
        "what": f"oracle (Algorithm 1, complex128) on {g.name}, p={len(gamma)}",
        "graph": g.name, "n": g.n, "m": g.m, "edges": g.edges.tolist(),
        "gamma": gamma.tolist(), "beta": beta.tolist(),
        "expectation": c, "norm": nrm,
        "sample_index": idx,
        "sample_re": [float(psi[i].real) for i in idx],
        "sample_im": [float(psi[i].imag) for i in idx],
        "oracle_seconds": time.time() - t0, "oracle_threads": oracle.threads(),
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, c, nrm, f"{time.time() - t0:.1f}s", flush=True)


def make_grad(name):
    g, gamma, beta = GRAD_CASES[name]()
    t0 = time.time()
    c, dg, db = oracle.adjoint_gradient(g, gamma, beta)
    rec = {
        "what": f"oracle FP64 adjoint gradient (Algorithm 1, complex128) on {g.name}, p={len(gamma)}",
        "graph": g.name, "n": g.n, "m": g.m, "edges": g.edges.tolist(),
        "gamma": gamma.tolist(), "beta": beta.tolist(),
        "expectation": c, "d_gamma": [float(x) for x in dg], "d_beta": [float(x) for x in db],
        "oracle_seconds": time.time() - t0, "oracle_threads": oracle.threads(),
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, c, f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(CASES) + list(GRAD_CASES)):
        (make_grad if nm in GRAD_CASES else make)(nm)
