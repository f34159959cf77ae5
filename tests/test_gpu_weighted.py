"""Edge-weighted graphs (Algorithm 2: C(z) = sum_e w_e (z_u xor z_v), real w_e) on the GPU
against the CPU oracle.

The kernels evaluate two fixed-point sums per amplitude (B = 32 bits for complex64, 64 for
complex128, exact modulo 2^B): the phase angle from per-edge angles gamma w_e / (2 pi) rounded to
2^-B turns, and the value C(z) from the weights rounded to 2^-S, S the largest power with
sum |w_e| 2^S <= 2^(B-2).  Tolerances follow from that:
  cut values: at most m 2^-(S+1) from the exact sum (bit-exact for integer weights);
  complex128: <C> within 1e-12 relative, state within 1e-12 in the 2-norm;
  complex64: <C> within 1e-5 sum |w|, fidelity >= 1 - 1e-5.
"""
import math

import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I
from tests.tolerances import c64_grad_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03019_b300 import build
    build.build()
    from paper_2312_03019_b300 import binding
    return binding


def weighted(g, seed, lo=0.1, hi=2.0):
    return I.random_weights(g, seed=seed, lo=lo, hi=hi)


def integer_weighted(g, seed):
    w = I.random_weights(g, seed=seed, lo=1.0, hi=6.0)
    return I.Graph(n=g.n, edges=w.edges, weights=np.floor(w.weights), name=g.name + "+int")


def value_tol(g, prec):
    tot = float(np.sum(np.abs(g.weights)))
    bits = 32 if prec == "c64" else 64
    s = bits - 2 - math.ceil(math.log2(tot))
    return g.m * 2.0 ** -(s + 1) + 1e-12 * tot


def oracle_weighted_cuts(g):
    """C(z) from Algorithm 2's totRotation, C = (W - totRotation) / 2, cross-checked against the
    oracle's plain edge loop."""
    import oracle
    W = float(np.sum(g.weights))
    out = np.empty(1 << g.n)
    for z in range(1 << g.n):
        out[z] = oracle.cut_value(g, z)
    for z in range(0, 1 << g.n, max(1, (1 << g.n) // 64)):
        assert abs((W - oracle.alg2_tot_rotation(g, z)) / 2 - out[z]) <= 1e-12 * max(1.0, W)
    return out


GRAPHS = [
    lambda n: weighted(I.regular3(n, n) if n % 2 == 0 else I.gnp(n, 0.3, n), 1),
    lambda n: weighted(I.gnp(n, 0.5, 2 * n), 2, lo=-1.0, hi=1.0),       # signed weights
    lambda n: weighted(I.complete(min(n, 12)), 3, lo=10.0, hi=100.0),   # large gamma w: many turns
]


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [6, 11, 14, 16])
def test_weighted_cut_values_every_geometry(B, prec, n):
    for mk in GRAPHS:
        g = mk(n)
        ref = oracle_weighted_cuts(g)
        tol = value_tol(g, prec)
        got = B.qaoa_cut_table_f64(g, prec)  # the path the size uses by default
        assert np.max(np.abs(got - ref)) <= tol, (g.name, prec)
        plan = B.qaoa_plan_describe(g.n, prec, 1)
        if not plan:  # whole state in one CTA: no tile geometries
            continue
        groups = plan[3]
        for grp in range(groups):
            for layout in range(3):
                got = B.qaoa_cut_table_f64(g, prec, grp, layout)
                assert np.max(np.abs(got - ref)) <= tol, (g.name, prec, grp, layout)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [9, 15])
def test_integer_weights_bit_exact(B, prec, n):
    g = integer_weighted(I.gnp(n, 0.4, 11), 4)
    ref = oracle_weighted_cuts(g)
    got = B.qaoa_cut_table_f64(g, prec)
    assert np.array_equal(got, ref)


def run(B, g, gamma, beta, prec):
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, beta)
    c, nrm = s.expectation()
    psi = s.amplitudes().astype(np.complex128)
    s.close()
    return c, nrm, psi


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,p,mk", [
    (2, 2, lambda: weighted(I._canonical(2, [(0, 1)], "edge"), 5)),
    (8, 3, lambda: weighted(I.complete(8), 6, lo=-2.0, hi=2.0)),
    (10, 2, lambda: weighted(I.regular3(10, 0), 7)),
    (13, 3, lambda: weighted(I.gnp(13, 0.4, 8), 8)),
    (14, 2, lambda: weighted(I.regular3(14, 1), 9, lo=5.0, hi=50.0)),
    (16, 4, lambda: weighted(I.gnp(16, 0.3, 9), 10)),
    (18, 3, lambda: weighted(I.regular3(18, 2), 11)),
    (20, 2, lambda: weighted(I.gnp(20, 0.25, 10), 12, lo=-1.0, hi=3.0)),
])
def test_weighted_state_parity(B, prec, n, p, mk):
    import oracle
    g = mk()
    gamma, beta = I.angles(p, seed=n + 40)
    ref = oracle.qaoa_state(g, gamma, beta)
    ref_c, _ = oracle.expectation(g, ref)
    c, nrm, psi = run(B, g, gamma, beta, prec)
    if prec == "c128":
        assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
        assert abs(nrm - 1.0) < 1e-12
        assert np.linalg.norm(psi - ref) <= 1e-12
    else:
        assert abs(c - ref_c) <= 1e-5 * float(np.sum(np.abs(g.weights)))
        assert abs(nrm - 1.0) < 1e-5
        assert abs(np.vdot(ref, psi)) ** 2 >= 1 - 1e-5


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n,p", [(24, 2), (25, 3)])
def test_weighted_state_parity_three_groups(B, prec, n, p):
    """Sizes with three mixer groups, where the weighted passes run their recipe kernels
    (complex64) and the interpreting kernel (complex128)."""
    import oracle
    g = weighted(I.regular3(n, 3) if n % 2 == 0 else I.gnp(n, 0.2, 3), 31, lo=-0.5, hi=2.0)
    gamma, beta = I.angles(p, seed=n + 90)
    ref = oracle.qaoa_state(g, gamma, beta)
    ref_c, _ = oracle.expectation(g, ref)
    c, nrm, psi = run(B, g, gamma, beta, prec)
    if prec == "c128":
        assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
        assert np.linalg.norm(psi - ref) <= 1e-12
    else:
        assert abs(c - ref_c) <= 1e-5 * float(np.sum(np.abs(g.weights)))
        assert abs(np.vdot(ref, psi)) ** 2 >= 1 - 1e-5


def test_weighted_phase_samples_n30(B):
    """n = 30, complex64, beta = 0: psi_z = 2^(-n/2) exp(-i sum gamma C(z)) with the weighted
    cut value, sampled amplitude by amplitude against the oracle."""
    import oracle
    import torch
    g = weighted(I.regular3(30, 4), 32, lo=0.1, hi=3.0)
    gamma = np.array([0.7, 1.9])
    n = g.n
    rng = np.random.default_rng(30)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 200), [0, (1 << n) - 1]]))
    s = B.QAOAState(g, "c64")
    s.apply_layers(gamma, np.zeros(2))
    t = s.as_tensor()
    samp = t[torch.tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)
    amp = 2 ** (-n / 2)
    ref = np.array([amp * np.exp(-1j * gamma.sum() * oracle.cut_value(g, int(z))) for z in idx])
    s.close()
    del t
    assert np.max(np.abs(samp - ref)) < 2e-5 * amp


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [11, 16])
def test_weighted_phase_every_amplitude(B, prec, n):
    """beta = 0: psi_z = 2^(-n/2) exp(-i sum_k gamma_k C(z)) exactly, so every amplitude checks the
    weighted phase (fixed-point angle sums, 256-step rotation table and the remainder's series)
    against exp of the oracle's cut value.  complex128: 1e-13 of the amplitude, far below a
    dropped series term (~2e-12) or a wrong table step (~0.02); complex64: 1e-6 (float
    rounding of the table and products over two levels).  n = 11 runs the small-state kernel,
    n = 16 the tile passes; the angles span many turns of the table."""
    g = weighted(I.regular3(n, n) if n % 2 == 0 else I.gnp(n, 0.3, n), 41, lo=0.1, hi=2.0)
    gamma = np.array([2.9, -5.3])
    cuts = oracle_weighted_cuts(g)
    amp = 2.0 ** (-n / 2)
    ref = amp * np.exp(-1j * gamma.sum() * cuts)
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, np.zeros(2))
    psi = s.amplitudes().astype(np.complex128)
    s.close()
    err = np.max(np.abs(psi - ref)) / amp
    assert err < (1e-13 if prec == "c128" else 1e-6), err


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [11, 16])
def test_weight_scale_covariance(B, prec, n):
    """Weights times 2^-600 with gamma times 2^600: the per-edge angles gamma w are the same
    doubles and the value rows the same integers (the scale 2^S moves with them), so the state
    is bit-identical and <C> exactly 2^-600 times the unscaled one; tiny weights keep their
    relative accuracy."""
    g = weighted(I.regular3(n, n) if n % 2 == 0 else I.gnp(n, 0.3, n), 43, lo=-1.0, hi=2.0)
    k = 2.0 ** -600
    gs = I.Graph(n=g.n, edges=g.edges, weights=g.weights * k)
    gamma, beta = np.array([0.45, -1.2]), np.array([0.3, 0.8])
    out = []
    for gg, gm in ((g, gamma), (gs, gamma / k)):
        s = B.QAOAState(gg, prec)
        s.apply_layers(gm, beta)
        c, nrm = s.expectation()
        out.append((s.amplitudes(), c, nrm))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[1][1] == out[0][1] * k
    assert out[1][2] == out[0][2]


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_weights_all_one_take_the_unit_path(B, prec):
    g = I.gnp(17, 0.4, 3)
    g1 = I.Graph(n=g.n, edges=g.edges, weights=np.ones(g.m), name=g.name + "+ones")
    gamma, beta = I.angles(3, 5)
    c0, _, psi0 = run(B, g, gamma, beta, prec)
    c1, _, psi1 = run(B, g1, gamma, beta, prec)
    assert c0 == c1 and np.array_equal(psi0, psi1)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_weighted_zero_levels_expectation(B, prec):
    """|+>^n: <C> = W / 2 exactly up to the value rounding, through the lazy initial state."""
    g = weighted(I.regular3(16, 4), 13)
    s = B.QAOAState(g, prec)
    c, nrm = s.expectation()
    s.close()
    assert abs(c - float(np.sum(g.weights)) / 2) <= value_tol(g, prec) + (1e-6 if prec == "c64" else 1e-12) * float(np.sum(g.weights))
    assert abs(nrm - 1.0) <= (1e-6 if prec == "c64" else 1e-13)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,p,mk", [
    (6, 3, lambda: weighted(I.complete(6), 20, lo=-1.0, hi=2.0)),
    (12, 2, lambda: weighted(I.gnp(12, 0.5, 21), 21)),
    (14, 3, lambda: weighted(I.regular3(14, 22), 22)),
    (16, 2, lambda: weighted(I.gnp(16, 0.3, 23), 23, lo=2.0, hi=20.0)),
    # the persistent sweep programs with edge weights (complex64, n >= 22)
    (22, 2, lambda: weighted(I.regular3(22, 24), 24)),
    (24, 2, lambda: weighted(I.gnp(24, 0.3, 25), 25, lo=0.1, hi=2.0)),
])
def test_weighted_gradient_matches_oracle_adjoint(B, prec, n, p, mk):
    import oracle
    import torch
    g = mk()
    gamma, beta = I.angles(p, seed=n + 70)
    ref_c, ref_dg, ref_db = oracle.adjoint_gradient(g, gamma, beta)
    s = B.QAOAState(g, prec)
    work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
    c, dg, db = B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)
    s.close()
    W = float(np.sum(np.abs(g.weights)))
    scale = max(1.0, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
    if prec == "c128":
        assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
        assert np.max(np.abs(dg - ref_dg)) <= 1e-10 * scale
        assert np.max(np.abs(db - ref_db)) <= 1e-10 * scale
    else:
        # the FP32 rounding bound of the unit-weight gradient (tests/tolerances.py): the weights
        # enter through the phase tables (angles rounded to 2^-32 turns) and the fixed-point
        # values (rounded to 2^-S with S such that sum |w| 2^S is near 2^30), both far below it
        tol = c64_grad_tol(n, p, g.m, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
        assert abs(c - ref_c) <= 1e-5 * W
        assert np.max(np.abs(dg - ref_dg)) <= tol
        assert np.max(np.abs(db - ref_db)) <= tol


def test_weighted_requests_through_the_server(B):
    reqs = [(weighted(I.gnp(n, 0.4, n), n), *I.angles(2, n), n % 2 == 0) for n in (9, 14, 18)]
    sv = B.qaoa_server_create(1 << 30, "c64", max_inflight=8, max_batch=8, streams=2)
    tickets = [B.qaoa_submit(sv, g, ga, be, grad) for g, ga, be, grad in reqs]
    got = {}
    import time
    t0 = time.time()
    while len(got) < len(tickets) and time.time() - t0 < 60:
        for t in tickets:
            if t not in got:
                r = B.qaoa_poll(sv, t)
                if r is not None:
                    got[t] = r
        time.sleep(0.001)
    stats = B.qaoa_server_stats_read(sv)
    B.qaoa_server_destroy(sv)
    assert stats["batched_requests"] == 0  # weighted requests always run alone
    import torch
    for (g, ga, be, grad), t in zip(reqs, tickets):
        r = got[t]
        assert r["status"] == 0
        s = B.QAOAState(g, "c64")
        if grad:
            work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
            c, dg, db = B.qaoa_gradient(s.handle, ga, be, work.data_ptr(), s.nbytes)
            assert np.array_equal(r["d_gamma"], dg) and np.array_equal(r["d_beta"], db)
        else:
            s.apply_layers(ga, be)
            c, _ = s.expectation()
        s.close()
        assert r["expectation"] == c
        # and against the oracle (<C_w> by the gate-level circuit, the gradient by its adjoint)
        import oracle
        W = float(np.sum(np.abs(g.weights)))
        if grad:
            rc, rdg, rdb = oracle.adjoint_gradient(g, ga, be)
            ref = np.concatenate([rdg, rdb])
            tol = c64_grad_tol(g.n, len(ga), g.m, float(np.max(np.abs(ref))))
            assert np.max(np.abs(np.concatenate([r["d_gamma"], r["d_beta"]]) - ref)) <= tol
        else:
            rc, _ = oracle.expectation(g, oracle.qaoa_state(g, ga, be))
        assert abs(r["expectation"] - rc) <= 1e-5 * W


def test_weighted_more_levels_than_one_coefficient_chunk(B):
    """p = 70 on a weighted graph: the fixed-point angle rows are rebuilt per 64-level chunk."""
    import oracle
    g = weighted(I.regular3(16, 9), 40)
    gamma, beta = I.angles(70, 41)
    ref = oracle.qaoa_state(g, gamma, beta)
    ref_c, _ = oracle.expectation(g, ref)
    c, nrm, psi = run(B, g, gamma, beta, "c128")
    assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
    assert np.linalg.norm(psi - ref) <= 1e-11


def test_weighted_rejections(B):
    g = I.gnp(10, 0.5, 1)
    bad = I.Graph(n=g.n, edges=g.edges, weights=np.full(g.m, np.nan))
    with pytest.raises(B.QAOAError):
        B.QAOAState(bad, "c64")
    huge = I.Graph(n=g.n, edges=g.edges, weights=np.full(g.m, 1e13))
    with pytest.raises(B.QAOAError):
        B.QAOAState(huge, "c64")
    with pytest.raises(B.QAOAError):  # the uint16 table is for cut counts only
        B.qaoa_cut_table(weighted(g, 1))


def test_weighted_max_size_n34(B):
    """n = 34 (128 GiB complex64, four groups, three passes per level) on the weighted path, with
    every weight 2: exp(-i gamma C_w) = exp(-i 2 gamma C), so beta = 0 gives
    psi_z = 2^(-n/2) exp(-2 i gamma C(z)) (sampled against the oracle's cut value) and the p = 1
    <C_w> is twice the unweighted closed form at 2 gamma."""
    import oracle
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g0 = I.regular3(34, 0)
    g = I.Graph(n=g0.n, edges=g0.edges, weights=np.full(g0.m, 2.0))
    n = g.n
    rng = np.random.default_rng(34)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 200), [0, (1 << n) - 1, (1 << 33) + 7]]))
    gamma = np.array([0.35, 1.1])
    amp = 2.0 ** (-n / 2)
    ref = amp * np.exp(-2j * gamma.sum() * np.array([oracle.cut_value(g0, int(z)) for z in idx]))
    s = B.QAOAState(g, "c64")
    s.apply_layers(gamma, np.zeros(2))
    t = s.as_tensor()
    samp = t[torch.tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)
    del t
    assert np.max(np.abs(samp - ref)) < 1e-6 * amp
    s.reset()
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    s.close()
    torch.cuda.empty_cache()
    assert abs(c - 2.0 * p1_closed_form(g0, 0.8, 0.3)) <= 1e-5 * float(np.sum(g.weights))
    assert abs(nrm - 1) < 1e-5
