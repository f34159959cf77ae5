"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: cut values bit-exact; complex128 <C> within 1e-12 relative and the state within
1e-12 in the 2-norm; complex64 <C> within 1e-5 * |E|, state fidelity >= 1 - 1e-5, and every
amplitude within the rounding bound of tests/tolerances.py (c64_amp_tol).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I
from tests.tolerances import C64_AMP_K, U32, c64_amp_tol

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03019_b300 import build
    build.build()
    from paper_2312_03019_b300 import binding
    return binding


def run(B, g, gamma, beta, prec):
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, beta)
    c, nrm = s.expectation()
    psi = s.amplitudes()
    s.close()
    return c, nrm, psi.astype(np.complex128)


def check_c128(g, c, nrm, psi, ref_psi, p=None):
    ref_c, _ = oracle_expectation(g, ref_psi)
    assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
    assert abs(nrm - 1.0) < 1e-12
    assert np.linalg.norm(psi - ref_psi) <= 1e-12


def check_c64(g, c, nrm, psi, ref_psi, p):
    ref_c, _ = oracle_expectation(g, ref_psi)
    assert abs(c - ref_c) <= 1e-5 * max(1, g.m)
    assert abs(nrm - 1.0) < 1e-5
    fid = abs(np.vdot(ref_psi, psi)) ** 2
    assert fid >= 1 - 1e-5
    err = float(np.max(np.abs(psi - ref_psi)))
    assert err <= c64_amp_tol(g.n, p, ref_psi), (err, c64_amp_tol(g.n, p, ref_psi))


def oracle_expectation(g, psi):
    import oracle
    return oracle.expectation(g, psi)


# ----------------------------------------------------------------------------- cut values

CUT_GRAPHS = [
    lambda n: I.empty(n), lambda n: I.complete(n), lambda n: I.star(n), lambda n: I.ring(n) if n >= 3 else I.empty(n),
    lambda n: I.gnp(n, 0.5, n), lambda n: I.gnp(n, 0.2, 100 + n),
    lambda n: I.regular3(n, n) if n >= 4 else I.empty(n),
]


@pytest.mark.parametrize("n", list(range(1, 23)))
def test_cut_table_bit_exact(B, n):
    import oracle
    for mk in CUT_GRAPHS:
        g = mk(n)
        if n > 18 and g.m > 120:
            continue  # keep the oracle's edge loop quick
        got = B.qaoa_cut_table(g)
        assert np.array_equal(got, oracle.cut_table(g)), g.name


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [15, 17, 20, 23, 26])
def test_cut_count_every_tile_geometry(B, prec, n):
    """The tile kernels split C(z) per CTA / thread / register (the on-the-fly Algorithm 3);
    every group geometry and register layout must reproduce the plain edge-loop count."""
    import oracle
    groups = B.qaoa_plan_describe(n, prec, 1)[3]
    for g in (I.gnp(n, 0.5, 7), I.regular3(n, 3) if n % 2 == 0 else I.gnp(n, 0.15, 9), I.complete(min(n, 26))):
        if g.n != n:
            continue
        ref = oracle.cut_table(g)
        for grp in range(groups):
            for layout in range(3):
                got = B.qaoa_cut_table_geometry(g, prec, grp, layout)
                assert np.array_equal(got, ref), (g.name, grp, layout)


# ----------------------------------------------------------------------------- small and mid sizes

@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,p,mk", [
    (1, 2, lambda n: I.empty(1)), (2, 3, lambda n: I._canonical(2, [(0, 1)], "edge")),
    (5, 2, lambda n: I.complete(5)), (8, 4, lambda n: I.gnp(8, 0.5, 1)), (10, 3, lambda n: I.regular3(10, 0)),
    (12, 2, lambda n: I.gnp(12, 0.3, 2)), (13, 5, lambda n: I.regular3(13, 1)), (14, 3, lambda n: I.gnp(14, 0.5, 3)),
    (15, 3, lambda n: I.gnp(15, 0.4, 4)), (16, 4, lambda n: I.regular3(16, 5)), (17, 2, lambda n: I.complete(17)),
    (18, 5, lambda n: I.gnp(18, 0.3, 6)), (19, 3, lambda n: I.regular3(19, 7)), (21, 2, lambda n: I.gnp(21, 0.25, 8)),
])
def test_state_parity(B, prec, n, p, mk):
    import oracle
    g = mk(n)
    gamma, beta = I.angles(p, seed=n)
    ref = oracle.qaoa_state(g, gamma, beta)
    c, nrm, psi = run(B, g, gamma, beta, prec)
    (check_c128 if prec == "c128" else check_c64)(g, c, nrm, psi, ref, p)


def test_config_n10_regular3_p1(B):
    """3-regular n=10, p=1, gamma=0.4, beta=0.3, complex128: full state, <C>, closed form."""
    import oracle
    from tests.test_oracle_pins import p1_closed_form
    g, gamma, beta = I.workload_n10_regular3_p1()
    ref = oracle.qaoa_state(g, gamma, beta)
    c, nrm, psi = run(B, g, gamma, beta, "c128")
    check_c128(g, c, nrm, psi, ref)
    assert abs(c - p1_closed_form(g, 0.4, 0.3)) < 1e-12 * g.m


@pytest.mark.parametrize("name,prec", [("regular3_n22_p6", "c128"), ("regular3_n22_p6", "c64"),
                                       ("gnp24_p10", "c128"), ("gnp24_p10", "c64"),
                                       ("gnp26_p4", "c128"), ("gnp26_p4", "c64")])
def test_golden_large(B, name, prec):
    """Stored oracle results (written by tests/golden/make_golden.py from the oracle only)."""
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{name}.json not generated")
    rec = json.load(open(path))
    g = I.Graph(rec["n"], np.array(rec["edges"], dtype=np.int32))
    s = B.QAOAState(g, prec)
    s.apply_layers(rec["gamma"], rec["beta"])
    c, nrm = s.expectation()
    t = s.as_tensor()
    import torch
    idx = torch.tensor(rec["sample_index"], dtype=torch.int64, device=t.device)
    samp = t[idx].cpu().numpy().astype(np.complex128)
    s.close()
    ref = np.array(rec["sample_re"]) + 1j * np.array(rec["sample_im"])
    if prec == "c128":
        assert abs(c - rec["expectation"]) <= 1e-12 * abs(rec["expectation"])
        assert abs(nrm - 1) < 1e-12
        assert np.max(np.abs(samp - ref)) < 1e-14
    else:
        assert abs(c - rec["expectation"]) <= 1e-5 * rec["m"]
        assert abs(nrm - 1) < 1e-5
        amp = 2 ** (-rec["n"] / 2)
        assert np.max(np.abs(samp - ref)) < 2e-5 * amp * math.sqrt(len(rec["gamma"]))


def test_c64_matches_c128_full_state_n26(B):
    g, gamma, beta = I.workload_gnp26_p4()
    c1, n1, a = run(B, g, gamma, beta, "c128")
    c2, n2, b = run(B, g, gamma, beta, "c64")
    assert abs(c1 - c2) <= 1e-5 * g.m
    assert abs(np.vdot(a, b)) ** 2 >= 1 - 1e-5
    assert np.max(np.abs(a - b)) <= c64_amp_tol(g.n, len(gamma), a)


# ----------------------------------------------------------------------------- semantics / edge cases

@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [9, 18])
def test_split_calls_equal_one_call(B, prec, n):
    g = I.gnp(n, 0.4, 3)
    gamma, beta = I.angles(5, 3)
    s1 = B.QAOAState(g, prec)
    s1.apply_layers(gamma, beta)
    a = s1.amplitudes()
    s2 = B.QAOAState(g, prec)
    s2.apply_layers(gamma[:2], beta[:2])
    s2.apply_layers(gamma[2:], beta[2:])
    b = s2.amplitudes()
    tol = 1e-13 if prec == "c128" else 1e-6
    assert np.max(np.abs(a - b)) < tol * 2 ** (-n / 2) * 10


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [16, 21])
def test_read_out_between_calls(B, prec, n):
    """Reading the state between calls (copy out, the torch view, which resolve the pending
    complement and the complex64 parity form) and continuing gives the oracle's state; so does
    a caller's write through the view."""
    import oracle
    import torch
    g = I.regular3(n, 9) if n % 2 == 0 else I.gnp(n, 0.3, 9)
    gamma, beta = I.angles(4, 11)
    beta[1] = 1.3  # |tan beta| > 1: a pending complement
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma[:1], beta[:1])
    mid = s.amplitudes()
    assert np.linalg.norm(mid - oracle.qaoa_state(g, gamma[:1], beta[:1])) <= (1e-12 if prec == "c128" else 1e-5)
    s.apply_layers(gamma[1:2], beta[1:2])
    view = s.as_tensor()  # canonical in place
    view.mul_(1.0)
    torch.cuda.synchronize()
    s.apply_layers(gamma[2:], beta[2:])
    c, _ = s.expectation()
    psi = s.amplitudes().astype(np.complex128)
    s.close()
    ref = oracle.qaoa_state(g, gamma, beta)
    (check_c128 if prec == "c128" else check_c64)(g, c, 1.0, psi, ref, len(gamma))


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [6, 16])
def test_initial_state_and_zero_levels(B, prec, n):
    g = I.gnp(n, 0.5, 1)
    s = B.QAOAState(g, prec)
    c, nrm = s.expectation()  # deferred |+>^n
    assert abs(c - g.m / 2) < 1e-12 * g.m + (1e-6 * g.m if prec == "c64" else 0)
    s.apply_layers([], [])  # p = 0 writes |+>^n out
    psi = s.amplitudes()
    assert np.allclose(psi, 2 ** (-n / 2), rtol=0, atol=1e-7 * 2 ** (-n / 2))
    c2, _ = s.expectation()
    assert abs(c2 - c) < 1e-6 * g.m


def test_invalid_angles_rejected(B):
    s = B.QAOAState(I.ring(6), "c64")
    with pytest.raises(B.QAOAError):
        s.apply_layers([float("nan")], [0.1])
    with pytest.raises(B.QAOAError):
        s.apply_layers([0.1], [float("inf")])


def test_deterministic_expectation(B):
    g, gamma, beta = I.workload_gnp24_p10()
    vals = []
    for _ in range(2):
        s = B.QAOAState(g, "c64")
        s.apply_layers(gamma, beta)
        vals.append(s.expectation())
        s.close()
    assert vals[0] == vals[1]


def test_many_levels_crosses_coefficient_chunks(B):
    import oracle
    g = I.regular3(16, 2)
    gamma, beta = I.angles(70, 2)
    ref = oracle.qaoa_state(g, gamma, beta)
    c, nrm, psi = run(B, g, gamma, beta, "c128")
    check_c128(g, c, nrm, psi, ref)


# ----------------------------------------------------------------------------- full size (n = 33)

@pytest.mark.slow
def test_full_size_n33_properties(B):
    """Near-3-regular n = 33 in complex64 (64 GiB): the run of the benchmark, checked where the
    oracle can compute values one by one: beta = 0 gives psi_z = 2^(-n/2) exp(-i sum gamma C(z))
    amplitude by amplitude; p = 1 matches the closed-form <C>; the p = 8 run keeps the norm,
    the complement symmetry and 0 <= <C> <= |E|."""
    import oracle
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g, gamma, beta = I.workload_regular3_n33_p8()
    n = g.n
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 256), [0, (1 << n) - 1, 1 << 32, (1 << 32) + 5]]))
    s = B.QAOAState(g, "c64")
    # beta = 0: pure cost phases, sampled amplitude by amplitude against the oracle's cut value
    s.apply_layers(gamma[:3], np.zeros(3))
    t = s.as_tensor()
    samp = t[torch.tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)
    amp = 2 ** (-n / 2)
    ref = np.array([amp * np.exp(-1j * gamma[:3].sum() * oracle.cut_value(g, int(z))) for z in idx])
    assert np.max(np.abs(samp - ref)) < 1e-5 * amp
    s.close()
    del t
    torch.cuda.empty_cache()
    # p = 1 closed form
    s = B.QAOAState(g, "c64")
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    assert abs(c - p1_closed_form(g, 0.4, 0.3)) <= 1e-5 * g.m
    assert abs(nrm - 1) < 1e-5
    s.close()
    torch.cuda.empty_cache()
    # the benchmark's p = 8 run
    s = B.QAOAState(g, "c64")
    s.apply_layers(gamma, beta)
    c, nrm = s.expectation()
    assert abs(nrm - 1) < 1e-4 and 0 <= c <= g.m
    t = s.as_tensor()
    a = t[torch.tensor(idx, device=t.device)].cpu().numpy()
    b = t[torch.tensor(((1 << n) - 1) ^ idx, device=t.device)].cpu().numpy()
    assert np.max(np.abs(a - b)) < 1e-5 * amp
    s.close()
    del t
    torch.cuda.empty_cache()


def test_max_size_n34_complex64(B):
    """The largest state the library takes, n = 34 (exact 3-regular, 51 edges; complex64, 128 GiB,
    four mixer groups): p = 1 matches the closed-form <C>; beta = 0 gives the cost phases
    amplitude by amplitude (sampled against the oracle's cut value, the highest index bits
    included); a p = 3 run keeps the norm and the complement symmetry."""
    import oracle
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g = I.regular3(34, 0)
    gamma, beta = I.angles(3, 34)
    n = g.n
    amp = 2 ** (-n / 2)
    rng = np.random.default_rng(34)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 256), [0, (1 << n) - 1, 1 << 33, (1 << 33) + 7]]))
    s = B.QAOAState(g, "c64")
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    assert abs(c - p1_closed_form(g, 0.4, 0.3)) <= 1e-5 * g.m
    assert abs(nrm - 1) < 1e-5
    s.reset()
    s.apply_layers(gamma, np.zeros(3))
    t = s.as_tensor()
    samp = t[torch.tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)
    ref = np.array([amp * np.exp(-1j * gamma.sum() * oracle.cut_value(g, int(z))) for z in idx])
    assert np.max(np.abs(samp - ref)) < 1e-5 * amp
    del t
    s.reset()
    s.apply_layers(gamma, beta)
    c, nrm = s.expectation()
    assert abs(nrm - 1) < 1e-4 and 0 <= c <= g.m
    t = s.as_tensor()
    a = t[torch.tensor(idx, device=t.device)].cpu().numpy()
    b = t[torch.tensor(((1 << n) - 1) ^ idx, device=t.device)].cpu().numpy()
    assert np.max(np.abs(a - b)) < 1e-5 * amp
    s.close()
    del t
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_max_size_n34_complex128_closed_form(B):
    """The largest complex128 state, n = 34 (256 GiB): p = 1 against the closed form to 1e-12."""
    import torch
    from tests.test_oracle_pins import p1_closed_form
    free, _ = torch.cuda.mem_get_info()
    if free < B.qaoa_state_bytes(34, "c128") + (2 << 30):
        pytest.skip("needs 258 GiB of free device memory")
    g = I.regular3(34, 0)
    s = B.QAOAState(g, "c128")
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    s.close()
    torch.cuda.empty_cache()
    assert abs(c - p1_closed_form(g, 0.4, 0.3)) <= 1e-12 * c
    assert abs(nrm - 1) < 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("n", [30, 33])
def test_full_size_c128_closed_form(B, n):
    """complex128 at n = 30 (16 GiB) and n = 33 (128 GiB): p = 1 <C> equals the closed form to
    1e-12 relative."""
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g = I.regular3(n, 0)
    s = B.QAOAState(g, "c128")
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    ref = p1_closed_form(g, 0.4, 0.3)
    assert abs(c - ref) <= 1e-12 * ref
    assert abs(nrm - 1) < 1e-12
    s.close()
    torch.cuda.empty_cache()


def _c64_against_c128_on_device(B, g, gamma, beta):
    """Runs the circuit in both precisions on the GPU and returns (fidelity, <C> c64, <C> c128,
    norm c128, largest amplitude difference), the overlap taken on the device in chunks."""
    import torch
    s128 = B.QAOAState(g, "c128")
    s128.apply_layers(gamma, beta)
    c128, n128 = s128.expectation()
    s64 = B.QAOAState(g, "c64")
    s64.apply_layers(gamma, beta)
    c64, n64 = s64.expectation()
    t128, t64 = s128.as_tensor(), s64.as_tensor()
    ip = torch.zeros((), dtype=torch.complex128, device=t64.device)
    worst, amax = 0.0, 0.0
    chunk = 1 << 28
    for i in range(0, t64.numel(), chunk):
        a = t64[i:i + chunk].to(torch.complex128)
        b = t128[i:i + chunk]
        ip += torch.vdot(b, a)
        worst = max(worst, (a - b).abs().max().item())
        amax = max(amax, b.abs().max().item())
        del a, b
    fid = abs(ip.item()) ** 2 / (n64 * n128)
    del t128, t64
    s128.close()
    s64.close()
    torch.cuda.empty_cache()
    return fid, c64, c128, n128, worst, amax


@pytest.mark.parametrize("n", [30, 33])
def test_full_size_c64_against_c128(B, n):
    """The benchmark's runs (3-regular n = 30 and near-3-regular n = 33, seed 0, p = 8 seeded
    levels) in complex64 against the same runs in complex128 on the GPU (at n = 33, 64 + 128 GiB
    on the device together): fidelity >= 1 - 1e-5 and <C> within 1e-5 |E|.  The complex128 path
    is pinned at these sizes by the p = 1 closed form."""
    g = I.regular3(n, 0)
    gamma, beta = I.angles(8, 0)
    fid, c64, c128, n128, worst, amax = _c64_against_c128_on_device(B, g, gamma, beta)
    assert abs(n128 - 1) < 1e-12
    assert fid >= 1 - 1e-5, fid
    assert abs(c64 - c128) <= 1e-5 * g.m, (c64, c128)
    tol = C64_AMP_K * U32 * math.sqrt(len(gamma) * (g.n + 2)) * amax
    assert worst <= tol, (worst, tol)


@pytest.mark.parametrize("n,prec", [(32, "c64"), (32, "c128"), (34, "c64")])
def test_complete_graph_cut_values_above_255(B, n, prec):
    """The complete graph K_n at n = 32 and 34 (496 and 561 edges, the most the library takes at
    n = 34): C(z) = |z| (n - |z|) reaches 256 and 289, beyond one byte, so the phase tables run
    past entry 255.  beta = 0 gives psi_z = 2^(-n/2) exp(-i sum gamma |z| (n - |z|)) for sampled
    z (balanced Hamming weights included), and p = 1 matches the closed form."""
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g = I.complete(n)
    assert g.m == n * (n - 1) // 2
    rng = np.random.default_rng(n)
    half = (1 << (n // 2)) - 1
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 200), [0, (1 << n) - 1, half, half << (n - n // 2),
                                                                    0x5555555555555555 & ((1 << n) - 1)]]))
    w = np.array([bin(int(z)).count("1") for z in idx])
    assert (w * (n - w)).max() == (n // 2) * (n - n // 2)
    gamma = np.array([0.7, 2.3])
    amp = 2.0 ** (-n / 2)
    ref = amp * np.exp(-1j * gamma.sum() * (w * (n - w)))
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, np.zeros(2))
    t = s.as_tensor()
    samp = t[torch.tensor(idx, device=t.device)].cpu().numpy().astype(np.complex128)
    del t
    assert np.max(np.abs(samp - ref)) < (1e-11 if prec == "c128" else 1e-6) * amp
    s.reset()
    s.apply_layers([0.4], [0.3])
    c, nrm = s.expectation()
    s.close()
    torch.cuda.empty_cache()
    ref_c = p1_closed_form(g, 0.4, 0.3)
    if prec == "c128":
        assert abs(c - ref_c) <= 1e-12 * abs(ref_c) and abs(nrm - 1) < 1e-12
    else:
        assert abs(c - ref_c) <= 1e-5 * g.m and abs(nrm - 1) < 1e-5


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,mk", [
    (5, lambda n: I.complete(n)), (11, lambda n: I.gnp(n, 0.4, 11)), (14, lambda n: I.regular3(n, 2)),
    (16, lambda n: I.gnp(n, 0.3, 16)), (19, lambda n: I.regular3(n, 3)), (21, lambda n: I.gnp(n, 0.25, 21)),
])
def test_mixer_only_and_phase_only(B, prec, n, mk):
    """The two halves of a level alone, whole state, every plan shape from one CTA to two and
    three groups.  gamma = 0: |+>^n is an eigenstate of every X, so psi_z = 2^(-n/2)
    exp(-i n sum beta) for every z (beta up to pi: the |tan beta| > 1 form with its pending
    complement is used).  beta = 0: psi_z = 2^(-n/2) exp(-i sum gamma C(z)) with the oracle's
    cut values."""
    import oracle
    g = mk(n)
    gamma, beta = I.angles(3, seed=n, gamma_hi=math.pi, beta_hi=math.pi)
    amp = 2.0 ** (-n / 2)
    tol = (1e-12 if prec == "c128" else 1e-5) * amp
    _, _, psi = run(B, g, np.zeros(3), beta, prec)
    assert np.max(np.abs(psi - amp * np.exp(-1j * n * beta.sum()))) < tol
    _, _, psi = run(B, g, gamma, np.zeros(3), prec)
    ref = amp * np.exp(-1j * gamma.sum() * oracle.cut_table(g).astype(np.float64))
    assert np.max(np.abs(psi - ref)) < (1e-12 if prec == "c128" else 1e-6) * amp


def test_states_on_concurrent_host_threads(B):
    """Distinct state handles used from four host threads at once, each on its own CUDA stream
    (small-state and tiled paths, both precisions): every result equals, bit for bit, the same
    run done alone."""
    import threading
    import torch
    jobs = [(I.regular3(n, n) if n % 2 == 0 else I.gnp(n, 0.4, n), prec, *I.angles(3, seed=n))
            for n, prec in ((9, "c64"), (16, "c64"), (22, "c128"), (24, "c64"), (13, "c128"), (26, "c64"),
                            (20, "c64"), (18, "c128"))]

    def run_one(job):
        g, prec, gamma, beta = job
        s = B.QAOAState(g, prec, stream=torch.cuda.Stream())
        with torch.cuda.stream(s.stream):
            s.apply_layers(gamma, beta)
            c, nrm = s.expectation()
            psi = s.amplitudes() if g.n <= 16 else None
        s.close()
        return c, nrm, psi

    serial = [run_one(j) for j in jobs]
    out = [None] * len(jobs)
    errors = []

    def worker(k):
        try:
            for i in range(k, len(jobs), 4):
                for _ in range(2):
                    out[i] = run_one(jobs[i])
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for (c0, n0, p0), (c1, n1, p1) in zip(serial, out):
        assert c0 == c1 and n0 == n1
        if p0 is not None:
            assert np.array_equal(p0, p1)
