"""GPU adjoint gradient d<C>/d(gamma_k, beta_k) (qaoa_gradient) against the FP64 CPU oracle adjoint
and against central finite differences (h = 1e-4) evaluated in complex128 on the GPU."""
import json
import os

import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I
from tests.tolerances import FD_TOL, c64_grad_tol

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


def gpu_gradient(B, g, gamma, beta, prec):
    import torch
    s = B.QAOAState(g, prec)
    work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
    c, dg, db = B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)
    s.close()
    return c, dg, db


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,p,mk", [
    (2, 2, lambda: I._canonical(2, [(0, 1)], "edge")), (6, 3, lambda: I.complete(6)),
    (10, 4, lambda: I.regular3(10, 0)), (12, 2, lambda: I.gnp(12, 0.5, 1)),
    (13, 3, lambda: I.regular3(13, 2)), (14, 5, lambda: I.gnp(14, 0.5, 0)),
    (16, 3, lambda: I.regular3(16, 4)), (18, 2, lambda: I.gnp(18, 0.3, 5)),
])
def test_gradient_matches_oracle_adjoint(B, prec, n, p, mk):
    import oracle
    g = mk()
    gamma, beta = I.angles(p, seed=n + 7)
    ref_c, ref_dg, ref_db = oracle.adjoint_gradient(g, gamma, beta)
    c, dg, db = gpu_gradient(B, g, gamma, beta, prec)
    scale = max(1.0, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
    if prec == "c128":
        assert abs(c - ref_c) <= 1e-12 * max(1.0, abs(ref_c))
        assert np.max(np.abs(dg - ref_dg)) <= 1e-10 * scale
        assert np.max(np.abs(db - ref_db)) <= 1e-10 * scale
    else:
        tol = c64_grad_tol(n, p, g.m, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
        assert abs(c - ref_c) <= 1e-5 * g.m
        assert np.max(np.abs(dg - ref_dg)) <= tol
        assert np.max(np.abs(db - ref_db)) <= tol


def test_gradient_workload_g24_p10_against_finite_differences(B):
    """G(24, 0.5), p = 10, complex64 adjoint gradient vs central differences (h = 1e-4) of <C>
    evaluated in complex128 on the GPU (40 evaluations)."""
    g, gamma, beta = I.workload_gnp24_p10()
    c, dg, db = gpu_gradient(B, g, gamma, beta, "c64")
    s = B.QAOAState(g, "c128")
    h = 1e-4

    def f(ga, be):
        s.reset()
        s.apply_layers(ga, be)
        return s.expectation()[0]

    c128 = f(gamma, beta)
    assert abs(c - c128) <= 1e-5 * g.m
    fd_g = np.zeros(10)
    fd_b = np.zeros(10)
    for k in range(10):
        e = np.zeros(10)
        e[k] = h
        fd_g[k] = (f(gamma + e, beta) - f(gamma - e, beta)) / (2 * h)
        fd_b[k] = (f(gamma, beta + e) - f(gamma, beta - e)) / (2 * h)
    s.close()
    scale = np.max(np.abs(np.concatenate([fd_g, fd_b])))
    tol = c64_grad_tol(g.n, 10, g.m, scale) + FD_TOL
    assert np.max(np.abs(dg - fd_g)) <= tol
    assert np.max(np.abs(db - fd_b)) <= tol


def test_gradient_fp64_cpu_adjoint_n14_p10(B):
    """The FP64 CPU adjoint on G(14, 0.5), p = 10 against both GPU precisions."""
    import oracle
    g = I.gnp(14, 0.5, 0)
    gamma, beta = I.angles(10, 0)
    ref_c, ref_dg, ref_db = oracle.adjoint_gradient(g, gamma, beta)
    scale = max(1.0, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
    c, dg, db = gpu_gradient(B, g, gamma, beta, "c128")
    assert np.max(np.abs(np.concatenate([dg - ref_dg, db - ref_db]))) <= 1e-10 * scale
    c, dg, db = gpu_gradient(B, g, gamma, beta, "c64")
    assert np.max(np.abs(np.concatenate([dg - ref_dg, db - ref_db]))) <= c64_grad_tol(14, 10, g.m, scale)


def test_gradient_then_state_is_plus_and_reusable(B):
    import torch
    g = I.regular3(18, 1)
    gamma, beta = I.angles(3, 1)
    s = B.QAOAState(g, "c64")
    work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
    c1, dg1, db1 = B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)
    c0, _ = s.expectation()  # |+>^n again
    assert abs(c0 - g.m / 2) < 1e-4 * g.m
    c2, dg2, db2 = B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)
    assert c1 == c2 and np.array_equal(dg1, dg2) and np.array_equal(db1, db2)  # run to run identical
    s.apply_layers(gamma, beta)
    c3, _ = s.expectation()
    assert abs(c3 - c1) < 1e-5 * g.m
    s.close()


def test_gradient_rejects_bad_work_buffer(B):
    import torch
    g = I.ring(16)
    s = B.QAOAState(g, "c64")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.QAOAError):
        B.qaoa_gradient(s.handle, [0.1], [0.2], small.data_ptr(), 64)
    with pytest.raises(B.QAOAError):
        B.qaoa_gradient(s.handle, [0.1], [0.2], s.buffer.data_ptr(), s.nbytes)
    with pytest.raises(B.QAOAError):
        B.qaoa_gradient(s.handle, [], [], s.buffer.data_ptr(), s.nbytes)
    s.close()


def test_autograd_function(B):
    import torch
    from paper_2312_03019_b300.autograd import qaoa_expectation_fn
    g = I.regular3(16, 3)
    gamma = torch.tensor(I.angles(4, 3)[0], requires_grad=True)
    beta = torch.tensor(I.angles(4, 3)[1], requires_grad=True)
    s = B.QAOAState(g, "c128")
    val = qaoa_expectation_fn(gamma, beta, s)
    (2.0 * val).backward()
    c, dg, db = gpu_gradient(B, g, gamma.detach().numpy(), beta.detach().numpy(), "c128")
    assert abs(val.item() - c) < 1e-12 * abs(c)
    assert np.allclose(gamma.grad.numpy(), 2.0 * dg, rtol=0, atol=1e-12)
    assert np.allclose(beta.grad.numpy(), 2.0 * db, rtol=0, atol=1e-12)
    s.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [10, 16])
def test_gradient_more_levels_than_one_coefficient_chunk(B, prec, n):
    """p = 70 crosses the 64-level coefficient chunks of the forward run; the adjoint sweep's
    tables cover all levels (one-CTA sweep at n = 10, tiled sweep at n = 16)."""
    import oracle
    g = I.regular3(n, 5)
    gamma, beta = I.angles(70, n + 200)
    gamma *= 0.2  # keep <C> away from its extremes, where all derivatives are tiny
    ref_c, ref_dg, ref_db = oracle.adjoint_gradient(g, gamma, beta)
    c, dg, db = gpu_gradient(B, g, gamma, beta, prec)
    scale = max(1.0, np.max(np.abs(np.concatenate([ref_dg, ref_db]))))
    tol = 1e-10 * scale if prec == "c128" else c64_grad_tol(n, 70, g.m, scale)
    assert abs(c - ref_c) <= (1e-12 * abs(ref_c) if prec == "c128" else 1e-5 * g.m)
    assert np.max(np.abs(dg - ref_dg)) <= tol
    assert np.max(np.abs(db - ref_db)) <= tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_empty_graph_tiled(B, prec):
    """No edges at n = 20 (tiled passes, a one-entry phase table): <C> = 0, the state is
    exp(-i n sum beta) |+>^n times 2^(-n/2) per amplitude, every derivative is 0."""
    g = I.empty(20)
    gamma, beta = I.angles(3, 7)
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, beta)
    c, nrm = s.expectation()
    psi = s.amplitudes().astype(np.complex128)
    s.close()
    assert c == 0.0 and abs(nrm - 1) < (1e-12 if prec == "c128" else 1e-5)
    want = 2 ** (-10) * np.exp(-1j * 20 * beta.sum())
    assert np.max(np.abs(psi - want)) < (1e-14 if prec == "c128" else 1e-7)
    c, dg, db = gpu_gradient(B, g, gamma, beta, prec)
    assert c == 0.0 and np.all(dg == 0) and np.all(db == 0)


def test_state_gradient_method_matches_the_c_call(B):
    g = I.gnp(16, 0.4, 2)
    gamma, beta = I.angles(3, 16)
    c0, dg0, db0 = gpu_gradient(B, g, gamma, beta, "c64")
    s = B.QAOAState(g, "c64")
    c1, dg1, db1 = s.gradient(gamma, beta)
    c2, dg2, db2 = s.gradient(gamma, beta)  # the kept work buffer is reused
    s.close()
    assert c0 == c1 == c2 and np.array_equal(dg0, dg1) and np.array_equal(db1, db2)


@pytest.mark.parametrize("n,prec", [(33, "c64"), (30, "c128")])
def test_gradient_full_size_p1_closed_form(B, n, prec):
    """Full size (n = 33 complex64: psi and lambda 64 GiB each; n = 30 complex128), p = 1: the
    adjoint gradient against the derivatives of the closed-form p = 1 <C> (central differences
    of the formula in FP64, h = 1e-5, accurate to about 1e-9)."""
    import torch
    from tests.test_oracle_pins import p1_closed_form
    g = I.regular3(n, 0)
    ga, be = 0.4, 0.3
    c, dg, db = gpu_gradient(B, g, [ga], [be], prec)
    torch.cuda.empty_cache()
    f = lambda x, y: p1_closed_form(g, x, y)
    h = 1e-5
    ref_dg = (f(ga + h, be) - f(ga - h, be)) / (2 * h)
    ref_db = (f(ga, be + h) - f(ga, be - h)) / (2 * h)
    if prec == "c128":
        assert abs(c - f(ga, be)) <= 1e-12 * f(ga, be)
        assert abs(dg[0] - ref_dg) <= 1e-7 * g.m and abs(db[0] - ref_db) <= 1e-7 * g.m
    else:
        tol = c64_grad_tol(n, 1, g.m, max(abs(ref_dg), abs(ref_db))) + 1e-7 * g.m
        assert abs(c - f(ga, be)) <= 1e-5 * g.m
        assert abs(dg[0] - ref_dg) <= tol and abs(db[0] - ref_db) <= tol


GRAD_GOLDEN = ["grad_regular3_n24_p3", "grad_regular3_n25_p3", "grad_regular3_n27_p2", "grad_regular3_n28_p2",
               "grad_regular3_n29_p2"]


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("name", GRAD_GOLDEN)
def test_gradient_stored_oracle_adjoint(B, name, prec):
    """The adjoint gradient at n = 24..29, where the sweep runs its compiled programs (the
    persistent prefetching form in complex64: the first, group-0, fused and last passes, with
    the masks of 6-, 7- and 8-bit high groups, and the three-layout programs of 9-bit groups),
    against the oracle's FP64 adjoint stored by tests/golden/make_golden.py (which calls only
    the oracle)."""
    path = os.path.join(os.path.dirname(__file__), "golden", f"{name}.json")
    rec = json.load(open(path))
    g = I.Graph(rec["n"], np.array(rec["edges"], dtype=np.int32))
    gamma, beta = np.array(rec["gamma"]), np.array(rec["beta"])
    ref_dg, ref_db = np.array(rec["d_gamma"]), np.array(rec["d_beta"])
    c, dg, db = gpu_gradient(B, g, gamma, beta, prec)
    import torch
    torch.cuda.empty_cache()
    big = np.max(np.abs(np.concatenate([ref_dg, ref_db])))
    if prec == "c128":
        scale = max(1.0, big)
        assert abs(c - rec["expectation"]) <= 1e-12 * max(1.0, abs(rec["expectation"]))
        assert np.max(np.abs(dg - ref_dg)) <= 1e-10 * scale
        assert np.max(np.abs(db - ref_db)) <= 1e-10 * scale
    else:
        tol = c64_grad_tol(g.n, len(gamma), g.m, big)
        assert abs(c - rec["expectation"]) <= 1e-5 * g.m
        assert np.max(np.abs(dg - ref_dg)) <= tol
        assert np.max(np.abs(db - ref_db)) <= tol


def test_gradient_many_passes_persistent_sweep(B):
    """n = 22, p = 40: 81 sweep passes in the persistent form, whose per-CTA partials are reduced
    in two batches (64 + 17 passes), against the same gradient in complex128 (one CTA per tile,
    one reduction per pass; pinned to the oracle by the tests above)."""
    g = I.regular3(22, 3)
    gamma, beta = I.angles(40, 321)
    gamma *= 0.2
    c64, dg64, db64 = gpu_gradient(B, g, gamma, beta, "c64")
    c128, dg128, db128 = gpu_gradient(B, g, gamma, beta, "c128")
    big = np.max(np.abs(np.concatenate([dg128, db128])))
    tol = c64_grad_tol(22, 40, g.m, big)
    assert abs(c64 - c128) <= 1e-5 * g.m
    assert np.max(np.abs(dg64 - dg128)) <= tol
    assert np.max(np.abs(db64 - db128)) <= tol
