"""qaoa_expectation_static: <C> and norm of a device state with no allocation at all.

Some callers cannot allocate device memory at the moment they need <C>: a serving runtime
that has already handed all of the GPU's memory to its own pool, or a tight optimisation loop
that must not pay the device-wide synchronisation that cudaMalloc/cudaFree can cause.  For them
the library has qaoa_expectation_static, which keeps its scratch in a fixed 1 MiB device array
inside the library instead of workspace it would allocate.

These tests call it through the C ABI on states produced by the regular entry points and
check it against qaoa_expectation (complex64: within 1e-5 * |E|; complex128: within 1e-12
relative), twice in a row, since consecutive calls reuse the same scratch array.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I

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


CASES = [
    (12, "c64", lambda: I.gnp(12, 0.5, 1)),      # whole state in one CTA
    (13, "c128", lambda: I.regular3(13, 2)),     # whole state in one CTA
    (20, "c64", lambda: I.regular3(20, 3)),      # tiled
    (22, "c128", lambda: I.gnp(22, 0.3, 4)),     # tiled
    (29, "c64", lambda: I.regular3(29, 5)),      # largest complex64 size the scratch allows
    (28, "c128", lambda: I.regular3(28, 6)),     # largest complex128 size
]


@pytest.mark.parametrize("n,prec,mk", CASES)
def test_static_expectation_matches_regular_entry(B, n, prec, mk):
    import torch
    g = mk()
    gamma, beta = I.angles(3, n)
    s = B.QAOAState(g, prec)
    s.apply_layers(gamma, beta)
    ref_c, ref_n = s.expectation()
    for _ in range(2):
        c, nrm = B.qaoa_expectation_static(g, prec, s.buffer.data_ptr(), s.nbytes, s.stream.cuda_stream)
        if prec == "c64":
            assert abs(c - ref_c) <= 1e-5 * max(1, g.m)
            assert abs(nrm - ref_n) <= 1e-5
        else:
            assert abs(c - ref_c) <= 1e-12 * abs(ref_c)
            assert abs(nrm - ref_n) <= 1e-12
    s.close()
    torch.cuda.empty_cache()


def test_static_expectation_alternating_sizes(B):
    """Back-to-back calls on different states reuse the scratch array without stale values."""
    states = []
    for n, prec, mk in CASES[:4]:
        g = mk()
        gamma, beta = I.angles(2, 100 + n)
        s = B.QAOAState(g, prec)
        s.apply_layers(gamma, beta)
        states.append((g, prec, s, s.expectation()))
    for _ in range(2):
        for g, prec, s, (ref_c, _) in states:
            c, _ = B.qaoa_expectation_static(g, prec, s.buffer.data_ptr(), s.nbytes, s.stream.cuda_stream)
            tol = 1e-5 * max(1, g.m) if prec == "c64" else 1e-12 * abs(ref_c)
            assert abs(c - ref_c) <= tol
    for *_, s, _r in states:
        s.close()


def test_static_expectation_matches_the_oracle(B):
    """One comparison with the oracle itself (not only with the library's other entry): the
    oracle's complex128 state is written to the device and both precisions of the static entry
    reduce it (complex128 within 1e-12 relative of the oracle's <C>; complex64, on the state
    rounded to complex64, within 1e-5 |E|).  A weights array of ones is the unit-weight graph."""
    import oracle
    import torch
    for n, mk in ((11, lambda: I.gnp(11, 0.4, 3)), (19, lambda: I.regular3(19, 4))):
        g = mk()
        gamma, beta = I.angles(3, 50 + n)
        psi = oracle.qaoa_state(g, gamma, beta)
        ref_c, ref_n = oracle.expectation(g, psi)
        ones = I.Graph(g.n, g.edges, np.ones(g.m))
        for prec, dt in (("c128", torch.complex128), ("c64", torch.complex64)):
            t = torch.from_numpy(psi).to(dt).cuda()
            nbytes = t.numel() * t.element_size()
            for gg in (g, ones):
                c, nrm = B.qaoa_expectation_static(gg, prec, t.data_ptr(), nbytes, 0)
                if prec == "c128":
                    assert abs(c - ref_c) <= 1e-12 * abs(ref_c) and abs(nrm - ref_n) <= 1e-12
                else:
                    assert abs(c - ref_c) <= 1e-5 * g.m and abs(nrm - ref_n) <= 1e-5
            del t


def test_static_expectation_refuses_bad_targets(B):
    """Refused on the host before any launch: a pinned host buffer, an unregistered host
    buffer, a stream under capture, and a weight other than 1."""
    import torch
    g = I.ring(10)
    nbytes = B.qaoa_state_bytes(10, "c64")
    pinned = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    plain = np.zeros(nbytes // 8 + 2, dtype=np.complex64)
    addr = plain.ctypes.data + (-plain.ctypes.data) % 16
    for ptr in (pinned.data_ptr(), addr):
        with pytest.raises(B.QAOAError) as ei:
            B.qaoa_expectation_static(g, "c64", ptr, nbytes, 0)
        assert ei.value.status == B.QAOA_ERR_INVALID
        assert "not device memory" in str(ei.value)
    dev = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(graph, stream=side):
        try:
            B.qaoa_expectation_static(g, "c64", dev.data_ptr(), nbytes, side.cuda_stream)
        except B.QAOAError as e:
            refused = e
    assert refused is not None and refused.status == B.QAOA_ERR_INVALID
    assert "captured" in str(refused)
    heavy = I.Graph(g.n, g.edges, np.full(g.m, 2.0))
    with pytest.raises(B.QAOAError) as ei:
        B.qaoa_expectation_static(heavy, "c64", dev.data_ptr(), nbytes, 0)
    assert ei.value.status == B.QAOA_ERR_UNSUPPORTED
    torch.cuda.synchronize()


def test_static_expectation_rejects_sizes_beyond_its_scratch(B):
    import torch
    buf = torch.empty(16, dtype=torch.uint8, device="cuda")
    # rejected on the host before any kernel runs
    for n, prec in [(30, "c64"), (29, "c128")]:
        g = I.ring(n)
        with pytest.raises(B.QAOAError) as ei:
            B.qaoa_expectation_static(g, prec, buf.data_ptr(), B.qaoa_state_bytes(n, prec), 0)
        assert ei.value.status == B.QAOA_ERR_INVALID
        assert "supports n <=" in str(ei.value)
    with pytest.raises(B.QAOAError):  # buffer smaller than the state
        B.qaoa_expectation_static(I.ring(10), "c64", buf.data_ptr(), 16, 0)
