"""Per-state workspace from the library's stream-ordered pool: creating and freeing states in a
loop (the plain one-request-at-a-time path) reuses the freed blocks, results stay the same, and
many states alive at once each get their own workspace."""
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


def test_create_free_loop_reuses_workspace(B):
    import torch
    n = 18
    g = I.regular3(n, 0)
    ga, be = I.angles(3, 0)
    nbytes = B.qaoa_state_bytes(n, "c64")
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def one(grad):
        h = B.qaoa_state_init(g, "c64", buf.data_ptr(), nbytes, stream)
        try:
            if grad:
                return B.qaoa_gradient(h, ga, be, work.data_ptr(), nbytes)
            B.qaoa_apply_layers(h, ga, be)
            return B.qaoa_expectation(h)
        finally:
            B.qaoa_state_free(h)

    ref_f, ref_g = one(False), one(True)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in range(400):
        grad = i % 4 == 3
        out = one(grad)
        if grad:
            assert out[0] == ref_g[0] and np.array_equal(out[1], ref_g[1]) and np.array_equal(out[2], ref_g[2])
        else:
            assert out == ref_f
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the pool hands the freed blocks to the next state instead of growing
    assert free0 - free1 < (64 << 20), (free0, free1)


def test_many_states_alive_at_once(B):
    import torch
    n, count = 16, 96
    graphs = [I.gnp(n, 0.4, s) for s in range(count)]
    ga, be = I.angles(2, 5)
    nbytes = B.qaoa_state_bytes(n, "c64")
    bufs = torch.empty((count, nbytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hs = [B.qaoa_state_init(g, "c64", bufs[i].data_ptr(), nbytes, stream) for i, g in enumerate(graphs)]
    try:
        for h in hs:
            B.qaoa_apply_layers(h, ga, be)
        got = [B.qaoa_expectation(h)[0] for h in hs]
    finally:
        for h in hs:
            B.qaoa_state_free(h)
    # each alone, one at a time: the same values (every state had its own workspace)
    for i, g in enumerate(graphs[:12]):
        s = B.QAOAState(g, "c64")
        s.apply_layers(ga, be)
        assert s.expectation()[0] == got[i]
        s.close()
