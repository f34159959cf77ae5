"""The paper-method CPU baseline (Opt_u, baseline/opt_u.c) computes the same QAOA state as the
oracle, up to the global phase exp(i gamma_k |E| / 2) per level that the paper's totRotation form
carries (Eq. UC_opt)."""
import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I


@pytest.mark.parametrize("n,p,mk", [
    (2, 2, lambda: I._canonical(2, [(0, 1)], "edge")), (6, 3, lambda: I.complete(6)),
    (10, 2, lambda: I.regular3(10, 0)), (12, 4, lambda: I.gnp(12, 0.4, 3)), (15, 2, lambda: I.regular3(15, 1)),
])
def test_opt_u_matches_oracle(n, p, mk):
    import baseline
    import oracle
    g = mk()
    gamma, beta = I.angles(p, seed=n)
    ref = oracle.qaoa_state(g, gamma, beta)
    got = baseline.run(g, gamma, beta)
    phase = np.exp(1j * np.sum(gamma) * g.m / 2)
    assert np.linalg.norm(got - phase * ref) <= 1e-12
    c, nrm = baseline.expectation(g, got)
    ref_c, _ = oracle.expectation(g, ref)
    assert abs(c - ref_c) <= 1e-12 * max(1.0, ref_c) and abs(nrm - 1.0) <= 1e-12
