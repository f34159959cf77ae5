"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test anchors the oracle to something other than itself: the paper's worked example
(Section 2.3, Fig. popcount), hand-enumerated cut values, the published closed form of
p = 1 QAOA on max-cut (Wang, Hadfield, Jiang, Rieffel, Phys. Rev. A 97, 022304, 2018),
textbook identities of the RX mixer (Walsh-Hadamard diagonalisation) and of the diagonal
cost operator, exact invariants, brute-force maximum cuts and finite differences.
"""
import math
import os

import numpy as np
import pytest

from paper_2312_03019_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers

def brute_cut_values(g):
    """C(z) for every z by direct enumeration in numpy (independent of the oracle's C)."""
    z = np.arange(1 << g.n, dtype=np.int64)
    c = np.zeros(1 << g.n, dtype=np.float64)
    w = np.ones(g.m) if g.weights is None else g.weights
    for e, (u, v) in enumerate(g.edges):
        c += w[e] * (((z >> u) ^ (z >> v)) & 1)
    return c


def fwht(a):
    """Unnormalised fast Walsh-Hadamard transform (textbook butterfly)."""
    a = a.copy()
    h = 1
    while h < len(a):
        a = a.reshape(-1, 2, h)
        x, y = a[:, 0, :].copy(), a[:, 1, :].copy()
        a[:, 0, :], a[:, 1, :] = x + y, x - y
        a = a.reshape(-1)
        h *= 2
    return a


def p1_closed_form(g, gamma, beta):
    """<C> of p = 1 QAOA for any unweighted graph (Wang et al. 2018, Eq. for general graphs),
    with cost exp(-i gamma C) and mixer exp(-i beta sum X)."""
    nbr = [set() for _ in range(g.n)]
    for u, v in g.edges:
        nbr[u].add(int(v))
        nbr[v].add(int(u))
    tot = 0.0
    for u, v in g.edges:
        du, dv = len(nbr[u]) - 1, len(nbr[v]) - 1
        lam = len(nbr[u] & nbr[v])
        term = 0.5 + 0.25 * math.sin(4 * beta) * math.sin(gamma) * (math.cos(gamma) ** du + math.cos(gamma) ** dv)
        term -= 0.25 * math.sin(2 * beta) ** 2 * math.cos(gamma) ** (du + dv - 2 * lam) * (1 - math.cos(2 * gamma) ** lam)
        tot += term
    return tot


def single_edge():
    return I._canonical(2, [(0, 1)], "edge")


def triangle():
    return I._canonical(3, [(0, 1), (1, 2), (0, 2)], "K3")


# --------------------------------------------------------------------------- Algorithm 3 worked example

def _read_golden_popcount():
    vals = {}
    with open(os.path.join(GOLDEN, "popcount_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = v
    return vals


def _from_printed(s):
    """Character k of the printed string becomes bit k (the paper's index counts from the left)."""
    return sum(1 << k for k, ch in enumerate(s) if ch == "1")


def test_alg3_worked_example(oracle_lib):
    g = _read_golden_popcount()
    b, row, i = _from_printed(g["b"]), _from_printed(g["graph_I"]), int(g["i"])
    # the reading: bit i of b is set, so b_I is all ones and b_I XOR b is the complement of b
    assert (b >> i) & 1 == 1
    assert (~b) & 0xFF == _from_printed(g["xor"])
    assert (~b) & row & 0xFF == _from_printed(g["and"])
    assert oracle_lib.alg3_term(b, row, i) == int(g["count"])
    # graph_I of node i is upper-triangular under this reading: all neighbours are > i
    assert all(k > i for k in range(8) if (row >> k) & 1)


def test_alg3_worked_example_lsb_form(oracle_lib):
    # the same example written with qubit u = bit u: b = 01101000, graph_I = 11010000 (MSB first)
    assert oracle_lib.alg3_term(0b01101000, 0b11010000, 3) == 2


# --------------------------------------------------------------------------- cut values

def test_cut_values_hand_enumerated(oracle_lib):
    assert list(oracle_lib.cut_table(single_edge())) == [0, 1, 1, 0]
    # triangle: 0 edges cut for 000/111, otherwise exactly 2
    assert list(oracle_lib.cut_table(triangle())) == [0, 2, 2, 2, 2, 2, 2, 0]
    # path 0-1-2: z=010 cuts both edges, z=001 and z=100 cut one each
    path = I._canonical(3, [(0, 1), (1, 2)], "P3")
    assert list(oracle_lib.cut_table(path)) == [0, 1, 2, 1, 1, 2, 1, 0]
    # star K_{1,3} centred at 0: C(z) = number of leaves on the other side of the centre
    st = I.star(4)
    tab = oracle_lib.cut_table(st)
    for z in range(16):
        c0 = z & 1
        assert tab[z] == sum(((z >> v) & 1) != c0 for v in (1, 2, 3))
    # weighted: edges (0,1) w=0.5 and (1,2) w=2: C(010) = 2.5, C(001) = 0.5, C(100) = 2
    wg = I.Graph(3, np.array([[0, 1], [1, 2]], dtype=np.int32), np.array([0.5, 2.0]), "w")
    assert oracle_lib.cut_value(wg, 0b010) == 2.5
    assert oracle_lib.cut_value(wg, 0b001) == 0.5
    assert oracle_lib.cut_value(wg, 0b100) == 2.0


@pytest.mark.parametrize("n,p,seed", [(6, 0.5, 1), (9, 0.4, 2), (11, 0.7, 3), (12, 0.3, 4)])
def test_alg3_matches_edge_loop_and_alg2(oracle_lib, n, p, seed):
    g = I.gnp(n, p, seed)
    graph_I = [0] * n
    for u, v in g.edges:
        graph_I[u] |= 1 << int(v)  # upper-triangular row mask (Table 1)
    tab = oracle_lib.cut_table(g)
    brute = brute_cut_values(g)
    assert np.array_equal(tab.astype(np.float64), brute)
    for z in range(1 << n):
        c, tot_rot = oracle_lib.alg3_cut(n, graph_I, g.m, z)
        assert c == tab[z]
        # totRotation = totEdge - 2 c_neg (Algorithm 3) = Algorithm 2's signed sum
        assert tot_rot == g.m - 2 * c
        assert oracle_lib.alg2_tot_rotation(g, z) == tot_rot


def test_cut_complement_symmetry(oracle_lib):
    g = I.gnp(12, 0.5, 7)
    tab = oracle_lib.cut_table(g)
    full = (1 << g.n) - 1
    z = np.arange(1 << g.n)
    assert np.array_equal(tab, tab[full ^ z])


# --------------------------------------------------------------------------- layers against definitions

def test_initial_layer_is_uniform(oracle_lib):
    psi = oracle_lib.initial_state(7)
    assert np.allclose(psi, 2 ** -3.5, atol=1e-15, rtol=0)


@pytest.mark.parametrize("weighted", [False, True])
def test_cost_layer_is_diagonal_phase(oracle_lib, weighted):
    g = I.gnp(9, 0.5, 11)
    if weighted:
        g = I.random_weights(g, 3)
    psi = I.random_state(g.n, 5)
    gamma = 0.731
    out = oracle_lib.cost_layer(g, gamma, psi)
    expect = np.exp(-1j * gamma * brute_cut_values(g)) * psi
    assert np.max(np.abs(out - expect)) < 1e-13


def test_cost_layer_matches_eq_uc_opt_up_to_global_phase(oracle_lib):
    # Eq. (UC_opt) / Algorithm 2: phase exp(-i/2 gamma_paper totRotation(b)); with gamma_paper
    # = -gamma the two operators differ only by the constant factor exp(-i gamma W / 2).
    g = I.random_weights(I.gnp(8, 0.6, 2), 9)
    psi = I.random_state(g.n, 6)
    gamma = 0.4
    ours = oracle_lib.cost_layer(g, gamma, psi)
    tot = np.array([oracle_lib.alg2_tot_rotation(g, z) for z in range(1 << g.n)])
    paper = np.exp(-0.5j * (-gamma) * tot) * psi
    ratio = ours / paper
    assert np.max(np.abs(ratio - np.exp(-0.5j * gamma * g.weights.sum()))) < 1e-13


def test_mixer_is_walsh_hadamard_diagonal(oracle_lib):
    # exp(-i beta sum_j X_j) = H^n diag(exp(-i beta (n - 2|y|))) H^n
    n = 10
    psi = I.random_state(n, 8)
    beta = 0.377
    out = oracle_lib.mixer_layer(n, beta, psi)
    y = np.arange(1 << n)
    hw = np.array([bin(v).count("1") for v in y])
    ref = fwht(np.exp(-1j * beta * (n - 2 * hw)) * fwht(psi)) / (1 << n)
    assert np.max(np.abs(out - ref)) < 1e-13


# --------------------------------------------------------------------------- p = 1 closed form

@pytest.mark.parametrize("name,gfun", [
    ("edge", single_edge), ("triangle", triangle), ("ring8", lambda: I.ring(8)),
    ("petersen", I.petersen), ("K4", lambda: I.complete(4)), ("star6", lambda: I.star(6)),
    ("reg3_n10", lambda: I.regular3(10, 0)), ("gnp9", lambda: I.gnp(9, 0.5, 3)),
])
@pytest.mark.parametrize("gamma,beta", [(0.4, 0.3), (1.1, -0.7), (2.9, 1.2)])
def test_p1_closed_form(oracle_lib, name, gfun, gamma, beta):
    g = gfun()
    psi = oracle_lib.qaoa_state(g, [gamma], [beta])
    c, nrm = oracle_lib.expectation(g, psi)
    assert abs(nrm - 1) < 1e-13
    assert abs(c - p1_closed_form(g, gamma, beta)) < 1e-12 * max(1.0, g.m)


def test_p1_single_edge_by_hand(oracle_lib):
    # Heisenberg-picture result for one edge: 1/2 + 1/2 sin(4 beta) sin(gamma)
    g = single_edge()
    for gamma, beta in [(0.4, 0.3), (1.3, 0.2), (-0.6, 0.9)]:
        c, _ = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, [gamma], [beta]))
        assert abs(c - (0.5 + 0.5 * math.sin(4 * beta) * math.sin(gamma))) < 1e-14


def test_published_p1_values(oracle_lib):
    # values of the closed form at gamma = 0.4, beta = 0.3, checked independently by brute force
    for g, ref in [(single_edge(), 0.68147655791211), (I.petersen(), 9.80934370049034),
                   (I.complete(4), 3.67763956976174)]:
        c, _ = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, [0.4], [0.3]))
        assert abs(c - ref) < 1e-11


# --------------------------------------------------------------------------- invariants

def test_gamma_beta_zero_gives_half_edges(oracle_lib):
    g = I.gnp(10, 0.5, 1)
    c, nrm = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, [0.0, 0.0], [0.0, 0.0]))
    assert abs(c - g.m / 2) < 1e-12 and abs(nrm - 1) < 1e-13


def test_gamma_zero_state(oracle_lib):
    g = I.gnp(9, 0.5, 2)
    betas = np.array([0.3, -0.8, 1.4])
    psi = oracle_lib.qaoa_state(g, np.zeros(3), betas)
    expect = np.exp(-1j * g.n * betas.sum()) * 2 ** (-g.n / 2)
    assert np.max(np.abs(psi - expect)) < 1e-13


def test_beta_zero_state(oracle_lib):
    g = I.gnp(9, 0.5, 3)
    gammas = np.array([0.3, 2.1, -0.4])
    psi = oracle_lib.qaoa_state(g, gammas, np.zeros(3))
    expect = 2 ** (-g.n / 2) * np.exp(-1j * gammas.sum() * brute_cut_values(g))
    assert np.max(np.abs(psi - expect)) < 1e-13


def test_complement_symmetry_and_bounds(oracle_lib):
    for seed in range(3):
        g = I.gnp(11, 0.45, seed)
        ga, be = I.angles(3, seed)
        psi = oracle_lib.qaoa_state(g, ga, be)
        z = np.arange(1 << g.n)
        assert np.max(np.abs(psi - psi[((1 << g.n) - 1) ^ z])) < 1e-13
        c, nrm = oracle_lib.expectation(g, psi)
        assert abs(nrm - 1) < 1e-12
        assert -1e-12 <= c <= oracle_lib.brute_maxcut(g) + 1e-12


def test_angle_sign_and_period_symmetry(oracle_lib):
    g = I.gnp(10, 0.5, 4)
    ga, be = I.angles(3, 4)
    c0, _ = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, ga, be))
    c1, _ = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, -ga, -be))
    c2, _ = oracle_lib.expectation(g, oracle_lib.qaoa_state(g, ga, be + math.pi / 2))
    assert abs(c0 - c1) < 1e-12 and abs(c0 - c2) < 1e-12


def test_brute_maxcut_known_values(oracle_lib):
    assert oracle_lib.brute_maxcut(I.petersen()) == 12
    assert oracle_lib.brute_maxcut(I.complete(5)) == 6
    assert oracle_lib.brute_maxcut(I.ring(7)) == 6
    assert oracle_lib.brute_maxcut(I.ring(8)) == 8


# --------------------------------------------------------------------------- adjoint gradient

@pytest.mark.parametrize("weighted", [False, True])
def test_adjoint_matches_central_differences(oracle_lib, weighted):
    g = I.gnp(8, 0.5, 5)
    if weighted:
        g = I.random_weights(g, 2)
    ga, be = I.angles(3, 5)
    c, dg, db = oracle_lib.adjoint_gradient(g, ga, be)
    h = 1e-5

    def f(gg, bb):
        return oracle_lib.expectation(g, oracle_lib.qaoa_state(g, gg, bb))[0]

    assert abs(c - f(ga, be)) < 1e-12
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd_g = (f(ga + e, be) - f(ga - e, be)) / (2 * h)
        fd_b = (f(ga, be + e) - f(ga, be - e)) / (2 * h)
        assert abs(fd_g - dg[k]) < 1e-7 * max(1, abs(fd_g))
        assert abs(fd_b - db[k]) < 1e-7 * max(1, abs(fd_b))


def test_adjoint_p1_single_edge_closed_form(oracle_lib):
    # d/dgamma and d/dbeta of 1/2 + 1/2 sin(4 beta) sin(gamma)
    g = single_edge()
    gamma, beta = 0.7, 0.2
    _, dg, db = oracle_lib.adjoint_gradient(g, [gamma], [beta])
    assert abs(dg[0] - 0.5 * math.sin(4 * beta) * math.cos(gamma)) < 1e-13
    assert abs(db[0] - 2.0 * math.cos(4 * beta) * math.sin(gamma)) < 1e-13
