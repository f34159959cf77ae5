/*
 * qaoa_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU simulator of QAOA for max-cut, used to check the
 * CUDA path.  Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * It follows the paper's "standard" simulation, Algorithm 1 (Section 2.1): start in
 * |0...0>, apply a Hadamard gate to every qubit (initial layer), then for each of the P
 * levels apply one RZZ rotation per edge (cost layer) and one RX rotation per qubit
 * (mixer layer).  Each RZZ is decomposed into the textbook CNOT - RZ - CNOT sequence.
 * Everything is complex128 (the paper does not state its precision).
 *
 * Readings of the paper used here (the paper's loop bounds and signs are ambiguous):
 *   - all loops in Algorithm 1 are 0-based and include qubit 0 and level 0: there are N
 *     Hadamard gates, N RX gates and one RZZ per edge in each of the P levels;
 *   - qubit u is bit u of the basis index z (Algorithm 3 extracts bit i as (b >> i) & 1);
 *   - cost layer of level k is exp(-i gamma_k C) with C(z) = sum over edges of
 *     w_uv * (z_u XOR z_v).  Per edge this is exp(+i gamma w Z_u Z_v / 2) (one CNOT - RZ -
 *     CNOT with RZ angle -gamma w) times the global phase exp(-i gamma w / 2).  The paper's
 *     Eq. (rewrite_UC) writes exp(-i gamma/2 sum w Z Z); its gamma is minus ours;
 *   - mixer of level k is RX(2 beta_k) = exp(-i beta_k X) on every qubit; the paper's
 *     RXGate angle is 2 beta_k;
 *   - the output is <C> = sum_z |psi_z|^2 C(z) with C from a plain loop over the edges.
 *
 * Weighted graphs (Algorithm 2) are supported through the edge weights; weights == NULL
 * means unit weights (Algorithm 3's setting).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2

/* ------------------------------------------------------------------ graph checks */

static int check_graph(int n, int m, const int32_t *edges)
{
    if (n < 1 || n > 40 || m < 0) return ORACLE_EINVAL;
    for (int e = 0; e < m; ++e) {
        int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return ORACLE_EINVAL;
    }
    return ORACLE_OK;
}

static double edge_weight(const double *w, int e) { return w ? w[e] : 1.0; }

/* Edges in the order Algorithm 1 visits them: i ascending, then j ascending, i < j. */
static int *sorted_edge_order(int m, const int32_t *edges)
{
    int *ord = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
    if (!ord) return NULL;
    for (int e = 0; e < m; ++e) ord[e] = e;
    /* insertion sort: m is at most a few hundred */
    for (int a = 1; a < m; ++a) {
        int x = ord[a];
        int xu = edges[2 * x] < edges[2 * x + 1] ? edges[2 * x] : edges[2 * x + 1];
        int xv = edges[2 * x] < edges[2 * x + 1] ? edges[2 * x + 1] : edges[2 * x];
        int b = a - 1;
        while (b >= 0) {
            int y = ord[b];
            int yu = edges[2 * y] < edges[2 * y + 1] ? edges[2 * y] : edges[2 * y + 1];
            int yv = edges[2 * y] < edges[2 * y + 1] ? edges[2 * y + 1] : edges[2 * y];
            if (yu < xu || (yu == xu && yv <= xv)) break;
            ord[b + 1] = y;
            --b;
        }
        ord[b + 1] = x;
    }
    return ord;
}

/* ------------------------------------------------------------------ cut values */

/* C(z) = sum over edges of w_uv * (bit u of z XOR bit v of z): the plain definition. */
double oracle_cut_value(int n, int m, const int32_t *edges, const double *w, uint64_t z)
{
    (void)n;
    double c = 0.0;
    for (int e = 0; e < m; ++e) {
        uint64_t bu = (z >> edges[2 * e]) & 1u, bv = (z >> edges[2 * e + 1]) & 1u;
        if (bu ^ bv) c += edge_weight(w, e);
    }
    return c;
}

/* Unweighted cut count of every basis state, by the same edge loop. */
int oracle_cut_table(int n, int m, const int32_t *edges, uint16_t *out)
{
    if (check_graph(n, m, edges) != ORACLE_OK || n > 30) return ORACLE_EINVAL;
    const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)dim; ++z) {
        int c = 0;
        for (int e = 0; e < m; ++e)
            c += (int)(((uint64_t)z >> edges[2 * e] ^ (uint64_t)z >> edges[2 * e + 1]) & 1u);
        out[z] = (uint16_t)c;
    }
    return ORACLE_OK;
}

/* Algorithm 3, one step (Section 2.3): b_I is bit i of b replicated into every bit, written
 * as the two's-complement negation of that bit; the term is popcount(graph_I AND (b_I XOR b)). */
static int popcount64(uint64_t x)
{
    int c = 0;
    while (x) {
        x &= x - 1;
        ++c;
    }
    return c;
}

int oracle_alg3_term(uint64_t b, uint64_t graph_row, int i)
{
    uint64_t bI = (uint64_t)0 - ((b >> i) & 1u);
    return popcount64(graph_row & (bI ^ b));
}

/* Algorithm 3: c_neg = number of cut edges, with graph_I[i] holding bit j iff edge (i, j),
 * j > i (row i of the upper-triangular adjacency matrix, Table 1).  Also returns
 * totRotation = totEdge - 2 c_neg through *tot_rotation when non-NULL. */
int oracle_alg3_cut(int n, const uint64_t *graph_I, int tot_edge, uint64_t b, int *tot_rotation)
{
    int c_neg = 0;
    for (int i = 0; i < n; ++i) c_neg += oracle_alg3_term(b, graph_I[i], i);
    if (tot_rotation) *tot_rotation = (tot_edge - c_neg) - c_neg;
    return c_neg;
}

/* Algorithm 2's totRotation for one basis state: sum of -w over cut edges and +w over
 * uncut edges, visiting the upper-triangular weight matrix row by row. */
double oracle_alg2_tot_rotation(int n, int m, const int32_t *edges, const double *w, uint64_t b)
{
    (void)n;
    double tot = 0.0;
    for (int e = 0; e < m; ++e) {
        uint64_t bi = (b >> edges[2 * e]) & 1u, bj = (b >> edges[2 * e + 1]) & 1u;
        if ((bi ^ bj) == 1u)
            tot -= edge_weight(w, e);
        else
            tot += edge_weight(w, e);
    }
    return tot;
}

/* ------------------------------------------------------------------ gates */

static void gate_h(zc *psi, int n, int q)
{
    const int64_t half = (int64_t)1 << (n - 1);
    const double r = 1.0 / sqrt(2.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < half; ++i) {
        uint64_t lo = (uint64_t)i & ((1ull << q) - 1);
        uint64_t a = (((uint64_t)i >> q) << (q + 1)) | lo;
        uint64_t b = a | (1ull << q);
        zc x = psi[a], y = psi[b];
        psi[a] = r * (x + y);
        psi[b] = r * (x - y);
    }
}

static void gate_cnot(zc *psi, int n, int ctl, int tgt)
{
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < dim; ++z) {
        if ((((uint64_t)z >> ctl) & 1u) && !(((uint64_t)z >> tgt) & 1u)) {
            uint64_t y = (uint64_t)z | (1ull << tgt);
            zc t = psi[z];
            psi[z] = psi[y];
            psi[y] = t;
        }
    }
}

/* RZ(theta) = diag(exp(-i theta/2), exp(+i theta/2)) on qubit q. */
static void gate_rz(zc *psi, int n, int q, double theta)
{
    const int64_t dim = (int64_t)1 << n;
    const zc f0 = cexp(-I * theta / 2.0), f1 = cexp(I * theta / 2.0);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < dim; ++z) psi[z] *= (((uint64_t)z >> q) & 1u) ? f1 : f0;
}

/* RX(theta) = [[cos(theta/2), -i sin(theta/2)], [-i sin(theta/2), cos(theta/2)]] on qubit q. */
static void gate_rx(zc *psi, int n, int q, double theta)
{
    const int64_t half = (int64_t)1 << (n - 1);
    const double c = cos(theta / 2.0), s = sin(theta / 2.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < half; ++i) {
        uint64_t lo = (uint64_t)i & ((1ull << q) - 1);
        uint64_t a = (((uint64_t)i >> q) << (q + 1)) | lo;
        uint64_t b = a | (1ull << q);
        zc x = psi[a], y = psi[b];
        psi[a] = c * x - I * s * y;
        psi[b] = -I * s * x + c * y;
    }
}

static void global_phase(zc *psi, int n, zc f)
{
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < dim; ++z) psi[z] *= f;
}

/* ------------------------------------------------------------------ layers */

/* Initial layer: |0...0> followed by one Hadamard per qubit. */
void oracle_initial_layer(int n, zc *psi)
{
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(zc) * (size_t)dim);
    psi[0] = 1.0;
    for (int q = 0; q < n; ++q) gate_h(psi, n, q);
}

/* Cost layer of one level: per edge (in Algorithm 1's order) CNOT(u->v), RZ_v(-gamma w),
 * CNOT(u->v), then the global phase exp(-i gamma W / 2), W = sum of weights.  Together:
 * exp(-i gamma C). */
int oracle_cost_layer(int n, int m, const int32_t *edges, const double *w, double gamma, zc *psi)
{
    if (check_graph(n, m, edges) != ORACLE_OK) return ORACLE_EINVAL;
    int *ord = sorted_edge_order(m, edges);
    if (!ord) return ORACLE_ENOMEM;
    double wsum = 0.0;
    for (int a = 0; a < m; ++a) {
        int e = ord[a];
        int u = edges[2 * e] < edges[2 * e + 1] ? edges[2 * e] : edges[2 * e + 1];
        int v = edges[2 * e] < edges[2 * e + 1] ? edges[2 * e + 1] : edges[2 * e];
        double we = edge_weight(w, e);
        gate_cnot(psi, n, u, v);
        gate_rz(psi, n, v, -gamma * we);
        gate_cnot(psi, n, u, v);
        wsum += we;
    }
    global_phase(psi, n, cexp(-I * gamma * wsum / 2.0));
    free(ord);
    return ORACLE_OK;
}

/* Mixer layer of one level: RX(2 beta) on every qubit. */
void oracle_mixer_layer(int n, double beta, zc *psi)
{
    for (int q = 0; q < n; ++q) gate_rx(psi, n, q, 2.0 * beta);
}

/* Algorithm 1: initial layer, then P levels of {cost layer, mixer layer}. */
int oracle_qaoa(int n, int m, const int32_t *edges, const double *w, int p, const double *gamma,
                const double *beta, zc *psi)
{
    if (check_graph(n, m, edges) != ORACLE_OK || p < 0) return ORACLE_EINVAL;
    oracle_initial_layer(n, psi);
    for (int k = 0; k < p; ++k) {
        int rc = oracle_cost_layer(n, m, edges, w, gamma[k], psi);
        if (rc) return rc;
        oracle_mixer_layer(n, beta[k], psi);
    }
    return ORACLE_OK;
}

/* <C> = sum_z |psi_z|^2 C(z) and the squared norm, with C from the plain edge loop. */
int oracle_expectation(int n, int m, const int32_t *edges, const double *w, const zc *psi,
                       double *out_c, double *out_norm)
{
    if (check_graph(n, m, edges) != ORACLE_OK) return ORACLE_EINVAL;
    const int64_t dim = (int64_t)1 << n;
    double sc = 0.0, sn = 0.0;
#pragma omp parallel for reduction(+ : sc, sn) schedule(static)
    for (int64_t z = 0; z < dim; ++z) {
        double pz = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
        sc += pz * oracle_cut_value(n, m, edges, w, (uint64_t)z);
        sn += pz;
    }
    *out_c = sc;
    *out_norm = sn;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ adjoint gradient */

/* Im <a| B |b> with B = sum_j X_j. */
static double im_braket_B(int n, const zc *a, const zc *b)
{
    const int64_t dim = (int64_t)1 << n;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
#pragma omp parallel for reduction(+ : s) schedule(static)
        for (int64_t z = 0; z < dim; ++z) s += cimag(conj(a[z]) * b[(uint64_t)z ^ (1ull << j)]);
    }
    return s;
}

/* Im <a| C |b> with C the diagonal cut operator. */
static double im_braket_C(int n, int m, const int32_t *edges, const double *w, const zc *a,
                          const zc *b)
{
    const int64_t dim = (int64_t)1 << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t z = 0; z < dim; ++z)
        s += oracle_cut_value(n, m, edges, w, (uint64_t)z) * cimag(conj(a[z]) * b[z]);
    return s;
}

/* FP64 adjoint: <C> and d<C>/d gamma_k, d<C>/d beta_k for the circuit of oracle_qaoa.
 * With psi_k the state after level k and lambda_k = (U_p ... U_{k+1})^dagger C psi_p:
 *   d/d beta_k  = 2 Im <lambda_k| B |psi_k>,
 *   d/d gamma_k = 2 Im <M_k^dagger lambda_k| C |M_k^dagger psi_k>,
 * and both vectors are uncomputed one level at a time with the inverse gates. */
int oracle_adjoint_gradient(int n, int m, const int32_t *edges, const double *w, int p,
                            const double *gamma, const double *beta, double *out_c,
                            double *d_gamma, double *d_beta)
{
    if (check_graph(n, m, edges) != ORACLE_OK || p < 0) return ORACLE_EINVAL;
    const int64_t dim = (int64_t)1 << n;
    zc *psi = (zc *)malloc(sizeof(zc) * (size_t)dim);
    zc *lam = (zc *)malloc(sizeof(zc) * (size_t)dim);
    if (!psi || !lam) {
        free(psi);
        free(lam);
        return ORACLE_ENOMEM;
    }
    int rc = oracle_qaoa(n, m, edges, w, p, gamma, beta, psi);
    if (rc) goto done;
    double norm;
    oracle_expectation(n, m, edges, w, psi, out_c, &norm);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < dim; ++z) lam[z] = oracle_cut_value(n, m, edges, w, (uint64_t)z) * psi[z];
    for (int k = p - 1; k >= 0; --k) {
        d_beta[k] = 2.0 * im_braket_B(n, lam, psi);
        oracle_mixer_layer(n, -beta[k], psi);
        oracle_mixer_layer(n, -beta[k], lam);
        d_gamma[k] = 2.0 * im_braket_C(n, m, edges, w, lam, psi);
        oracle_cost_layer(n, m, edges, w, -gamma[k], psi);
        oracle_cost_layer(n, m, edges, w, -gamma[k], lam);
    }
done:
    free(psi);
    free(lam);
    return rc;
}

/* ------------------------------------------------------------------ misc */

/* Brute-force maximum cut (n small). */
double oracle_brute_maxcut(int n, int m, const int32_t *edges, const double *w)
{
    double best = 0.0;
    for (uint64_t z = 0; z < (1ull << n); ++z) {
        double c = oracle_cut_value(n, m, edges, w, z);
        if (c > best) best = c;
    }
    return best;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
