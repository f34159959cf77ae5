/* opt_u.c -- the paper's optimised CPU simulation of p-level QAOA on an unweighted graph,
 * "Opt_u" of Section 3 (Table 2), written from its description as a timing baseline.  It is
 * neither the oracle nor the GPU path and shares no code with either.
 *
 * What it does, per the paper:
 *   - launch control (Section 2.2): the initial state is written as 2^(-N/2) everywhere instead
 *     of applying N Hadamard gates;
 *   - rotation compression (Eq. UC_opt, Algorithm 2): one pass over the 2^N amplitudes per cost
 *     layer, each multiplied by a single rotation exp(-i/2 gamma totRotation(b));
 *   - the unweighted count (Algorithm 3): totRotation = totEdge - 2 c_neg with
 *     c_neg = sum_i popcount(graph_I & (b_I xor b)), b_I = -(bit i of b) (all ones or zero),
 *     graph_I = row i of the upper-triangular adjacency matrix;
 *   - the mixer as in Algorithm 1: RX(beta) = exp(-i beta X / 2) on each qubit in turn;
 *   - thread-level parallelism (Section 2.4): OpenMP over the state loop of every layer.
 * Angles are in the paper's convention (gamma_paper, beta_paper).  The AVX variant (Opt_uAVX,
 * a lookup-table popcount for processors without one) is not reproduced: the hardware popcount
 * instruction is used. */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    double re, im;
} cplx;

static int build_rows(int n, int m, const int32_t *edges, uint64_t *row) {
    for (int i = 0; i < n; ++i) row[i] = 0;
    for (int e = 0; e < m; ++e) {
        int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return -1;
        if (u > v) {
            const int t = u;
            u = v;
            v = t;
        }
        row[u] |= 1ull << v;
    }
    return 0;
}

/* Algorithm 3: number of cut edges of basis state b. */
static inline int cut_edges(int n, const uint64_t *row, uint64_t b) {
    int c = 0;
    for (int i = 0; i < n; ++i) {
        const uint64_t bI = 0ull - ((b >> i) & 1ull);
        c += __builtin_popcountll(row[i] & (bI ^ b));
    }
    return c;
}

int optu_threads(void) { return omp_get_max_threads(); }
void optu_set_threads(int t) { omp_set_num_threads(t); }

/* p levels from launch control; psi receives 2^n interleaved (re, im) doubles. */
int optu_qaoa(int n, int m, const int32_t *edges, int p, const double *gamma_paper, const double *beta_paper,
              double *psi_out) {
    if (n < 1 || n > 34 || m < 0 || p < 0) return -1;
    uint64_t row[64];
    if (build_rows(n, m, edges, row)) return -1;
    const int64_t dim = (int64_t)1 << n;
    cplx *psi = (cplx *)psi_out;
    const double amp = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < dim; ++b) {
        psi[b].re = amp;
        psi[b].im = 0.0;
    }
    for (int k = 0; k < p; ++k) {
        const double g = gamma_paper[k];
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < dim; ++b) {
            const int cneg = cut_edges(n, row, (uint64_t)b);
            const int tot = (m - cneg) - cneg; /* c_pos - c_neg */
            const double a = -0.5 * g * (double)tot;
            const double c = cos(a), s = sin(a);
            const double re = psi[b].re, im = psi[b].im;
            psi[b].re = re * c - im * s;
            psi[b].im = re * s + im * c;
        }
        const double c = cos(0.5 * beta_paper[k]), s = sin(0.5 * beta_paper[k]);
        for (int q = 0; q < n; ++q) {
            const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < dim / 2; ++i) {
                const int64_t lo = i & (bit - 1);
                const int64_t z0 = ((i - lo) << 1) | lo, z1 = z0 | bit;
                const cplx a0 = psi[z0], a1 = psi[z1];
                /* [[c, -is], [-is, c]] */
                psi[z0].re = c * a0.re + s * a1.im;
                psi[z0].im = c * a0.im - s * a1.re;
                psi[z1].re = c * a1.re + s * a0.im;
                psi[z1].im = c * a1.im - s * a0.re;
            }
        }
    }
    return 0;
}

/* <C> = sum_b |psi_b|^2 (cut edges of b) and the norm. */
int optu_expectation(int n, int m, const int32_t *edges, const double *psi_in, double *out_c, double *out_norm) {
    uint64_t row[64];
    if (n < 1 || n > 34 || build_rows(n, m, edges, row)) return -1;
    const int64_t dim = (int64_t)1 << n;
    const cplx *psi = (const cplx *)psi_in;
    double sc = 0.0, sn = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sc, sn)
    for (int64_t b = 0; b < dim; ++b) {
        const double pr = psi[b].re * psi[b].re + psi[b].im * psi[b].im;
        sn += pr;
        sc += pr * (double)cut_edges(n, row, (uint64_t)b);
    }
    *out_c = sc;
    *out_norm = sn;
    return 0;
}
