/* Host-side check of the oracle (oracle/qaoa_oracle.c), built with AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_host_sanitizers.py: every entry point runs on small
 * graphs (unit and signed weights, n = 2..10, p = 0..3), with consistency checks between them
 * (norm 1, 0 <= <C> <= the brute-force maximum cut, Algorithm 2's totRotation = W - 2 C and
 * Algorithm 3's popcount cut against the plain edge loop for every z).  Any out-of-bounds access
 * or undefined behaviour stops the run with a report. */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef double complex zc;

double oracle_cut_value(int n, int m, const int32_t *edges, const double *w, uint64_t z);
int oracle_cut_table(int n, int m, const int32_t *edges, uint16_t *out);
int oracle_alg3_cut(int n, const uint64_t *graph_I, int tot_edge, uint64_t b, int *tot_rotation);
double oracle_alg2_tot_rotation(int n, int m, const int32_t *edges, const double *w, uint64_t b);
int oracle_qaoa(int n, int m, const int32_t *edges, const double *w, int p, const double *gamma,
                const double *beta, zc *psi);
int oracle_expectation(int n, int m, const int32_t *edges, const double *w, const zc *psi,
                       double *out_c, double *out_norm);
int oracle_adjoint_gradient(int n, int m, const int32_t *edges, const double *w, int p,
                            const double *gamma, const double *beta, double *out_c,
                            double *d_gamma, double *d_beta);
double oracle_brute_maxcut(int n, int m, const int32_t *edges, const double *w);

static int fails = 0;
#define CHECK(c)                                                                   \
    do {                                                                           \
        if (!(c)) {                                                                \
            fprintf(stderr, "check failed: %s (n=%d m=%d)\n", #c, n, m);           \
            ++fails;                                                               \
        }                                                                          \
    } while (0)

static uint64_t lcg = 12345;
static double u01(void)
{
    lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg >> 11) * 0x1p-53;
}

static void run_graph(int n, int m, const int32_t *edges, const double *w)
{
    const double gamma[3] = {0.4, 1.3, -0.7}, beta[3] = {0.3, 1.1, 2.0};
    const uint64_t dim = 1ull << n;
    zc *psi = malloc(dim * sizeof(zc));
    uint16_t *tab = malloc(dim * sizeof(uint16_t));
    double tot_w = 0.0;
    for (int e = 0; e < m; ++e) tot_w += w ? w[e] : 1.0;
    const double maxcut = oracle_brute_maxcut(n, m, edges, w);
    for (int p = 0; p <= 3; ++p) {
        double c = 0.0, nrm = 0.0, c2 = 0.0, dg[3], db[3];
        CHECK(oracle_qaoa(n, m, edges, w, p, gamma, beta, psi) == 0);
        CHECK(oracle_expectation(n, m, edges, w, psi, &c, &nrm) == 0);
        CHECK(fabs(nrm - 1.0) < 1e-12);
        if (!w) CHECK(c >= -1e-12 && c <= maxcut + 1e-9);
        if (p > 0) {
            CHECK(oracle_adjoint_gradient(n, m, edges, w, p, gamma, beta, &c2, dg, db) == 0);
            CHECK(fabs(c2 - c) < 1e-10 * (1.0 + fabs(c)));
        }
    }
    if (!w) {
        CHECK(oracle_cut_table(n, m, edges, tab) == 0);
        uint64_t rows[64] = {0};
        for (int e = 0; e < m; ++e) {
            const int u = edges[2 * e] < edges[2 * e + 1] ? edges[2 * e] : edges[2 * e + 1];
            const int v = edges[2 * e] ^ edges[2 * e + 1] ^ u;
            rows[u] |= 1ull << v;
        }
        for (uint64_t z = 0; z < dim; ++z) {
            int tot_rot = 0;
            const int c3 = oracle_alg3_cut(n, rows, m, z, &tot_rot);
            CHECK(c3 == (int)tab[z]);
            CHECK(fabs(oracle_cut_value(n, m, edges, NULL, z) - tab[z]) == 0.0);
        }
    }
    for (uint64_t z = 0; z < dim; z += 1 + dim / 64)
        CHECK(fabs(oracle_alg2_tot_rotation(n, m, edges, w, z) -
                   (tot_w - 2.0 * oracle_cut_value(n, m, edges, w, z))) < 1e-9 * (1.0 + fabs(tot_w)));
    free(tab);
    free(psi);
}

int main(void)
{
    int32_t edges[2 * 45];
    double w[45];
    int graphs = 0;
    for (int n = 2; n <= 10; ++n) {
        for (int kind = 0; kind < 3; ++kind) {
            int m = 0;
            for (int u = 0; u < n; ++u)
                for (int v = u + 1; v < n; ++v) {
                    const int take = kind == 0 ? (v == u + 1) : kind == 1 ? 1 : (u01() < 0.4);
                    if (take) {
                        edges[2 * m] = u;
                        edges[2 * m + 1] = v;
                        w[m] = -1.0 + 3.0 * u01();
                        ++m;
                    }
                }
            run_graph(n, m, edges, NULL);
            run_graph(n, m, edges, w);
            graphs += 2;
        }
    }
    {
        const int n = 3, m = 1;
        const int32_t loop[2] = {1, 1};
        double c = 0.0, nrm = 0.0;
        zc psi[8];
        CHECK(oracle_qaoa(n, m, loop, NULL, 1, (const double[]){0.1}, (const double[]){0.2}, psi) != 0);
        CHECK(oracle_expectation(n, m, loop, NULL, psi, &c, &nrm) != 0);
    }
    printf("%d graphs checked, %d failures\n", graphs, fails);
    return fails == 0 ? 0 : 1;
}
